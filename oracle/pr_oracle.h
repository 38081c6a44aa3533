/*
 * Plain CPU FP64 oracle for the kinetic-fluid parareal method of Laidin & Rey
 * (arXiv 2502.02704).  TEST INFRASTRUCTURE ONLY: it is used by tests/, by
 * __graft_entry__.smoke() and by bench.py's cpu_baseline / reference leg.  The
 * product path (the CUDA library) never links, loads or calls it, and it shares
 * no code, header or constant with that path.
 *
 * Everything is double precision, naive loops, in the order the paper states
 * the scheme.  Readings of garbled or silent passages are listed with each
 * function.  Conventions:
 *   primitive  U = (rho, u_x, u_y, u_z, theta)   stored [5][nx]
 *   conserved  V = (rho, rho u_x, rho u_y, rho u_z, E), E = rho|u|^2/2 + 3 rho theta/2
 *   f[i][j], i = 0..nx-1 (x cell), j = (jx*nv + jy)*nv + jz (velocity cell)
 */
#ifndef PR_ORACLE_H
#define PR_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

/* Compensated summation (Neumaier 1974, the improved Kahan-Babuska sum) for the
 * velocity sums of Eq. (18).  The moments are defined as exact sums over the
 * nv^3 cells; a plain running sum of that many terms drifts by ~sqrt(n) ulps
 * (about 1e-14 relative at 24^3), while s + c below is the exact sum of the
 * terms to within a couple of ulps in any order.  Each addition's rounding
 * error is recovered exactly (Knuth's two-sum, ordered by magnitude). */
typedef struct {
    double s, c;
} or_csum;

static inline void or_cadd(or_csum* a, double x)
{
    double t = a->s + x;
    if ((a->s < 0 ? -a->s : a->s) >= (x < 0 ? -x : x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

static inline double or_cval(const or_csum* a) { return a->s + a->c; }

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2
#define OR_ENONPHYS -5

#define OR_BC_PERIODIC 0
#define OR_BC_OUTFLOW 1
#define OR_BC_REFLECT 2

#define OR_UPWIND 0
#define OR_MUSCL 1

#define OR_SOUND_GAMMA53 0
#define OR_SOUND_SQRT_THETA 1

#define OR_COARSE_EULER 0  /* Eqs. (14)-(16)                                   */
#define OR_COARSE_CNS 1    /* Eq. (8), viscous terms of reading R22            */

typedef struct {
    int nx;        /* x cells on [x0, x1]                                  */
    double x0, x1;
    int bc;        /* OR_BC_*                                              */
    int nv;        /* velocity cells per direction on [-L, L]^3            */
    double L;
    double eps;    /* Knudsen number; +inf means collisionless (no BGK)    */
    int scheme;    /* OR_UPWIND or OR_MUSCL                                */
} or_kin;

typedef struct {
    or_kin kin;
    double T;      /* final time                                           */
    int N;         /* number of coarse slices N_g                          */
    double cfl_f;  /* fine CFL (x transport)                               */
    double cfl_g;  /* coarse CFL (Rusanov)                                 */
    int sound;     /* OR_SOUND_*                                           */
    int nf;        /* fine steps per slice; <= 0: derived from cfl_f       */
    int coarse;    /* OR_COARSE_EULER or OR_COARSE_CNS                     */
    int lift;      /* lifting order: 0 (Def. 2) or 1 (Def. 3, L = 1)       */
} or_pr;

void or_set_threads(int n);
int or_get_threads(void);

void or_velocity_nodes(int nv, double L, double* v);
void or_prim_to_cons(int nx, const double* U, double* V);
int or_cons_to_prim(int nx, const double* V, double* U);

int or_lift(const or_kin* k, const double* U, double* f);
int or_project(const or_kin* k, const double* f, double* U);
int or_project_cons(const or_kin* k, const double* f, double* V);

double or_fine_dt_stab(const or_kin* k, double cfl);
int or_fine_nsteps(const or_pr* p, double* dt_out);
int or_fine_step(const or_kin* k, double dt, const double* f, double* fout);
int or_fine_run(const or_kin* k, double dt, int nsteps, double* f);

int or_coarse_run(int nx, double x0, double x1, int bc, double cfl, int sound,
                  double dT, const double* Vin, double* Vout, int* nsub);
/* The compressible Navier-Stokes coarse model of Eq. (8) (reading R22) with
 * Knudsen number eps > 0 and an optional exterior force E [nx]. */
int or_coarse_run_cns(int nx, double x0, double x1, int bc, double cfl, int sound, double dT, double eps,
                      const double* E, const double* Vin, double* Vout, int* nsub);
/* First-order lifting L^(1) of Def. 3 (reading R23). */
int or_lift_ce(const or_kin* k, const double* U, double* f);
void or_prim_gradients(int nx, int bc, double dx, const double* U, int i, double* d);
void or_ce_column(const double* vx, int nvx, const double* vp, int nvp, const double* U5, const double* d,
                  double eps, double* fc);

int or_fine_propagate(const or_pr* p, const double* Vin, double* Vout);
int or_coarse_propagate(const or_pr* p, const double* Vin, double* Vout);

int or_parareal(const or_pr* p, const double* U0, int K, double tol, int alg,
                double* Uall, double* errs, int* k_done);

/* A propagator V(T^{n-1}) -> V(T^n) on conserved [5][nx] states. */
typedef int (*or_prop)(const void* ctx, const double* Vin, double* Vout);

/* The loop of Algorithms 1 and 2 over the propagators fine (P F L) and coarse (G);
 * same conventions as or_parareal. */
int or_parareal_core(int nx, int N, or_prop fine, or_prop coarse, const void* ctx, const double* U0,
                     int K, double tol, int alg, double* Uall, double* errs, int* k_done);

/* ---------------- exterior force E != 0 (pr_oracle_force.c) ----------------
 * Eq. (11) with the force term E . grad_v f, the velocity flux G of Eq. (13)
 * along v_x, and the Euler source of Eq. (5).  The velocity grid is
 * anisotropic (Test 3): nvx cells along v_x and nvp along each of v_y, v_z,
 * all on [-L, L].  f[i][j] with j = (jx*nvp + jy)*nvp + jz. */
typedef struct {
    int nx;
    double x0, x1;
    int bc;
    int nvx;          /* velocity cells along v_x                              */
    int nvp;          /* velocity cells along each of v_y and v_z              */
    double L;
    double eps;       /* Knudsen number; +inf means collisionless              */
    int scheme;       /* x transport: OR_UPWIND or OR_MUSCL                    */
    const double* E;  /* [nx] exterior force at the cell centres; NULL: E = 0  */
} or_vkin;

typedef struct {
    or_vkin kin;
    double T;
    int N;
    double cfl_f, cfl_g;
    int sound;
    int nf;
    int coarse;       /* OR_COARSE_EULER or OR_COARSE_CNS                   */
    int lift;         /* lifting order 0 or 1                               */
} or_vpr;

int or_coarse_run_force(int nx, double x0, double x1, int bc, double cfl, int sound,
                        double dT, const double* E, const double* Vin, double* Vout, int* nsub);
int or_v_lift(const or_vkin* k, const double* U, double* f);
int or_v_lift_ce(const or_vkin* k, const double* U, double* f);
int or_v_project(const or_vkin* k, const double* f, double* U);
int or_v_project_cons(const or_vkin* k, const double* f, double* V);
double or_v_fine_dt_stab(const or_vkin* k, double cfl);
int or_v_fine_nsteps(const or_vpr* p, double* dt_out);
int or_v_fine_step(const or_vkin* k, double dt, const double* f, double* fout);
int or_v_fine_run(const or_vkin* k, double dt, int nsteps, double* f);
int or_v_fine_propagate(const or_vpr* p, const double* Vin, double* Vout);
int or_v_coarse_propagate(const or_vpr* p, const double* Vin, double* Vout);
int or_v_parareal(const or_vpr* p, const double* U0, int K, double tol, int alg,
                  double* Uall, double* errs, int* k_done);

/* Gradient of J(V(T)) w.r.t. the primitive initial state U0 [5][nx] and log eps,
 * given lamV = dJ/dV(T) [5][nx] (conserved final moments); upwind scheme. */
int or_adjoint(const or_kin* k, double dt, int nsteps, const double* U0, const double* lamV,
               double* dU0, double* dlogeps);

#ifdef __cplusplus
}
#endif
#endif
