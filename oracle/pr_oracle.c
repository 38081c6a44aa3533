/*
 * Plain CPU FP64 oracle for the kinetic-fluid parareal method of Laidin & Rey
 * (arXiv 2502.02704).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference leg may load this.  The CUDA library never links or
 * calls it and the two share no code.
 *
 * What is followed, function by function:
 *   velocity grid           Sec. 3 (finite-volume cells K_ij, uniform cubes on [-L,L]^3),
 *                           nodes at the cube centres
 *   or_lift                 Def. 2 and the discrete lifting, Eq. (17)
 *   or_project              Def. 1 and the discrete projection, Eq. (18)
 *   or_fine_step            the IMEX scheme, Eqs. (11)-(13): explicit x-transport with
 *                           the upwind flux (flux limiter of Sec. 3.1 as MUSCL-minmod),
 *                           moments of the transported f (explicit by conservation),
 *                           implicit BGK relaxation of Eq. (7)
 *   or_coarse_run           Euler system Eq. (14), explicit update Eq. (15) with the
 *                           Rusanov flux Eq. (16), CFL-limited local steps (Sec. 2.2)
 *   or_parareal             Algorithm 1 (alg=1) and Algorithm 2 (alg=2), stopping
 *                           error of Eq. (10)
 *
 * Readings of garbled or silent passages (each also noted where it is used):
 *   R1  upwind flux sign: F_{i+1/2} = v^+ f_i - v^- f_{i+1} with v^- = -min(v,0) >= 0
 *       (Eq. 13 prints a plus sign, which would not be upwind).
 *   R2  the missing 1/dx in Eq. (12) and dt/dx in Eq. (15) are inserted.
 *   R3  tau = 1: the relaxation rate is 1/eps (Eq. 7 leaves tau unspecified).
 *   R4  Rusanov flux: (h(V_i)+h(V_{i+1}))/2 - S (V_{i+1}-V_i)/2 on conserved V
 *       (Eq. 16 prints a difference of h and U in place of V).
 *   R5  sound speed: sqrt(5 theta/3) (gamma = 5/3 of the monoatomic Euler system,
 *       Eq. 5) by default; the printed sqrt(theta) is selectable.
 *   R6  parareal state corrected and stored in conserved variables.
 *   R7  error = max over slices, cells and the 5 conserved components of |dV|.
 *   R8  parareal correction in the standard form of the ODE statement in Sec. 1:
 *       U^{n,k} = G(U^{n-1,k}) + PFL(U^{n-1,k-1}) - G(U^{n-1,k-1}); at iteration k
 *       Algorithm 2 recomputes only the slices n >= k.
 *   R9  fine steps per slice: n_f = ceil(dT_g / dt_stab), dt_stab = cfl dx / max|v_x|,
 *       uniform dt = dT_g / n_f inside the slice.
 *   R10 MUSCL: minmod slopes, forward Euler in time.
 *   R11 boundary ghosts: periodic wrap; outflow (the paper's "absorbing") copies the
 *       boundary cell; reflecting mirrors the cell and reverses v_x.
 *   R12 a non-positive density or temperature is an error (no clamping).
 *
 * Higher-order coupling (Eq. 8, Remark 1 / Def. 3 with L = 1), not run by the
 * paper; readings:
 *   R22 compressible Navier-Stokes coarse model of Eq. (8) for BGK with tau = 1:
 *       mu = rho theta, kappa = 5 rho theta / 2 (the first-order Chapman-Enskog
 *       moments of the BGK model, Prandtl number 1).  1-D in x: the viscous flux
 *       of (rho u, E) is -eps (mu (4/3) du_x, mu du_y, mu du_z) and
 *       -eps (mu (4/3) u_x du_x + mu u_y du_y + mu u_z du_z + kappa dtheta), with
 *       the gradients (V_{i+1} - V_i)/dx and mu, kappa, u averaged over the two
 *       cells of the face, added to the Rusanov flux; local steps
 *       dt = cfl min(dx / max S, dx^2 / (2 eps (5/3) max theta)).
 *   R23 first-order lifting f = M + eps g1, g1 = -(d_t + v d_x) M with the Euler
 *       time derivatives: g1 = -M [ (c_x (c . du) - |c|^2 du_x / 3) / theta
 *       + c_x (|c|^2 / (2 theta) - 5/2) dtheta / theta ], c = v - u; the
 *       gradients of u and theta by central differences through the ghosts.
 *       An exterior force cancels in g1 (its terms in d_t M and E d_v M are
 *       opposite), so the force path lifts with the same formula.
 */
#include "pr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

void or_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int or_get_threads(void) { return g_threads; }

/* Velocity cell centres on [-L, L] with nv uniform cells (Sec. 3, cubes V_j). */
void or_velocity_nodes(int nv, double L, double* v)
{
    double dv = 2.0 * L / nv;
    for (int j = 0; j < nv; ++j) v[j] = -L + (j + 0.5) * dv;
}

/* Conserved variables of the Euler system, Eq. (14): V = (rho, rho u, E),
 * E = rho |u|^2 / 2 + 3 rho theta / 2 (Eq. 5 with d_v = 3). */
void or_prim_to_cons(int nx, const double* U, double* V)
{
    for (int i = 0; i < nx; ++i) {
        double rho = U[0 * nx + i], ux = U[1 * nx + i], uy = U[2 * nx + i];
        double uz = U[3 * nx + i], th = U[4 * nx + i];
        V[0 * nx + i] = rho;
        V[1 * nx + i] = rho * ux;
        V[2 * nx + i] = rho * uy;
        V[3 * nx + i] = rho * uz;
        V[4 * nx + i] = 0.5 * rho * (ux * ux + uy * uy + uz * uz) + 1.5 * rho * th;
    }
}

int or_cons_to_prim(int nx, const double* V, double* U)
{
    int bad = 0;
    for (int i = 0; i < nx; ++i) {
        double rho = V[0 * nx + i];
        double ux = V[1 * nx + i] / rho, uy = V[2 * nx + i] / rho, uz = V[3 * nx + i] / rho;
        double th = (2.0 * V[4 * nx + i] / rho - (ux * ux + uy * uy + uz * uz)) / 3.0;
        if (!(rho > 0.0) || !(th > 0.0)) bad = 1;
        U[0 * nx + i] = rho;
        U[1 * nx + i] = ux;
        U[2 * nx + i] = uy;
        U[3 * nx + i] = uz;
        U[4 * nx + i] = th;
    }
    return bad ? OR_ENONPHYS : OR_OK;
}

static int check_kin(const or_kin* k)
{
    if (!k || k->nx < 1 || k->nv < 1 || !(k->L > 0.0) || !(k->x1 > k->x0)) return OR_EINVAL;
    if (k->bc < 0 || k->bc > 2 || k->scheme < 0 || k->scheme > 1) return OR_EINVAL;
    if (!(k->eps > 0.0)) return OR_EINVAL;
    /* MUSCL needs two ghost cells; a reflecting wall can only mirror them
     * from two interior cells. */
    if (k->scheme == OR_MUSCL && k->bc == OR_BC_REFLECT && k->nx < 2) return OR_EINVAL;
    return OR_OK;
}

/* Discrete lifting, Eq. (17): pointwise Maxwellian of Eq. (4) at the velocity
 * nodes, evaluated directly with exp (no factorisation). */
int or_lift(const or_kin* k, const double* U, double* f)
{
    int rc = check_kin(k);
    if (rc) return rc;
    int nx = k->nx, nv = k->nv;
    long nv3 = (long)nv * nv * nv;
    double* v = malloc(sizeof(double) * nv);
    if (!v) return OR_ENOMEM;
    or_velocity_nodes(nv, k->L, v);
    const double pi = 3.14159265358979323846;
    int bad = 0;
    for (int i = 0; i < nx; ++i) {
        double rho = U[0 * nx + i], ux = U[1 * nx + i], uy = U[2 * nx + i];
        double uz = U[3 * nx + i], th = U[4 * nx + i];
        if (!(rho > 0.0) || !(th > 0.0)) bad = 1;
        double pref = rho / pow(2.0 * pi * th, 1.5);
        for (int jx = 0; jx < nv; ++jx)
            for (int jy = 0; jy < nv; ++jy)
                for (int jz = 0; jz < nv; ++jz) {
                    double cx = v[jx] - ux, cy = v[jy] - uy, cz = v[jz] - uz;
                    double c2 = cx * cx + cy * cy + cz * cz;
                    f[(long)i * nv3 + ((long)jx * nv + jy) * nv + jz] = pref * exp(-c2 / (2.0 * th));
                }
    }
    free(v);
    return bad ? OR_ENONPHYS : OR_OK;
}

/* Moments of one x column by the first-order quadrature of Eq. (18), the
 * terms taken in lexicographic (jx, jy, jz) order and summed with
 * compensation (or_cadd): rho = sum f dv^3, rho u = sum v f dv^3,
 * 3 rho theta = sum |v - u|^2 f dv^3 (two passes: u first, then theta). */
static void column_moments(int nv, const double* v, double dv3, const double* fc,
                           double* rho, double* u, double* th)
{
    or_csum s0 = {0, 0}, sx = {0, 0}, sy = {0, 0}, sz = {0, 0};
    for (int jx = 0; jx < nv; ++jx)
        for (int jy = 0; jy < nv; ++jy)
            for (int jz = 0; jz < nv; ++jz) {
                double fv = fc[((long)jx * nv + jy) * nv + jz];
                or_cadd(&s0, fv * dv3);
                or_cadd(&sx, v[jx] * fv * dv3);
                or_cadd(&sy, v[jy] * fv * dv3);
                or_cadd(&sz, v[jz] * fv * dv3);
            }
    double r = or_cval(&s0);
    double ux = or_cval(&sx) / r, uy = or_cval(&sy) / r, uz = or_cval(&sz) / r;
    or_csum s2 = {0, 0};
    for (int jx = 0; jx < nv; ++jx)
        for (int jy = 0; jy < nv; ++jy)
            for (int jz = 0; jz < nv; ++jz) {
                double fv = fc[((long)jx * nv + jy) * nv + jz];
                double cx = v[jx] - ux, cy = v[jy] - uy, cz = v[jz] - uz;
                or_cadd(&s2, (cx * cx + cy * cy + cz * cz) * fv * dv3);
            }
    *rho = r;
    u[0] = ux;
    u[1] = uy;
    u[2] = uz;
    *th = or_cval(&s2) / (3.0 * r);
}

/* Discrete projection P, Def. 1 / Eq. (18), primitive output [5][nx]. */
int or_project(const or_kin* k, const double* f, double* U)
{
    int rc = check_kin(k);
    if (rc) return rc;
    int nx = k->nx, nv = k->nv;
    long nv3 = (long)nv * nv * nv;
    double* v = malloc(sizeof(double) * nv);
    if (!v) return OR_ENOMEM;
    or_velocity_nodes(nv, k->L, v);
    double dv = 2.0 * k->L / nv, dv3 = dv * dv * dv;
    int bad = 0;
    for (int i = 0; i < nx; ++i) {
        double rho, u[3], th;
        column_moments(nv, v, dv3, f + (long)i * nv3, &rho, u, &th);
        if (!(rho > 0.0) || !(th > 0.0)) bad = 1;
        U[0 * nx + i] = rho;
        U[1 * nx + i] = u[0];
        U[2 * nx + i] = u[1];
        U[3 * nx + i] = u[2];
        U[4 * nx + i] = th;
    }
    free(v);
    return bad ? OR_ENONPHYS : OR_OK;
}

int or_project_cons(const or_kin* k, const double* f, double* V)
{
    double* U = malloc(sizeof(double) * 5 * k->nx);
    if (!U) return OR_ENOMEM;
    int rc = or_project(k, f, U);
    or_prim_to_cons(k->nx, U, V);
    free(U);
    return rc;
}

/* Value of f at x cell c (possibly a ghost, -2 <= c <= nx+1) and velocity
 * (jx, jy, jz), through the boundary condition (reading R11). */
static double ext_value(const or_kin* k, const double* f, long nv3, int c, int jx, int jy, int jz)
{
    int nx = k->nx, nv = k->nv;
    int cc = c, jxx = jx;
    if (c < 0 || c >= nx) {
        if (k->bc == OR_BC_PERIODIC) {
            cc = ((c % nx) + nx) % nx;
        } else if (k->bc == OR_BC_OUTFLOW) {
            cc = c < 0 ? 0 : nx - 1;
        } else { /* reflecting: mirror cell, reversed v_x */
            cc = c < 0 ? -1 - c : 2 * nx - 1 - c;
            jxx = nv - 1 - jx;
        }
    }
    return f[(long)cc * nv3 + ((long)jxx * nv + jy) * nv + jz];
}

static double minmod(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/* Numerical flux F_{c+1/2} at velocity (jx, jy, jz), Eq. (13) with reading R1;
 * for MUSCL the interface values are the minmod-limited reconstructions
 * f_c + sigma_c / 2 (from the left) and f_{c+1} - sigma_{c+1} / 2 (from the right). */
static double xflux(const or_kin* k, const double* f, long nv3, double vx, int c, int jx, int jy, int jz)
{
    double fl, fr;
    if (k->scheme == OR_UPWIND) {
        fl = ext_value(k, f, nv3, c, jx, jy, jz);
        fr = ext_value(k, f, nv3, c + 1, jx, jy, jz);
    } else {
        double fm = ext_value(k, f, nv3, c - 1, jx, jy, jz);
        double f0 = ext_value(k, f, nv3, c, jx, jy, jz);
        double f1 = ext_value(k, f, nv3, c + 1, jx, jy, jz);
        double f2 = ext_value(k, f, nv3, c + 2, jx, jy, jz);
        fl = f0 + 0.5 * minmod(f0 - fm, f1 - f0);
        fr = f1 - 0.5 * minmod(f1 - f0, f2 - f1);
    }
    double vplus = vx > 0.0 ? vx : 0.0;
    double vminus = vx < 0.0 ? -vx : 0.0;
    return vplus * fl - vminus * fr;
}

/* One fine step of the IMEX scheme, Eqs. (11)-(13):
 *   f*_ij   = f_ij - dt/dx (F_{i+1/2,j} - F_{i-1/2,j})         (explicit transport)
 *   (rho,u,theta)_i = P(f*_i)                                 (explicit by conservation)
 *   f^{n+1}_ij = (eps f*_ij + dt M_ij) / (eps + dt)            (implicit BGK, R3)
 * With E = 0 the velocity flux G of Eq. (13) vanishes.  eps = +inf drops BGK. */
int or_fine_step(const or_kin* k, double dt, const double* f, double* fout)
{
    int rc = check_kin(k);
    if (rc) return rc;
    if (!(dt > 0.0)) return OR_EINVAL;
    int nx = k->nx, nv = k->nv;
    long nv3 = (long)nv * nv * nv;
    double dx = (k->x1 - k->x0) / nx;
    double dv = 2.0 * k->L / nv, dv3 = dv * dv * dv;
    double* v = malloc(sizeof(double) * nv);
    if (!v) return OR_ENOMEM;
    or_velocity_nodes(nv, k->L, v);
    const double pi = 3.14159265358979323846;
    int collide = isfinite(k->eps);
    int bad = 0;

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads) reduction(| : bad)
#endif
    for (int i = 0; i < nx; ++i) {
        double* out = fout + (long)i * nv3;
        /* transport */
        for (int jx = 0; jx < nv; ++jx)
            for (int jy = 0; jy < nv; ++jy)
                for (int jz = 0; jz < nv; ++jz) {
                    double fr = xflux(k, f, nv3, v[jx], i, jx, jy, jz);
                    double fl = xflux(k, f, nv3, v[jx], i - 1, jx, jy, jz);
                    long j = ((long)jx * nv + jy) * nv + jz;
                    out[j] = f[(long)i * nv3 + j] - dt / dx * (fr - fl);
                }
        if (!collide) continue;
        /* moments of f*, then the Maxwellian and the implicit relaxation */
        double rho, u[3], th;
        column_moments(nv, v, dv3, out, &rho, u, &th);
        if (!(rho > 0.0) || !(th > 0.0)) bad = 1;
        double pref = rho / pow(2.0 * pi * th, 1.5);
        for (int jx = 0; jx < nv; ++jx)
            for (int jy = 0; jy < nv; ++jy)
                for (int jz = 0; jz < nv; ++jz) {
                    long j = ((long)jx * nv + jy) * nv + jz;
                    double cx = v[jx] - u[0], cy = v[jy] - u[1], cz = v[jz] - u[2];
                    double M = pref * exp(-(cx * cx + cy * cy + cz * cz) / (2.0 * th));
                    out[j] = (k->eps * out[j] + dt * M) / (k->eps + dt);
                }
    }
    free(v);
    return bad ? OR_ENONPHYS : OR_OK;
}

int or_fine_run(const or_kin* k, double dt, int nsteps, double* f)
{
    int rc = check_kin(k);
    if (rc) return rc;
    if (nsteps < 0) return OR_EINVAL;
    long n = (long)k->nx * k->nv * k->nv * k->nv;
    double* tmp = malloc(sizeof(double) * n);
    if (!tmp) return OR_ENOMEM;
    for (int s = 0; s < nsteps; ++s) {
        rc = or_fine_step(k, dt, f, tmp);
        memcpy(f, tmp, sizeof(double) * n);
        if (rc) break;
    }
    free(tmp);
    return rc;
}

/* Stable fine step for the x transport: dt_stab = cfl dx / max|v_x|, max|v_x|
 * being the outermost velocity node (Sec. 2.2, local steps). */
double or_fine_dt_stab(const or_kin* k, double cfl)
{
    double dx = (k->x1 - k->x0) / k->nx;
    double dv = 2.0 * k->L / k->nv;
    double vmax = k->L - 0.5 * dv;
    return cfl * dx / vmax;
}

/* Reading R9: n_f = ceil(dT_g / dt_stab); a relative slack of 1e-9 keeps an
 * exact ratio (e.g. 12.000000000000002) from adding a step. */
int or_fine_nsteps(const or_pr* p, double* dt_out)
{
    double dTg = p->T / p->N;
    int nf = p->nf;
    if (nf <= 0) {
        double r = dTg / or_fine_dt_stab(&p->kin, p->cfl_f);
        nf = (int)ceil(r * (1.0 - 1e-9));
        if (nf < 1) nf = 1;
    }
    if (dt_out) *dt_out = dTg / nf;
    return nf;
}

/* ---------------- coarse propagator: Euler, Rusanov (Eqs. 14-16) ---------------- */

static void euler_prim(const double* Vc, double* ux, double* uy, double* uz, double* p, double* th)
{
    double rho = Vc[0];
    *ux = Vc[1] / rho;
    *uy = Vc[2] / rho;
    *uz = Vc[3] / rho;
    *th = (2.0 * Vc[4] / rho - (*ux * *ux + *uy * *uy + *uz * *uz)) / 3.0;
    *p = rho * *th;
}

/* Physical flux h(V) of Eq. (14). */
static void euler_flux(const double* Vc, double* h)
{
    double ux, uy, uz, p, th;
    euler_prim(Vc, &ux, &uy, &uz, &p, &th);
    h[0] = Vc[1];
    h[1] = Vc[1] * ux + p;
    h[2] = Vc[1] * uy;
    h[3] = Vc[1] * uz;
    h[4] = ux * (Vc[4] + p);
}

static double wave_speed(const double* Vc, int sound)
{
    double ux, uy, uz, p, th;
    euler_prim(Vc, &ux, &uy, &uz, &p, &th);
    double c = sound == OR_SOUND_SQRT_THETA ? sqrt(th) : sqrt(5.0 * th / 3.0);
    return fabs(ux) + c;
}

/* Ghost cell value for the fluid state (reading R11; reflecting negates rho u_x). */
static void ext_state(int nx, int bc, const double* V, int c, double* out)
{
    int cc = c, flip = 0;
    if (c < 0 || c >= nx) {
        if (bc == OR_BC_PERIODIC) cc = ((c % nx) + nx) % nx;
        else if (bc == OR_BC_OUTFLOW) cc = c < 0 ? 0 : nx - 1;
        else {
            cc = c < 0 ? -1 - c : 2 * nx - 1 - c;
            flip = 1;
        }
    }
    for (int q = 0; q < 5; ++q) out[q] = V[q * nx + cc];
    if (flip) out[1] = -out[1];
}

/* Rusanov flux H_{c+1/2} (reading R4). */
static void rusanov(int nx, int bc, int sound, const double* V, int c, double* H)
{
    double a[5], b[5], ha[5], hb[5];
    ext_state(nx, bc, V, c, a);
    ext_state(nx, bc, V, c + 1, b);
    euler_flux(a, ha);
    euler_flux(b, hb);
    double sa = wave_speed(a, sound), sb = wave_speed(b, sound);
    double S = sa > sb ? sa : sb;
    for (int q = 0; q < 5; ++q) H[q] = 0.5 * (ha[q] + hb[q]) - 0.5 * S * (b[q] - a[q]);
}

/* G over dT: explicit Rusanov updates, Eq. (15) with reading R2, local steps
 * dt = min(cfl dx / max S, remaining) until dT is reached (Sec. 2.2).  With an
 * exterior force E [nx] (NULL: none) each local step adds dt S(V_i), the source
 * S = (0, rho E_i, 0, 0, rho u_x E_i) of the Euler system Eq. (5) (reading R18:
 * forward Euler, the force at the cell centre). */
/* Viscous flux D_{c+1/2} of Eq. (8) (reading R22), added to the Rusanov flux. */
static void viscous(int nx, int bc, double dx, double eps, const double* V, int c, double* D)
{
    double a[5], b[5];
    ext_state(nx, bc, V, c, a);
    ext_state(nx, bc, V, c + 1, b);
    double uxa, uya, uza, pa, tha, uxb, uyb, uzb, pb, thb;
    euler_prim(a, &uxa, &uya, &uza, &pa, &tha);
    euler_prim(b, &uxb, &uyb, &uzb, &pb, &thb);
    double mu = 0.5 * (pa + pb);  /* rho theta averaged over the face */
    double kappa = 2.5 * mu;
    double dux = (uxb - uxa) / dx, duy = (uyb - uya) / dx, duz = (uzb - uza) / dx, dth = (thb - tha) / dx;
    double ux = 0.5 * (uxa + uxb), uy = 0.5 * (uya + uyb), uz = 0.5 * (uza + uzb);
    double sxx = -eps * mu * (4.0 / 3.0) * dux, sxy = -eps * mu * duy, sxz = -eps * mu * duz;
    double q = -eps * kappa * dth;
    D[0] = 0.0;
    D[1] = sxx;
    D[2] = sxy;
    D[3] = sxz;
    D[4] = sxx * ux + sxy * uy + sxz * uz + q;
}

static int coarse_run_impl(int nx, double x0, double x1, int bc, double cfl, int sound,
                           double dT, double visc, const double* E, const double* Vin, double* Vout, int* nsub)
{
    if (nx < 1 || !(x1 > x0) || !(cfl > 0.0) || dT < 0.0) return OR_EINVAL;
    double dx = (x1 - x0) / nx;
    double* V = malloc(sizeof(double) * 5 * nx);
    double* W = malloc(sizeof(double) * 5 * nx);
    if (!V || !W) {
        free(V);
        free(W);
        return OR_ENOMEM;
    }
    memcpy(V, Vin, sizeof(double) * 5 * nx);
    double t = 0.0;
    int steps = 0, rc = OR_OK;
    while (t < dT) {
        double smax = 0.0, thmax = 0.0;
        for (int i = 0; i < nx; ++i) {
            double Vc[5];
            for (int q = 0; q < 5; ++q) Vc[q] = V[q * nx + i];
            double ux, uy, uz, p, th;
            euler_prim(Vc, &ux, &uy, &uz, &p, &th);
            if (!(Vc[0] > 0.0) || !(th > 0.0)) rc = OR_ENONPHYS;
            double s = wave_speed(Vc, sound);
            if (s > smax) smax = s;
            if (th > thmax) thmax = th;
        }
        if (rc) break;
        double rem = dT - t;
        double dt = cfl * dx / smax;
        if (visc > 0.0) {
            double dtv = cfl * dx * dx / (2.0 * visc * (5.0 / 3.0) * thmax);
            if (dtv < dt) dt = dtv;
        }
        int last = 0;
        if (dt >= rem) {
            dt = rem;
            last = 1;
        }
        for (int i = 0; i < nx; ++i) {
            double Hr[5], Hl[5];
            rusanov(nx, bc, sound, V, i, Hr);
            rusanov(nx, bc, sound, V, i - 1, Hl);
            if (visc > 0.0) {
                double Dr[5], Dl[5];
                viscous(nx, bc, dx, visc, V, i, Dr);
                viscous(nx, bc, dx, visc, V, i - 1, Dl);
                for (int q = 0; q < 5; ++q) {
                    Hr[q] += Dr[q];
                    Hl[q] += Dl[q];
                }
            }
            for (int q = 0; q < 5; ++q) W[q * nx + i] = V[q * nx + i] - dt / dx * (Hr[q] - Hl[q]);
            if (E) {
                W[1 * nx + i] += dt * V[0 * nx + i] * E[i];
                W[4 * nx + i] += dt * V[1 * nx + i] * E[i];
            }
        }
        memcpy(V, W, sizeof(double) * 5 * nx);
        ++steps;
        if (last) break;
        t += dt;
    }
    memcpy(Vout, V, sizeof(double) * 5 * nx);
    if (nsub) *nsub = steps;
    free(V);
    free(W);
    return rc;
}

int or_coarse_run(int nx, double x0, double x1, int bc, double cfl, int sound,
                  double dT, const double* Vin, double* Vout, int* nsub)
{
    return coarse_run_impl(nx, x0, x1, bc, cfl, sound, dT, 0.0, NULL, Vin, Vout, nsub);
}

int or_coarse_run_force(int nx, double x0, double x1, int bc, double cfl, int sound,
                        double dT, const double* E, const double* Vin, double* Vout, int* nsub)
{
    return coarse_run_impl(nx, x0, x1, bc, cfl, sound, dT, 0.0, E, Vin, Vout, nsub);
}

int or_coarse_run_cns(int nx, double x0, double x1, int bc, double cfl, int sound, double dT, double eps,
                      const double* E, const double* Vin, double* Vout, int* nsub)
{
    if (!(eps > 0.0) || !isfinite(eps)) return OR_EINVAL;
    return coarse_run_impl(nx, x0, x1, bc, cfl, sound, dT, eps, E, Vin, Vout, nsub);
}

/* Gradients (d u_x, d u_y, d u_z, d theta) at cell i of a primitive state
 * [5][nx] by central differences through the ghost cells (reading R23; a
 * reflecting ghost negates u_x). */
void or_prim_gradients(int nx, int bc, double dx, const double* U, int i, double* d)
{
    double g[2][5];
    for (int s = 0; s < 2; ++s) {
        int c = i + (s == 0 ? -1 : 1), cc = c, flip = 0;
        if (c < 0 || c >= nx) {
            if (bc == OR_BC_PERIODIC) cc = ((c % nx) + nx) % nx;
            else if (bc == OR_BC_OUTFLOW) cc = c < 0 ? 0 : nx - 1;
            else {
                cc = c < 0 ? -1 - c : 2 * nx - 1 - c;
                flip = 1;
            }
        }
        for (int q = 0; q < 5; ++q) g[s][q] = U[q * nx + cc];
        if (flip) g[s][1] = -g[s][1];
    }
    for (int q = 0; q < 4; ++q) d[q] = (g[1][q + 1] - g[0][q + 1]) / (2.0 * dx);
}

/* One column of the first-order lifting (reading R23): f = M (1 - eps P(c))
 * at the nodes vx[nvx] x vp[nvp] x vp[nvp], U5 primitive, d = gradients. */
void or_ce_column(const double* vx, int nvx, const double* vp, int nvp, const double* U5, const double* d,
                  double eps, double* fc)
{
    const double pi = 3.14159265358979323846;
    double rho = U5[0], ux = U5[1], uy = U5[2], uz = U5[3], th = U5[4];
    double pref = rho / pow(2.0 * pi * th, 1.5);
    for (int jx = 0; jx < nvx; ++jx)
        for (int jy = 0; jy < nvp; ++jy)
            for (int jz = 0; jz < nvp; ++jz) {
                double cx = vx[jx] - ux, cy = vp[jy] - uy, cz = vp[jz] - uz;
                double c2 = cx * cx + cy * cy + cz * cz;
                double M = pref * exp(-c2 / (2.0 * th));
                double P = (cx * (cx * d[0] + cy * d[1] + cz * d[2]) - c2 * d[0] / 3.0) / th +
                           cx * (c2 / (2.0 * th) - 2.5) * d[3] / th;
                fc[((long)jx * nvp + jy) * nvp + jz] = M * (1.0 - eps * P);
            }
}

/* First-order lifting L^(1) (Def. 3, reading R23) on the isotropic grid. */
int or_lift_ce(const or_kin* k, const double* U, double* f)
{
    int rc = check_kin(k);
    if (rc) return rc;
    if (!isfinite(k->eps)) return OR_EINVAL;
    int nx = k->nx, nv = k->nv;
    long nv3 = (long)nv * nv * nv;
    double dx = (k->x1 - k->x0) / nx;
    double* v = malloc(sizeof(double) * nv);
    if (!v) return OR_ENOMEM;
    or_velocity_nodes(nv, k->L, v);
    int bad = 0;
    for (int i = 0; i < nx; ++i) {
        double U5[5], d[4];
        for (int q = 0; q < 5; ++q) U5[q] = U[q * nx + i];
        if (!(U5[0] > 0.0) || !(U5[4] > 0.0)) bad = 1;
        or_prim_gradients(nx, k->bc, dx, U, i, d);
        or_ce_column(v, nv, v, nv, U5, d, k->eps, f + (long)i * nv3);
    }
    free(v);
    return bad ? OR_ENONPHYS : OR_OK;
}

/* ---------------- propagators and the parareal algorithms ---------------- */

/* P F L: lift the conserved state (Eq. 17), n_f fine steps, project (Eq. 18). */
int or_fine_propagate(const or_pr* p, const double* Vin, double* Vout)
{
    const or_kin* k = &p->kin;
    int nx = k->nx;
    long n = (long)nx * k->nv * k->nv * k->nv;
    double dt;
    int nf = or_fine_nsteps(p, &dt);
    double* U = malloc(sizeof(double) * 5 * nx);
    double* f = malloc(sizeof(double) * n);
    if (!U || !f) {
        free(U);
        free(f);
        return OR_ENOMEM;
    }
    int rc = or_cons_to_prim(nx, Vin, U);
    if (!rc) rc = p->lift == 1 ? or_lift_ce(k, U, f) : or_lift(k, U, f);
    if (!rc) rc = or_fine_run(k, dt, nf, f);
    if (!rc) rc = or_project_cons(k, f, Vout);
    free(U);
    free(f);
    return rc;
}

int or_coarse_propagate(const or_pr* p, const double* Vin, double* Vout)
{
    const or_kin* k = &p->kin;
    if (p->coarse == OR_COARSE_CNS)
        return or_coarse_run_cns(k->nx, k->x0, k->x1, k->bc, p->cfl_g, p->sound, p->T / p->N, k->eps, NULL, Vin,
                                 Vout, 0);
    return or_coarse_run(k->nx, k->x0, k->x1, k->bc, p->cfl_g, p->sound, p->T / p->N, Vin, Vout, 0);
}

/* Algorithms 1 and 2 (reading R8).  U0 is primitive [5][nx].  Uall receives
 * every level: Uall[(k*(N+1) + n)*5*nx + q*nx + i], conserved, k = 0..K.
 * errs[k-1] is the Eq. (10) error of iteration k (reading R7).  With tol > 0
 * the loop stops after the first iteration whose error is below tol; levels
 * after *k_done are left as copies of level *k_done. */
static int prop_fine(const void* p, const double* Vin, double* Vout)
{
    return or_fine_propagate((const or_pr*)p, Vin, Vout);
}

static int prop_coarse(const void* p, const double* Vin, double* Vout)
{
    return or_coarse_propagate((const or_pr*)p, Vin, Vout);
}

int or_parareal(const or_pr* p, const double* U0, int K, double tol, int alg,
                double* Uall, double* errs, int* k_done)
{
    int rc = check_kin(&p->kin);
    if (rc) return rc;
    return or_parareal_core(p->kin.nx, p->N, prop_fine, prop_coarse, p, U0, K, tol, alg, Uall, errs, k_done);
}

/* The loop of Algorithms 1 and 2 over any pair of propagators PFL and G. */
int or_parareal_core(int nx, int N, or_prop fine, or_prop coarse, const void* ctx, const double* U0,
                     int K, double tol, int alg, double* Uall, double* errs, int* k_done)
{
    int rc = OR_OK;
    if (nx < 1 || N < 1 || K < 0 || (alg != 1 && alg != 2)) return OR_EINVAL;
    long lvl = (long)(N + 1) * 5 * nx;
    double* D = malloc(sizeof(double) * lvl);  /* jumps Delta^n */
    double* a = malloc(sizeof(double) * 5 * nx);
    double* b = malloc(sizeof(double) * 5 * nx);
    if (!D || !a || !b) {
        free(D);
        free(a);
        free(b);
        return OR_ENOMEM;
    }
#define UL(kk, n) (Uall + (long)(kk) * lvl + (long)(n) * 5 * nx)
    or_prim_to_cons(nx, U0, UL(0, 0));
    for (int n = 1; n <= N && !rc; ++n) rc = coarse(ctx, UL(0, n - 1), UL(0, n));
    int done = 0;
    for (int k = 1; k <= K && !rc; ++k) {
        int start = alg == 2 ? k : 1;
        if (start > N + 1) start = N + 1;
        for (int n = 0; n < start && n <= N; ++n) memcpy(UL(k, n), UL(k - 1, n), sizeof(double) * 5 * nx);
        for (int n = start; n <= N && !rc; ++n) {
            rc = fine(ctx, UL(k - 1, n - 1), a);
            if (!rc) rc = coarse(ctx, UL(k - 1, n - 1), b);
            for (int q = 0; q < 5 * nx; ++q) D[(long)n * 5 * nx + q] = a[q] - b[q];
        }
        for (int n = start; n <= N && !rc; ++n) {
            rc = coarse(ctx, UL(k, n - 1), b);
            for (int q = 0; q < 5 * nx; ++q) UL(k, n)[q] = b[q] + D[(long)n * 5 * nx + q];
        }
        double err = 0.0;
        for (int n = 0; n <= N; ++n)
            for (int q = 0; q < 5 * nx; ++q) {
                double d = fabs(UL(k, n)[q] - UL(k - 1, n)[q]);
                if (d > err) err = d;
            }
        if (errs) errs[k - 1] = err;
        done = k;
        if (tol > 0.0 && err < tol) break;
    }
    for (int k = done + 1; k <= K; ++k) memcpy(UL(k, 0), UL(done, 0), sizeof(double) * lvl);
#undef UL
    if (k_done) *k_done = done;
    free(D);
    free(a);
    free(b);
    return rc;
}

/* ---------------- reference gradient (adjoint of the fine run) ----------------
 *
 * Not in the paper: the gradient of a scalar J(V(T)) of the final conserved
 * moments V(T) = P(f^N) with respect to the primitive initial state U0 of the
 * lifted distribution f^0 = L(U0) and to log(eps), for the upwind scheme.
 * Derived by hand from the forward steps above and written plainly: all
 * states are stored, the transport transpose is formed by scattering every
 * coefficient of the forward stencil (through the same ghost mapping), and
 * the BGK step is differentiated through the Maxwellian parameters
 * (rho, u, theta) of the transported column.
 */

/* g = T(f): the transport half of or_fine_step. */
static void transport_only(const or_kin* k, double dt, const double* v, const double* f, double* g)
{
    int nx = k->nx, nv = k->nv;
    long nv3 = (long)nv * nv * nv;
    double dx = (k->x1 - k->x0) / nx;
    for (int i = 0; i < nx; ++i)
        for (int jx = 0; jx < nv; ++jx)
            for (int jy = 0; jy < nv; ++jy)
                for (int jz = 0; jz < nv; ++jz) {
                    long j = ((long)jx * nv + jy) * nv + jz;
                    double fr = xflux(k, f, nv3, v[jx], i, jx, jy, jz);
                    double fl = xflux(k, f, nv3, v[jx], i - 1, jx, jy, jz);
                    g[(long)i * nv3 + j] = f[(long)i * nv3 + j] - dt / dx * (fr - fl);
                }
}

/* Add w * lg to lf at the stored cell of (possibly ghost) x cell c. */
static void scatter(const or_kin* k, double* lf, long nv3, int c, int jx, int jy, int jz, double w)
{
    int nx = k->nx, nv = k->nv;
    int cc = c, jxx = jx;
    if (c < 0 || c >= nx) {
        if (k->bc == OR_BC_PERIODIC) cc = ((c % nx) + nx) % nx;
        else if (k->bc == OR_BC_OUTFLOW) cc = c < 0 ? 0 : nx - 1;
        else {
            cc = c < 0 ? -1 - c : 2 * nx - 1 - c;
            jxx = nv - 1 - jx;
        }
    }
    lf[(long)cc * nv3 + ((long)jxx * nv + jy) * nv + jz] += w;
}

/* lf = T^T lg for the upwind transport: g_i = f_i - dt/dx (F_{i+1/2} - F_{i-1/2}),
 * F_{c+1/2} = v+ f_c - v- f_{c+1}; every coefficient is scattered back. */
static void transport_transpose(const or_kin* k, double dt, const double* v, const double* lg, double* lf)
{
    int nx = k->nx, nv = k->nv;
    long nv3 = (long)nv * nv * nv;
    double r = dt / ((k->x1 - k->x0) / nx);
    memset(lf, 0, sizeof(double) * nx * nv3);
    for (int i = 0; i < nx; ++i)
        for (int jx = 0; jx < nv; ++jx) {
            double vp = v[jx] > 0.0 ? v[jx] : 0.0, vm = v[jx] < 0.0 ? -v[jx] : 0.0;
            for (int jy = 0; jy < nv; ++jy)
                for (int jz = 0; jz < nv; ++jz) {
                    double l = lg[(long)i * nv3 + ((long)jx * nv + jy) * nv + jz];
                    scatter(k, lf, nv3, i, jx, jy, jz, l);              /* f_i        */
                    scatter(k, lf, nv3, i, jx, jy, jz, -r * vp * l);    /* -r F_{i+1/2}: v+ f_i   */
                    scatter(k, lf, nv3, i + 1, jx, jy, jz, r * vm * l); /*               -v- f_{i+1} */
                    scatter(k, lf, nv3, i - 1, jx, jy, jz, r * vp * l); /* +r F_{i-1/2}: v+ f_{i-1} */
                    scatter(k, lf, nv3, i, jx, jy, jz, -r * vm * l);    /*               -v- f_i  */
                }
        }
}

int or_adjoint(const or_kin* k, double dt, int nsteps, const double* U0, const double* lamV,
               double* dU0, double* dlogeps)
{
    int rc = check_kin(k);
    if (rc) return rc;
    if (k->scheme != OR_UPWIND || nsteps < 0 || !(dt > 0.0)) return OR_EINVAL;
    int nx = k->nx, nv = k->nv;
    long nv3 = (long)nv * nv * nv, n = (long)nx * nv3;
    double dv = 2.0 * k->L / nv, dv3 = dv * dv * dv;
    const double pi = 3.14159265358979323846;
    int collide = isfinite(k->eps);
    double a = collide ? k->eps / (k->eps + dt) : 1.0, b = collide ? dt / (k->eps + dt) : 0.0;
    double* v = malloc(sizeof(double) * nv);
    double* F = malloc(sizeof(double) * n * (nsteps + 1)); /* f^0 .. f^N */
    double* g = malloc(sizeof(double) * n);
    double* lam = malloc(sizeof(double) * n);
    double* lg = malloc(sizeof(double) * n);
    if (!v || !F || !g || !lam || !lg) {
        free(v); free(F); free(g); free(lam); free(lg);
        return OR_ENOMEM;
    }
    or_velocity_nodes(nv, k->L, v);
    rc = or_lift(k, U0, F);
    for (int s = 0; s < nsteps && !rc; ++s) rc = or_fine_step(k, dt, F + s * n, F + (s + 1) * n);
    /* seed: dJ/df^N_ij = dv^3 sum_q lamV_q,i phi_q(v_j), phi = (1, v, |v|^2/2) */
    for (int i = 0; i < nx; ++i)
        for (int jx = 0; jx < nv; ++jx)
            for (int jy = 0; jy < nv; ++jy)
                for (int jz = 0; jz < nv; ++jz) {
                    double e = 0.5 * (v[jx] * v[jx] + v[jy] * v[jy] + v[jz] * v[jz]);
                    lam[(long)i * nv3 + ((long)jx * nv + jy) * nv + jz] =
                        dv3 * (lamV[i] + lamV[nx + i] * v[jx] + lamV[2 * nx + i] * v[jy] + lamV[3 * nx + i] * v[jz] +
                               lamV[4 * nx + i] * e);
                }
    double deps = 0.0;
    for (int s = nsteps - 1; s >= 0 && !rc; --s) {
        /* step s: f^{s+1} = a g + b M[rho,u,theta of g], g = T(f^s) */
        transport_only(k, dt, v, F + s * n, g);
        for (int i = 0; i < nx; ++i) {
            const double* gc = g + (long)i * nv3;
            const double* lc = lam + (long)i * nv3;
            double* lgc = lg + (long)i * nv3;
            if (!collide) {
                memcpy(lgc, lc, sizeof(double) * nv3);
                continue;
            }
            double rho, u[3], th;
            column_moments(nv, v, dv3, gc, &rho, u, &th);
            double pref = rho / pow(2.0 * pi * th, 1.5);
            double Ar = 0.0, Au[3] = {0.0, 0.0, 0.0}, At = 0.0;
            for (int jx = 0; jx < nv; ++jx)
                for (int jy = 0; jy < nv; ++jy)
                    for (int jz = 0; jz < nv; ++jz) {
                        long j = ((long)jx * nv + jy) * nv + jz;
                        double c[3] = {v[jx] - u[0], v[jy] - u[1], v[jz] - u[2]};
                        double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
                        double M = pref * exp(-c2 / (2.0 * th));
                        double l = lc[j];
                        Ar += l * M / rho;
                        for (int d = 0; d < 3; ++d) Au[d] += l * M * c[d] / th;
                        At += l * M * (c2 / (2.0 * th * th) - 1.5 / th);
                        deps += l * a * b * (gc[j] - M);
                    }
            /* d rho/dg_j = dv3, d u/dg_j = dv3 (v_j - u)/rho, d theta/dg_j = dv3 (|v_j-u|^2 - 3 theta)/(3 rho) */
            for (int jx = 0; jx < nv; ++jx)
                for (int jy = 0; jy < nv; ++jy)
                    for (int jz = 0; jz < nv; ++jz) {
                        long j = ((long)jx * nv + jy) * nv + jz;
                        double c[3] = {v[jx] - u[0], v[jy] - u[1], v[jz] - u[2]};
                        double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
                        double dM = Ar * dv3 + (Au[0] * c[0] + Au[1] * c[1] + Au[2] * c[2]) * dv3 / rho +
                                    At * dv3 * (c2 - 3.0 * th) / (3.0 * rho);
                        lgc[j] = a * lc[j] + b * dM;
                    }
        }
        transport_transpose(k, dt, v, lg, lam);
    }
    /* lift: f^0_ij = M[rho_i, u_i, theta_i](v_j) */
    for (int i = 0; i < nx && !rc; ++i) {
        double rho = U0[i], u[3] = {U0[nx + i], U0[2 * nx + i], U0[3 * nx + i]}, th = U0[4 * nx + i];
        double pref = rho / pow(2.0 * pi * th, 1.5);
        double s[5] = {0, 0, 0, 0, 0};
        for (int jx = 0; jx < nv; ++jx)
            for (int jy = 0; jy < nv; ++jy)
                for (int jz = 0; jz < nv; ++jz) {
                    long j = ((long)jx * nv + jy) * nv + jz;
                    double c[3] = {v[jx] - u[0], v[jy] - u[1], v[jz] - u[2]};
                    double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
                    double M = pref * exp(-c2 / (2.0 * th));
                    double l = lam[(long)i * nv3 + j];
                    s[0] += l * M / rho;
                    for (int d = 0; d < 3; ++d) s[1 + d] += l * M * c[d] / th;
                    s[4] += l * M * (c2 / (2.0 * th * th) - 1.5 / th);
                }
        for (int q = 0; q < 5; ++q) dU0[q * nx + i] = s[q];
    }
    if (dlogeps) *dlogeps = deps;
    free(v); free(F); free(g); free(lam); free(lg);
    return rc;
}
