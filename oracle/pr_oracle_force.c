/*
 * Plain CPU FP64 oracle, exterior-force part: the collisional Vlasov equation
 * with E != 0 (Laidin & Rey, arXiv 2502.02704, Eq. (1) with alpha = 0, the
 * scheme of Eqs. (11)-(13), the Euler system with source Eq. (5), Test 3).
 *
 * TEST INFRASTRUCTURE ONLY, like pr_oracle.c: used by tests/, smoke() and the
 * bench's CPU leg; the CUDA library never links or calls it.
 *
 * Readings of garbled or silent passages (continuing R1-R15 of pr_oracle.c):
 *   R16 sign of the force term: Eq. (1) prints v.grad_x f - E.grad_v f, while
 *       Eq. (11), the flux G = E f of Eq. (13), the momentum balance of Eq. (5)
 *       (d_t(rho u) = ... + rho E) and Test 3 (E pushes mass towards x = 1) all
 *       need d_t f + v.grad_x f + E.grad_v f; that sign is taken.  E acts along
 *       v_x only (one space dimension).
 *   R17 velocity flux: Eq. (13) prints a viscosity term E_max/2 (f_{j+1} - f_{j+1}),
 *       identically zero.  It is read as the Rusanov flux
 *         G_{i,jx+1/2} = E_i/2 (f_{i,jx} + f_{i,jx+1}) - E_max/2 (f_{i,jx+1} - f_{i,jx}),
 *       E_max = max_i |E_i| (the printed max over i), with the 1/dv_x of the
 *       divergence inserted (as R2 does for 1/dx).  The velocity box is closed:
 *       G = 0 through v_x = -L and v_x = +L, so mass is conserved exactly.
 *   R18 coarse source: forward Euler, S(V_i) = (0, rho_i E_i, 0, 0, (rho u_x)_i E_i),
 *       added to each local Rusanov step (pr_oracle.c, or_coarse_run_force).
 *   R19 fine time step: the x and v_x fluxes together keep the update monotone
 *       when dt (max|v_x|/dx + E_max/dv_x) <= 1; dt_stab = cfl / (max|v_x|/dx +
 *       E_max/dv_x), which is R9's cfl dx / max|v_x| when E = 0.
 *   R20 the parareal state starts from U^0 = P(f_0); every slice, the first
 *       included, lifts its initial moments (Algorithms 1 and 2 take moments
 *       only).  A non-Maxwellian f_0 (Test 3's two beams) enters through its
 *       moments; the kinetic reference run starts from f_0 itself.
 */
#include "pr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int check_vkin(const or_vkin* k)
{
    if (!k || k->nx < 1 || k->nvx < 1 || k->nvp < 1 || !(k->L > 0.0) || !(k->x1 > k->x0)) return OR_EINVAL;
    if (k->bc < 0 || k->bc > 2 || k->scheme < 0 || k->scheme > 1) return OR_EINVAL;
    if (!(k->eps > 0.0)) return OR_EINVAL;
    if (k->scheme == OR_MUSCL && k->bc == OR_BC_REFLECT && k->nx < 2) return OR_EINVAL;
    return OR_OK;
}

static long ncol(const or_vkin* k) { return (long)k->nvx * k->nvp * k->nvp; }

/* Cell centres of the v_x and v_y = v_z grids (Sec. 3, cells V_j). */
static void nodes(const or_vkin* k, double* vx, double* vp)
{
    or_velocity_nodes(k->nvx, k->L, vx);
    or_velocity_nodes(k->nvp, k->L, vp);
}

static double cell_volume(const or_vkin* k)
{
    double dvx = 2.0 * k->L / k->nvx, dvp = 2.0 * k->L / k->nvp;
    return dvx * dvp * dvp;
}

static double force_max(const or_vkin* k)
{
    double m = 0.0;
    if (k->E)
        for (int i = 0; i < k->nx; ++i)
            if (fabs(k->E[i]) > m) m = fabs(k->E[i]);
    return m;
}

/* Discrete lifting, Eq. (17), on the anisotropic grid. */
int or_v_lift(const or_vkin* k, const double* U, double* f)
{
    int rc = check_vkin(k);
    if (rc) return rc;
    int nx = k->nx, nvx = k->nvx, nvp = k->nvp;
    long nc = ncol(k);
    double* vx = malloc(sizeof(double) * nvx);
    double* vp = malloc(sizeof(double) * nvp);
    if (!vx || !vp) {
        free(vx);
        free(vp);
        return OR_ENOMEM;
    }
    nodes(k, vx, vp);
    const double pi = 3.14159265358979323846;
    int bad = 0;
    for (int i = 0; i < nx; ++i) {
        double rho = U[0 * nx + i], ux = U[1 * nx + i], uy = U[2 * nx + i];
        double uz = U[3 * nx + i], th = U[4 * nx + i];
        if (!(rho > 0.0) || !(th > 0.0)) bad = 1;
        double pref = rho / pow(2.0 * pi * th, 1.5);
        for (int jx = 0; jx < nvx; ++jx)
            for (int jy = 0; jy < nvp; ++jy)
                for (int jz = 0; jz < nvp; ++jz) {
                    double cx = vx[jx] - ux, cy = vp[jy] - uy, cz = vp[jz] - uz;
                    double c2 = cx * cx + cy * cy + cz * cz;
                    f[(long)i * nc + ((long)jx * nvp + jy) * nvp + jz] = pref * exp(-c2 / (2.0 * th));
                }
    }
    free(vx);
    free(vp);
    return bad ? OR_ENONPHYS : OR_OK;
}

/* First-order lifting L^(1) (Def. 3, reading R23 of pr_oracle.c) on the
 * anisotropic grid; the force does not enter g1. */
int or_v_lift_ce(const or_vkin* k, const double* U, double* f)
{
    int rc = check_vkin(k);
    if (rc) return rc;
    if (!isfinite(k->eps)) return OR_EINVAL;
    int nx = k->nx;
    long nc = ncol(k);
    double dx = (k->x1 - k->x0) / nx;
    double* vx = malloc(sizeof(double) * k->nvx);
    double* vp = malloc(sizeof(double) * k->nvp);
    if (!vx || !vp) {
        free(vx);
        free(vp);
        return OR_ENOMEM;
    }
    nodes(k, vx, vp);
    int bad = 0;
    for (int i = 0; i < nx; ++i) {
        double U5[5], d[4];
        for (int q = 0; q < 5; ++q) U5[q] = U[q * nx + i];
        if (!(U5[0] > 0.0) || !(U5[4] > 0.0)) bad = 1;
        or_prim_gradients(nx, k->bc, dx, U, i, d);
        or_ce_column(vx, k->nvx, vp, k->nvp, U5, d, k->eps, f + (long)i * nc);
    }
    free(vx);
    free(vp);
    return bad ? OR_ENONPHYS : OR_OK;
}

/* Moments of one column by the quadrature of Eq. (18) (u first, then theta),
 * summed with compensation (or_cadd) as the E = 0 oracle does. */
static void vcolumn_moments(const or_vkin* k, const double* vx, const double* vp, double dv3, const double* fc,
                            double* rho, double* u, double* th)
{
    int nvx = k->nvx, nvp = k->nvp;
    or_csum s0 = {0, 0}, sx = {0, 0}, sy = {0, 0}, sz = {0, 0};
    for (int jx = 0; jx < nvx; ++jx)
        for (int jy = 0; jy < nvp; ++jy)
            for (int jz = 0; jz < nvp; ++jz) {
                double fv = fc[((long)jx * nvp + jy) * nvp + jz];
                or_cadd(&s0, fv * dv3);
                or_cadd(&sx, vx[jx] * fv * dv3);
                or_cadd(&sy, vp[jy] * fv * dv3);
                or_cadd(&sz, vp[jz] * fv * dv3);
            }
    double r = or_cval(&s0);
    double ux = or_cval(&sx) / r, uy = or_cval(&sy) / r, uz = or_cval(&sz) / r;
    or_csum s2 = {0, 0};
    for (int jx = 0; jx < nvx; ++jx)
        for (int jy = 0; jy < nvp; ++jy)
            for (int jz = 0; jz < nvp; ++jz) {
                double fv = fc[((long)jx * nvp + jy) * nvp + jz];
                double cx = vx[jx] - ux, cy = vp[jy] - uy, cz = vp[jz] - uz;
                or_cadd(&s2, (cx * cx + cy * cy + cz * cz) * fv * dv3);
            }
    *rho = r;
    u[0] = ux;
    u[1] = uy;
    u[2] = uz;
    *th = or_cval(&s2) / (3.0 * r);
}

int or_v_project(const or_vkin* k, const double* f, double* U)
{
    int rc = check_vkin(k);
    if (rc) return rc;
    int nx = k->nx;
    long nc = ncol(k);
    double* vx = malloc(sizeof(double) * k->nvx);
    double* vp = malloc(sizeof(double) * k->nvp);
    if (!vx || !vp) {
        free(vx);
        free(vp);
        return OR_ENOMEM;
    }
    nodes(k, vx, vp);
    double dv3 = cell_volume(k);
    int bad = 0;
    for (int i = 0; i < nx; ++i) {
        double rho, u[3], th;
        vcolumn_moments(k, vx, vp, dv3, f + (long)i * nc, &rho, u, &th);
        if (!(rho > 0.0) || !(th > 0.0)) bad = 1;
        U[0 * nx + i] = rho;
        U[1 * nx + i] = u[0];
        U[2 * nx + i] = u[1];
        U[3 * nx + i] = u[2];
        U[4 * nx + i] = th;
    }
    free(vx);
    free(vp);
    return bad ? OR_ENONPHYS : OR_OK;
}

int or_v_project_cons(const or_vkin* k, const double* f, double* V)
{
    double* U = malloc(sizeof(double) * 5 * k->nx);
    if (!U) return OR_ENOMEM;
    int rc = or_v_project(k, f, U);
    or_prim_to_cons(k->nx, U, V);
    free(U);
    return rc;
}

/* f at x cell c (ghosts allowed) and velocity (jx, jp), jp = jy*nvp + jz,
 * through the boundary condition (R11; a reflecting wall reverses v_x). */
static double vext(const or_vkin* k, const double* f, long nc, int c, int jx, int jp)
{
    int nx = k->nx, cc = c, jxx = jx;
    if (c < 0 || c >= nx) {
        if (k->bc == OR_BC_PERIODIC) {
            cc = ((c % nx) + nx) % nx;
        } else if (k->bc == OR_BC_OUTFLOW) {
            cc = c < 0 ? 0 : nx - 1;
        } else {
            cc = c < 0 ? -1 - c : 2 * nx - 1 - c;
            jxx = k->nvx - 1 - jx;
        }
    }
    return f[(long)cc * nc + (long)jxx * k->nvp * k->nvp + jp];
}

static double minmod(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/* x flux F_{c+1/2} (Eq. 13 with R1; MUSCL-minmod interface values, R10). */
static double vxflux(const or_vkin* k, const double* f, long nc, double vxj, int c, int jx, int jp)
{
    double fl, fr;
    if (k->scheme == OR_UPWIND) {
        fl = vext(k, f, nc, c, jx, jp);
        fr = vext(k, f, nc, c + 1, jx, jp);
    } else {
        double fm = vext(k, f, nc, c - 1, jx, jp);
        double f0 = vext(k, f, nc, c, jx, jp);
        double f1 = vext(k, f, nc, c + 1, jx, jp);
        double f2 = vext(k, f, nc, c + 2, jx, jp);
        fl = f0 + 0.5 * minmod(f0 - fm, f1 - f0);
        fr = f1 - 0.5 * minmod(f1 - f0, f2 - f1);
    }
    double vplus = vxj > 0.0 ? vxj : 0.0;
    double vminus = vxj < 0.0 ? -vxj : 0.0;
    return vplus * fl - vminus * fr;
}

/* v_x flux G_{i, a+1/2} between velocity cells a and a+1 of column fc (R17);
 * zero through the two ends of the velocity box. */
static double vflux(const or_vkin* k, const double* fc, double Ei, double Emax, int a, int jp)
{
    if (a < 0 || a >= k->nvx - 1) return 0.0;
    long s = (long)k->nvp * k->nvp;
    double f0 = fc[(long)a * s + jp], f1 = fc[(long)(a + 1) * s + jp];
    return 0.5 * Ei * (f0 + f1) - 0.5 * Emax * (f1 - f0);
}

/* One fine step of Eqs. (11)-(13) with the force (R16, R17):
 *   f*_ij = f_ij - dt/dx (F_{i+1/2,j} - F_{i-1/2,j}) - dt/dv_x (G_{i,j+1/2} - G_{i,j-1/2})
 *   (rho, u, theta)_i = P(f*_i),  f^{n+1}_ij = (eps f*_ij + dt M_ij) / (eps + dt). */
int or_v_fine_step(const or_vkin* k, double dt, const double* f, double* fout)
{
    int rc = check_vkin(k);
    if (rc) return rc;
    if (!(dt > 0.0)) return OR_EINVAL;
    int nx = k->nx, nvx = k->nvx, nvp = k->nvp;
    long nc = ncol(k);
    double dx = (k->x1 - k->x0) / nx, dvx = 2.0 * k->L / nvx, dv3 = cell_volume(k);
    double Emax = force_max(k);
    double* vx = malloc(sizeof(double) * nvx);
    double* vp = malloc(sizeof(double) * nvp);
    if (!vx || !vp) {
        free(vx);
        free(vp);
        return OR_ENOMEM;
    }
    nodes(k, vx, vp);
    const double pi = 3.14159265358979323846;
    int collide = isfinite(k->eps);
    int bad = 0;

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(or_get_threads()) reduction(| : bad)
#endif
    for (int i = 0; i < nx; ++i) {
        const double* fc = f + (long)i * nc;
        double* out = fout + (long)i * nc;
        double Ei = k->E ? k->E[i] : 0.0;
        for (int jx = 0; jx < nvx; ++jx)
            for (int jy = 0; jy < nvp; ++jy)
                for (int jz = 0; jz < nvp; ++jz) {
                    int jp = jy * nvp + jz;
                    double Fr = vxflux(k, f, nc, vx[jx], i, jx, jp);
                    double Fl = vxflux(k, f, nc, vx[jx], i - 1, jx, jp);
                    double Gr = vflux(k, fc, Ei, Emax, jx, jp);
                    double Gl = vflux(k, fc, Ei, Emax, jx - 1, jp);
                    long j = (long)jx * nvp * nvp + jp;
                    out[j] = fc[j] - dt / dx * (Fr - Fl) - dt / dvx * (Gr - Gl);
                }
        if (!collide) continue;
        double rho, u[3], th;
        vcolumn_moments(k, vx, vp, dv3, out, &rho, u, &th);
        if (!(rho > 0.0) || !(th > 0.0)) bad = 1;
        double pref = rho / pow(2.0 * pi * th, 1.5);
        for (int jx = 0; jx < nvx; ++jx)
            for (int jy = 0; jy < nvp; ++jy)
                for (int jz = 0; jz < nvp; ++jz) {
                    long j = ((long)jx * nvp + jy) * nvp + jz;
                    double cx = vx[jx] - u[0], cy = vp[jy] - u[1], cz = vp[jz] - u[2];
                    double M = pref * exp(-(cx * cx + cy * cy + cz * cz) / (2.0 * th));
                    out[j] = (k->eps * out[j] + dt * M) / (k->eps + dt);
                }
    }
    free(vx);
    free(vp);
    return bad ? OR_ENONPHYS : OR_OK;
}

int or_v_fine_run(const or_vkin* k, double dt, int nsteps, double* f)
{
    int rc = check_vkin(k);
    if (rc) return rc;
    if (nsteps < 0) return OR_EINVAL;
    long n = (long)k->nx * ncol(k);
    double* tmp = malloc(sizeof(double) * n);
    if (!tmp) return OR_ENOMEM;
    for (int s = 0; s < nsteps; ++s) {
        rc = or_v_fine_step(k, dt, f, tmp);
        memcpy(f, tmp, sizeof(double) * n);
        if (rc) break;
    }
    free(tmp);
    return rc;
}

/* R19: dt_stab = cfl / (max|v_x| / dx + E_max / dv_x). */
double or_v_fine_dt_stab(const or_vkin* k, double cfl)
{
    double dx = (k->x1 - k->x0) / k->nx;
    double dvx = 2.0 * k->L / k->nvx;
    double vmax = k->L - 0.5 * dvx;
    double Emax = force_max(k);
    if (Emax == 0.0) return cfl * dx / vmax; /* R9 exactly */
    return cfl / (vmax / dx + Emax / dvx);
}

/* n_f = ceil(dT_g / dt_stab) as in R9, uniform dt = dT_g / n_f. */
int or_v_fine_nsteps(const or_vpr* p, double* dt_out)
{
    double dTg = p->T / p->N;
    int nf = p->nf;
    if (nf <= 0) {
        double r = dTg / or_v_fine_dt_stab(&p->kin, p->cfl_f);
        nf = (int)ceil(r * (1.0 - 1e-9));
        if (nf < 1) nf = 1;
    }
    if (dt_out) *dt_out = dTg / nf;
    return nf;
}

/* P F L with the force: lift (Eq. 17), n_f fine steps, project (Eq. 18). */
int or_v_fine_propagate(const or_vpr* p, const double* Vin, double* Vout)
{
    const or_vkin* k = &p->kin;
    int nx = k->nx;
    long n = (long)nx * ncol(k);
    double dt;
    int nf = or_v_fine_nsteps(p, &dt);
    double* U = malloc(sizeof(double) * 5 * nx);
    double* f = malloc(sizeof(double) * n);
    if (!U || !f) {
        free(U);
        free(f);
        return OR_ENOMEM;
    }
    int rc = or_cons_to_prim(nx, Vin, U);
    if (!rc) rc = p->lift == 1 ? or_v_lift_ce(k, U, f) : or_v_lift(k, U, f);
    if (!rc) rc = or_v_fine_run(k, dt, nf, f);
    if (!rc) rc = or_v_project_cons(k, f, Vout);
    free(U);
    free(f);
    return rc;
}

/* G with the Euler source (R18). */
int or_v_coarse_propagate(const or_vpr* p, const double* Vin, double* Vout)
{
    const or_vkin* k = &p->kin;
    if (p->coarse == OR_COARSE_CNS)
        return or_coarse_run_cns(k->nx, k->x0, k->x1, k->bc, p->cfl_g, p->sound, p->T / p->N, k->eps, k->E, Vin,
                                 Vout, 0);
    return or_coarse_run_force(k->nx, k->x0, k->x1, k->bc, p->cfl_g, p->sound, p->T / p->N, k->E, Vin, Vout, 0);
}

static int prop_fine(const void* p, const double* Vin, double* Vout)
{
    return or_v_fine_propagate((const or_vpr*)p, Vin, Vout);
}

static int prop_coarse(const void* p, const double* Vin, double* Vout)
{
    return or_v_coarse_propagate((const or_vpr*)p, Vin, Vout);
}

/* Algorithms 1 and 2 with the force propagators (R20 for the initial state). */
int or_v_parareal(const or_vpr* p, const double* U0, int K, double tol, int alg,
                  double* Uall, double* errs, int* k_done)
{
    int rc = check_vkin(&p->kin);
    if (rc) return rc;
    return or_parareal_core(p->kin.nx, p->N, prop_fine, prop_coarse, p, U0, K, tol, alg, Uall, errs, k_done);
}
