// Adjoint (vector-Jacobian product) of the float64 upwind fine run, for
// gradients of a scalar J(V(T)) of the final conserved moments with respect to
// the primitive initial state U0 of the lifted f^0 = L(U0) and to log(eps).
// Not in the paper; it differentiates the fine scheme of Eqs. (11)-(13), (17),
// (18).  One fine step reads
//     g = T f  (upwind transport),   f' = a g + b M[m(g)],
// with m(g) the conserved moments of g and M the Maxwellian of (rho, u, theta)(m):
// rho = m0, u = m_d/rho, theta = (2 E/rho - |u|^2)/3, E = m4.  Given
// lam' = dJ/df', the adjoint of the step is
//     A_rho = sum lam' M/rho,  A_u = sum lam' M (v - u)/theta,
//     A_th  = sum lam' M (|v-u|^2/(2 theta^2) - 3/(2 theta)),
//     lam_g = a lam' + b dv^3 [c0 + c.v + c4 |v|^2]   (chain rule through m(g)),
//     lam   = T^T lam_g,
//     dJ/dlog eps += sum lam' a b (g - M)            (da/dlog eps = a b = -db/dlog eps),
// and the lift contributes dJ/dU0 = sum lam^0 dM/d(rho, u, theta).
#include <math.h>

#include "pr_kernels.h"

namespace prk {

namespace {

constexpr int AT = 256;
constexpr double PI = 3.14159265358979323846;

__device__ __forceinline__ void node(const Inst& I, int v, double& vx, double& vy, double& vz)
{
    const int nv = I.nv;
    const int jz = v % nv, jy = (v / nv) % nv, jx = v / (nv * nv);
    vx = -I.L + (jx + 0.5) * I.dv;
    vy = -I.L + (jy + 0.5) * I.dv;
    vz = -I.L + (jz + 0.5) * I.dv;
}

// seed: lam[c][v] = dv^3 (l0 + l1 vx + l2 vy + l3 vz + l4 |v|^2/2), l = dJ/dV(T)[.][c]
__global__ void k_adj_seed(Inst I, const double* lamV, double* lam)
{
    const int c = blockIdx.x, v = blockIdx.y * AT + threadIdx.x;
    if (v >= I.nv3) return;
    double vx, vy, vz;
    node(I, v, vx, vy, vz);
    const int nx = I.nx;
    lam[(size_t)c * I.nv3 + v] = I.dv3 * (lamV[c] + lamV[nx + c] * vx + lamV[2 * nx + c] * vy + lamV[3 * nx + c] * vz +
                                         lamV[4 * nx + c] * 0.5 * (vx * vx + vy * vy + vz * vz));
}

// Per x cell c, one CTA: the conserved moments m(g) of the transported
// state g (the step's f*), the Maxwellian of m(g) in its separable form
// M = rho (2 pi theta)^{-3/2} e_x[jx] e_y[jy] e_z[jz] (1-D factors in shared
// memory, 3 nv exponentials per cell instead of nv^3), then the sums A_rho,
// A_u, A_theta and the log-eps term, folded into the five coefficients of the
// BGK part of lam_g.  Threads own (jy, jz) pairs of the velocity plane and
// walk jx, so node indices come without divisions and each jx plane is read
// coalesced.
constexpr int ACT = 512;

// One exchange of a transposed butterfly over lane bit w: lanes with the bit
// clear keep values 0..n-1 and send n..2n-1 (the others the reverse).
template <int n>
__device__ __forceinline__ void adj_xchg(double (&y)[8], int lane, int w)
{
    const bool up = (lane & w) != 0;
#pragma unroll
    for (int j = 0; j < n; ++j) {
        const double send = up ? y[j] : y[j + n];
        const double keep = up ? y[j + n] : y[j];
        y[j] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
}

// Warp sums of eight values: lanes 4q .. 4q+3 return the sum of value q.
__device__ __forceinline__ double warp_sum8(double (&y)[8], int lane)
{
    adj_xchg<4>(y, lane, 16);
    adj_xchg<2>(y, lane, 8);
    adj_xchg<1>(y, lane, 4);
    y[0] += __shfl_xor_sync(0xffffffffu, y[0], 2);
    y[0] += __shfl_xor_sync(0xffffffffu, y[0], 1);
    return y[0];
}

// Sum of NV (<= 8) per-thread values over the CTA, the totals in every
// thread: a transposed butterfly in each warp, the warp sums through shared
// memory (sh: ADJ_SH doubles), the same butterfly over them in warp 0.
constexpr int ADJ_SH = 32 * 8 + 8;
template <int NV>
__device__ void block_sum_n(double (&x)[NV], double* sh)
{
    static_assert(NV <= 8, "at most eight sums");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    double y[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = q < NV ? x[q] : 0.0;
    double r = warp_sum8(y, lane);
    if ((lane & 3) == 0) sh[warp * 8 + (lane >> 2)] = r;
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) y[q] = lane < nw ? sh[lane * 8 + q] : 0.0;
        r = warp_sum8(y, lane);
        if ((lane & 3) == 0) sh[32 * 8 + (lane >> 2)] = r;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) x[q] = sh[32 * 8 + q];
    __syncthreads();
}

// 1-D Maxwellian factors of (u, theta) into e[3][nv] (e[0] carries pref).
__device__ void maxwell_factors(const Inst& I, double ux, double uy, double uz, double th, double pref, double* e)
{
    const int nv = I.nv;
    const double i2t = 0.5 / th;
    for (int k = threadIdx.x; k < 3 * nv; k += blockDim.x) {
        const int d = k / nv, j = k - d * nv;
        const double c = -I.L + (j + 0.5) * I.dv - (d == 0 ? ux : d == 1 ? uy : uz);
        const double x = exp(-c * c * i2t);
        e[k] = d == 0 ? pref * x : x;
    }
}

__global__ void __launch_bounds__(ACT) k_adj_coef(Inst I, const double* lam, const double* g, const double* msum,
                                                 double* coef, double* eps_acc)
{
    extern __shared__ double ash[];  // e[3][nv], tx[2][nv], then the block-sum scratch
    const int c = blockIdx.x, nv = I.nv, np = nv * nv;
    double* e = ash;
    double* tx = ash + 3 * nv;  // v_x, then v_x - u_x
    double* sh = ash + 5 * nv;
    const double* gc = g + (size_t)c * I.ldv;
    const double* lc = lam + (size_t)c * I.nv3;
    for (int j = threadIdx.x; j < nv; j += blockDim.x) tx[j] = -I.L + (j + 0.5) * I.dv;
    __syncthreads();
    // moments of g: recorded by the forward kernel (sums in grid units,
    // v = k dv), or summed here (over the plane, then over jx)
    double m[5] = {0, 0, 0, 0, 0};
    if (msum) {
        const double* q = msum + (size_t)c * 5;
        m[0] = q[0];
        m[1] = q[1] * I.dv;
        m[2] = q[2] * I.dv;
        m[3] = q[3] * I.dv;
        m[4] = q[4] * I.dv * I.dv;
    } else {
        for (int p = threadIdx.x; p < np; p += blockDim.x) {
            const int jy = p / nv, jz = p - jy * nv;
            const double vy = -I.L + (jy + 0.5) * I.dv, vz = -I.L + (jz + 0.5) * I.dv;
            double s0 = 0, sx = 0, sxx = 0;
            for (int jx = 0; jx < nv; ++jx) {
                const double vx = tx[jx], f = gc[(size_t)jx * np + p];
                s0 += f;
                sx += vx * f;
                sxx += vx * vx * f;
            }
            m[0] += s0;
            m[1] += sx;
            m[2] += vy * s0;
            m[3] += vz * s0;
            m[4] += sxx + (vy * vy + vz * vz) * s0;
        }
        block_sum_n<5>(m, sh);
    }
    const double rho = m[0] * I.dv3, ir = 1.0 / rho;
    const double u[3] = {m[1] * I.dv3 * ir, m[2] * I.dv3 * ir, m[3] * I.dv3 * ir};
    const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double th = (m[4] * I.dv3 * ir - u2) / 3.0, ith = 1.0 / th;
    const double tp = 2.0 * PI * th, pref = rho / (tp * sqrt(tp));
    maxwell_factors(I, u[0], u[1], u[2], th, pref, e);
    for (int j = threadIdx.x; j < nv; j += blockDim.x) tx[nv + j] = tx[j] - u[0];
    __syncthreads();
    double s[6] = {0, 0, 0, 0, 0, 0};  // A_rho, A_u (3), A_theta, eps term
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int jy = p / nv, jz = p - jy * nv;
        const double cy = -I.L + (jy + 0.5) * I.dv - u[1], cz = -I.L + (jz + 0.5) * I.dv - u[2];
        const double eyz = e[nv + jy] * e[2 * nv + jz], cyz2 = cy * cy + cz * cz;
        double a0 = 0, ax = 0, axx = 0, ae = 0;
        for (int jx = 0; jx < nv; ++jx) {
            const double cx = tx[nv + jx];
            const double M = e[jx] * eyz, l = lc[(size_t)jx * np + p], lM = l * M;
            a0 += lM;
            ax += lM * cx;
            axx += lM * cx * cx;
            ae += l * (gc[(size_t)jx * np + p] - M);
        }
        s[0] += a0;
        s[1] += ax;
        s[2] += a0 * cy;
        s[3] += a0 * cz;
        s[4] += axx + a0 * cyz2;  // sum lM |v - u|^2
        s[5] += ae;
    }
    block_sum_n<6>(s, sh);
    if (threadIdx.x == 0) {
        // A_rho = sum lM / rho, A_u = sum lM c / theta, A_theta = sum lM (|c|^2/(2 theta^2) - 3/(2 theta))
        const double Ar = s[0] * ir, Ax = s[1] * ith, Ay = s[2] * ith, Az = s[3] * ith;
        const double At = 0.5 * s[4] * ith * ith - 1.5 * s[0] * ith;
        const double k3 = 1.0 / (3.0 * rho), w = I.b * I.dv3;
        coef[c * 5 + 0] = w * (Ar - (Ax * u[0] + Ay * u[1] + Az * u[2]) * ir + At * (u2 - 3.0 * th) * k3);
        coef[c * 5 + 1] = w * (Ax * ir - 2.0 * At * u[0] * k3);
        coef[c * 5 + 2] = w * (Ay * ir - 2.0 * At * u[1] * k3);
        coef[c * 5 + 3] = w * (Az * ir - 2.0 * At * u[2] * k3);
        coef[c * 5 + 4] = w * At * k3;
        eps_acc[c] += I.a * I.b * s[5];
    }
}

// lam_out = T^T lam_g for the upwind transport (periodic or outflow ghosts),
// lam_g = a lam + P_c(v), P_c(v) = k0 + k1 v_x + k2 v_y + k3 v_z + k4 |v|^2
// with cell c's coefficients.  For v_x > 0 the step reads
// g_i = (1 - cr) f_i + cr f_{i-1}, so lam_i = (1 - cr) lam_g,i + cr lam_g,i+1;
// for v_x < 0, g_i = (1 + cr) f_i - cr f_{i+1}, so lam_i = (1 + cr) lam_g,i -
// cr lam_g,i-1 (cr = v_x dt/dx with sign); an outflow ghost copies the end
// cell, which adds its weight to the end cell itself.  One CTA per (cell,
// part of the (v_y, v_z) plane); each thread walks v_x.  The per-v_x weights
// and the v_x parts of P for the cell and for its upwind neighbour come from
// shared-memory tables.
constexpr int APT = 256;

__global__ void __launch_bounds__(APT) k_adj_apply(Inst I, const double* lam, const double* coef, double* out)
{
    extern __shared__ double ap[];  // [nv] each: self weight, neighbour weight, P_x of c, P_x of the neighbour
    const int c = blockIdx.x, nx = I.nx, nv = I.nv, np = nv * nv;
    double* ws = ap;
    double* wn = ap + nv;
    double* pc = ap + 2 * nv;
    double* pn = ap + 3 * nv;
    int up = c + 1, dn = c - 1;
    bool has_up = true, has_dn = true;
    if (up >= nx) {
        if (I.bc == 0) up -= nx;
        else has_up = false;
    }
    if (dn < 0) {
        if (I.bc == 0) dn += nx;
        else has_dn = false;
    }
    const double* kc = coef + c * 5;
    const double* ku = coef + (has_up ? up : c) * 5;
    const double* kd = coef + (has_dn ? dn : c) * 5;
    for (int j = threadIdx.x; j < nv; j += blockDim.x) {
        const double vx = -I.L + (j + 0.5) * I.dv, cr = I.nu * vx;
        pc[j] = vx * (kc[1] + kc[4] * vx);
        if (vx > 0.0) {
            double self = 1.0 - cr;
            if (I.bc == 1 && c == 0) self += cr;  // outflow ghost f_{-1} = f_0
            ws[j] = self;
            wn[j] = has_up ? cr : 0.0;
            pn[j] = vx * (ku[1] + ku[4] * vx);
        } else if (vx < 0.0) {
            double self = 1.0 + cr;
            if (I.bc == 1 && c == nx - 1) self -= cr;  // outflow ghost f_{nx} = f_{nx-1}
            ws[j] = self;
            wn[j] = has_dn ? -cr : 0.0;
            pn[j] = vx * (kd[1] + kd[4] * vx);
        } else {
            ws[j] = 1.0;
            wn[j] = 0.0;
            pn[j] = 0.0;
        }
    }
    __syncthreads();
    const int p = blockIdx.y * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int jy = p / nv, jz = p - jy * nv;
    const double vy = -I.L + (jy + 0.5) * I.dv, vz = -I.L + (jz + 0.5) * I.dv, vyz2 = vy * vy + vz * vz;
    const double bc_ = kc[0] + kc[2] * vy + kc[3] * vz + kc[4] * vyz2;
    const double bu = ku[0] + ku[2] * vy + ku[3] * vz + ku[4] * vyz2;
    const double bd = kd[0] + kd[2] * vy + kd[3] * vz + kd[4] * vyz2;
    const double a = I.a;
    const double* lc = lam + (size_t)c * I.nv3 + p;
    const double* lu = lam + (size_t)(has_up ? up : c) * I.nv3 + p;
    const double* ld = lam + (size_t)(has_dn ? dn : c) * I.nv3 + p;
    double* o = out + (size_t)c * I.nv3 + p;
    const int half = nv / 2;  // v_x < 0 for jx < nv/2 (cube centres, even nv)
    for (int jx = 0; jx < nv; ++jx) {
        const size_t k = (size_t)jx * np;
        const double gself = a * lc[k] + bc_ + pc[jx];
        const double gn = jx < half ? a * ld[k] + bd + pn[jx] : a * lu[k] + bu + pn[jx];
        o[k] = ws[jx] * gself + wn[jx] * gn;
    }
}

// dJ/dU0[q][c] = sum_v lam^0 dM/dU_q with U = (rho, u, theta) from the
// conserved Uin (the separable Maxwellian, as in k_adj_coef)
__global__ void __launch_bounds__(ACT) k_adj_lift(Inst I, const double* lam, const double* Uin, double* dU0)
{
    extern __shared__ double ash[];
    const int c = blockIdx.x, nx = I.nx, nv = I.nv, np = nv * nv;
    double* e = ash;
    double* sh = ash + 3 * nv;
    const double rho = Uin[c], ir = 1.0 / rho;
    const double u[3] = {Uin[nx + c] * ir, Uin[2 * nx + c] * ir, Uin[3 * nx + c] * ir};
    const double th = (2.0 * Uin[4 * nx + c] * ir - (u[0] * u[0] + u[1] * u[1] + u[2] * u[2])) / 3.0, ith = 1.0 / th;
    const double tp = 2.0 * PI * th, pref = rho / (tp * sqrt(tp));
    maxwell_factors(I, u[0], u[1], u[2], th, pref, e);
    __syncthreads();
    const double* lc = lam + (size_t)c * I.nv3;
    double s[5] = {0, 0, 0, 0, 0};
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int jy = p / nv, jz = p - jy * nv;
        const double cy = -I.L + (jy + 0.5) * I.dv - u[1], cz = -I.L + (jz + 0.5) * I.dv - u[2];
        const double eyz = e[nv + jy] * e[2 * nv + jz], cyz2 = cy * cy + cz * cz;
        double a0 = 0, ax = 0, axx = 0;
        for (int jx = 0; jx < nv; ++jx) {
            const double cx = -I.L + (jx + 0.5) * I.dv - u[0];
            const double lM = lc[(size_t)jx * np + p] * e[jx] * eyz;
            a0 += lM;
            ax += lM * cx;
            axx += lM * cx * cx;
        }
        s[0] += a0;
        s[1] += ax;
        s[2] += a0 * cy;
        s[3] += a0 * cz;
        s[4] += axx + a0 * cyz2;
    }
    block_sum_n<5>(s, sh);
    if (threadIdx.x == 0) {
        dU0[c] = s[0] * ir;
        dU0[(size_t)nx + c] = s[1] * ith;
        dU0[(size_t)2 * nx + c] = s[2] * ith;
        dU0[(size_t)3 * nx + c] = s[3] * ith;
        dU0[(size_t)4 * nx + c] = 0.5 * s[4] * ith * ith - 1.5 * s[0] * ith;
    }
}

}  // namespace

cudaError_t adj_seed(const Inst& I, const double* lamV, double* lam, cudaStream_t s)
{
    k_adj_seed<<<dim3(I.nx, (I.nv3 + AT - 1) / AT), AT, 0, s>>>(I, lamV, lam);
    return cudaGetLastError();
}

static size_t adj_smem(const Inst& I) { return (5 * (size_t)I.nv + ADJ_SH) * sizeof(double); }

// Threads of the per-column kernels: two (v_y, v_z) planes each (nv^2 / 2,
// rounded up to whole warps, at most ACT), so the planes split evenly and two
// CTAs share an SM at the kernels' register counts.
static int adj_threads(const Inst& I)
{
    const int t = ((I.nv * I.nv + 1) / 2 + 31) / 32 * 32;
    return t < 32 ? 32 : (t > ACT ? ACT : t);
}

cudaError_t adj_step(const Inst& I, const double* lam_in, const double* g, const double* msum, double* coef,
                     double* eps_acc, double* lam_out, cudaStream_t s)
{
    k_adj_coef<<<I.nx, adj_threads(I), adj_smem(I), s>>>(I, lam_in, g, msum, coef, eps_acc);
    k_adj_apply<<<dim3(I.nx, (I.nv * I.nv + APT - 1) / APT), APT, 4 * (size_t)I.nv * sizeof(double), s>>>(
        I, lam_in, coef, lam_out);
    return cudaGetLastError();
}

cudaError_t adj_lift(const Inst& I, const double* lam, const double* Uin, double* dU0, cudaStream_t s)
{
    k_adj_lift<<<I.nx, adj_threads(I), adj_smem(I), s>>>(I, lam, Uin, dU0);
    return cudaGetLastError();
}


}  // namespace prk
