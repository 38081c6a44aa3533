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

template <int NV>
__device__ void block_sum(double (&x)[NV], double* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int o = 16; o; o >>= 1) x[q] += __shfl_xor_sync(0xffffffffu, x[q], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[warp * NV + q] = x[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double t = 0.0;
        for (int w = 0; w < AT / 32; ++w) t += sh[w * NV + q];
        x[q] = t;
    }
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

// conserved moments of g (stride ldv) per x cell: m[5][nx]
__global__ void __launch_bounds__(AT) k_adj_moments(Inst I, const double* g, double* m)
{
    __shared__ double sh[(AT / 32) * 5];
    const int c = blockIdx.x;
    double s[5] = {0, 0, 0, 0, 0};
    for (int v = threadIdx.x; v < I.nv3; v += AT) {
        double vx, vy, vz;
        node(I, v, vx, vy, vz);
        double f = g[(size_t)c * I.ldv + v];
        s[0] += f;
        s[1] += vx * f;
        s[2] += vy * f;
        s[3] += vz * f;
        s[4] += 0.5 * (vx * vx + vy * vy + vz * vz) * f;
    }
    block_sum<5>(s, sh);
    if (threadIdx.x < 5) m[(size_t)threadIdx.x * I.nx + c] = s[threadIdx.x] * I.dv3;
}

// per x cell: coefficients of the BGK part of lam_g and the log-eps term
__global__ void __launch_bounds__(AT) k_adj_coef(Inst I, const double* lam, const double* g, const double* m,
                                                double* coef, double* eps_acc)
{
    __shared__ double sh[(AT / 32) * 6];
    const int c = blockIdx.x, nx = I.nx;
    const double rho = m[c], ux = m[nx + c] / rho, uy = m[2 * nx + c] / rho, uz = m[3 * nx + c] / rho;
    const double th = (2.0 * m[4 * nx + c] / rho - (ux * ux + uy * uy + uz * uz)) / 3.0;
    const double tp = 2.0 * PI * th, pref = rho / (tp * sqrt(tp));
    double s[6] = {0, 0, 0, 0, 0, 0};  // A_rho, A_u (3), A_theta, eps term
    for (int v = threadIdx.x; v < I.nv3; v += AT) {
        double vx, vy, vz;
        node(I, v, vx, vy, vz);
        double cx = vx - ux, cy = vy - uy, cz = vz - uz, c2 = cx * cx + cy * cy + cz * cz;
        double M = pref * exp(-c2 / (2.0 * th));
        double l = lam[(size_t)c * I.nv3 + v], lM = l * M;
        s[0] += lM / rho;
        s[1] += lM * cx / th;
        s[2] += lM * cy / th;
        s[3] += lM * cz / th;
        s[4] += lM * (c2 / (2.0 * th * th) - 1.5 / th);
        s[5] += l * (g[(size_t)c * I.ldv + v] - M);
    }
    block_sum<6>(s, sh);
    if (threadIdx.x == 0) {
        const double Ar = s[0], Ax = s[1], Ay = s[2], Az = s[3], At = s[4];
        const double u2 = ux * ux + uy * uy + uz * uz, k3 = 1.0 / (3.0 * rho), w = I.b * I.dv3;
        coef[c * 5 + 0] = w * (Ar - (Ax * ux + Ay * uy + Az * uz) / rho + At * (u2 - 3.0 * th) * k3);
        coef[c * 5 + 1] = w * (Ax / rho - 2.0 * At * ux * k3);
        coef[c * 5 + 2] = w * (Ay / rho - 2.0 * At * uy * k3);
        coef[c * 5 + 3] = w * (Az / rho - 2.0 * At * uz * k3);
        coef[c * 5 + 4] = w * At * k3;
        eps_acc[c] += I.a * I.b * s[5];
    }
}

__device__ __forceinline__ double lam_g(const Inst& I, const double* lam, const double* coef, int c, int v, double vx,
                                        double vy, double vz)
{
    const double* k = coef + c * 5;
    return I.a * lam[(size_t)c * I.nv3 + v] + k[0] + k[1] * vx + k[2] * vy + k[3] * vz +
           k[4] * (vx * vx + vy * vy + vz * vz);
}

// lam_out = T^T lam_g for the upwind transport (periodic or outflow ghosts)
__global__ void k_adj_apply(Inst I, const double* lam, const double* coef, double* out)
{
    const int c = blockIdx.x, v = blockIdx.y * AT + threadIdx.x;
    if (v >= I.nv3) return;
    double vx, vy, vz;
    node(I, v, vx, vy, vz);
    const int nx = I.nx;
    const double cr = I.nu * vx;  // Courant number with sign
    double r;
    if (vx > 0.0) {
        // g_i = (1 - cr) f_i + cr f_{i-1}
        int up = c + 1;
        bool has_up = true;
        if (up >= nx) {
            if (I.bc == 0) up -= nx;
            else has_up = false;
        }
        double self = (1.0 - cr);
        if (I.bc == 1 && c == 0) self += cr;  // outflow ghost f_{-1} = f_0
        r = self * lam_g(I, lam, coef, c, v, vx, vy, vz);
        if (has_up) r += cr * lam_g(I, lam, coef, up, v, vx, vy, vz);
    } else if (vx < 0.0) {
        // g_i = (1 + cr) f_i - cr f_{i+1}
        int dn = c - 1;
        bool has_dn = true;
        if (dn < 0) {
            if (I.bc == 0) dn += nx;
            else has_dn = false;
        }
        double self = (1.0 + cr);
        if (I.bc == 1 && c == nx - 1) self -= cr;  // outflow ghost f_{nx} = f_{nx-1}
        r = self * lam_g(I, lam, coef, c, v, vx, vy, vz);
        if (has_dn) r -= cr * lam_g(I, lam, coef, dn, v, vx, vy, vz);
    } else {
        r = lam_g(I, lam, coef, c, v, vx, vy, vz);
    }
    out[(size_t)c * I.nv3 + v] = r;
}

// dJ/dU0[q][c] = sum_v lam^0 dM/dU_q with U = (rho, u, theta) from the conserved Uin
__global__ void __launch_bounds__(AT) k_adj_lift(Inst I, const double* lam, const double* Uin, double* dU0)
{
    __shared__ double sh[(AT / 32) * 5];
    const int c = blockIdx.x, nx = I.nx;
    const double rho = Uin[c], ux = Uin[nx + c] / rho, uy = Uin[2 * nx + c] / rho, uz = Uin[3 * nx + c] / rho;
    const double th = (2.0 * Uin[4 * nx + c] / rho - (ux * ux + uy * uy + uz * uz)) / 3.0;
    const double tp = 2.0 * PI * th, pref = rho / (tp * sqrt(tp));
    double s[5] = {0, 0, 0, 0, 0};
    for (int v = threadIdx.x; v < I.nv3; v += AT) {
        double vx, vy, vz;
        node(I, v, vx, vy, vz);
        double cx = vx - ux, cy = vy - uy, cz = vz - uz, c2 = cx * cx + cy * cy + cz * cz;
        double lM = lam[(size_t)c * I.nv3 + v] * pref * exp(-c2 / (2.0 * th));
        s[0] += lM / rho;
        s[1] += lM * cx / th;
        s[2] += lM * cy / th;
        s[3] += lM * cz / th;
        s[4] += lM * (c2 / (2.0 * th * th) - 1.5 / th);
    }
    block_sum<5>(s, sh);
    if (threadIdx.x < 5) dU0[(size_t)threadIdx.x * nx + c] = s[threadIdx.x];
}

// copy the float64 stored state g[cur] of instance b into dst [nx][ldv]
__global__ void k_copy_state(const Inst* insts, const InstState* st, int b, double* dst)
{
    const Inst& I = insts[b];
    const double* src = reinterpret_cast<const double*>(I.g[st[b].cur]);
    const size_t n = (size_t)I.nx * I.ldv;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        dst[k] = src[k];
}

}  // namespace

cudaError_t adj_seed(const Inst& I, const double* lamV, double* lam, cudaStream_t s)
{
    k_adj_seed<<<dim3(I.nx, (I.nv3 + AT - 1) / AT), AT, 0, s>>>(I, lamV, lam);
    return cudaGetLastError();
}

cudaError_t adj_moments(const Inst& I, const double* g, double* m, cudaStream_t s)
{
    k_adj_moments<<<I.nx, AT, 0, s>>>(I, g, m);
    return cudaGetLastError();
}

cudaError_t adj_step(const Inst& I, const double* lam_in, const double* g, const double* m, double* coef,
                     double* eps_acc, double* lam_out, cudaStream_t s)
{
    k_adj_coef<<<I.nx, AT, 0, s>>>(I, lam_in, g, m, coef, eps_acc);
    k_adj_apply<<<dim3(I.nx, (I.nv3 + AT - 1) / AT), AT, 0, s>>>(I, lam_in, coef, lam_out);
    return cudaGetLastError();
}

cudaError_t adj_lift(const Inst& I, const double* lam, const double* Uin, double* dU0, cudaStream_t s)
{
    k_adj_lift<<<I.nx, AT, 0, s>>>(I, lam, Uin, dU0);
    return cudaGetLastError();
}

cudaError_t adj_copy_state(const Inst* insts, const InstState* st, int b, double* dst, cudaStream_t s)
{
    k_copy_state<<<512, 256, 0, s>>>(insts, st, b, dst);
    return cudaGetLastError();
}

}  // namespace prk
