// First-order lifting L^(1) of Def. 3 (Laidin & Rey, arXiv 2502.02704,
// Remark 1, L = 1) for both fine paths:
//   f = M (1 - eps P(c)),  c = v - u,
//   P(c) = (c_x (c . du) - |c|^2 du_x / 3) / theta + c_x (|c|^2 / (2 theta) - 5/2) dtheta / theta,
// the first Chapman-Enskog correction g1 = -(d_t + v d_x) M of the BGK model
// with the Euler time derivatives (an exterior force cancels in g1).  The
// gradients of u and theta are central differences of the cell values through
// the boundary ghosts (periodic wrap, outflow copy, reflecting mirror with u_x
// negated).
//
// E = 0 path: the lifted f is written as a general state of the fine kernel
// (g = f, zero factor tables, weight a0 = 1), so the first fine step reads it
// like a loaded distribution.  Force path: written into buffer 0, cur <- 0.
#include <math.h>

#include "pr_kernels.h"

namespace prk {

namespace {

constexpr int LT = 256;  // threads per CTA

// Primitive state (rho, u_x, u_y, u_z, theta) of cell c (ghosts allowed) from
// a conserved [5][nx] array, through the boundary rule.
__device__ __forceinline__ void prim_cell(const double* V, int nx, int bc, int c, double* p)
{
    int cc = c;
    bool flip = false;
    if (c < 0 || c >= nx) {
        if (bc == 0) cc = ((c % nx) + nx) % nx;
        else if (bc == 1) cc = c < 0 ? 0 : nx - 1;
        else {
            cc = c < 0 ? -1 - c : 2 * nx - 1 - c;
            flip = true;
        }
    }
    const double rho = V[cc], ux = V[nx + cc] / rho, uy = V[2 * nx + cc] / rho, uz = V[3 * nx + cc] / rho;
    p[0] = rho;
    p[1] = flip ? -ux : ux;
    p[2] = uy;
    p[3] = uz;
    p[4] = (2.0 * V[4 * nx + cc] / rho - (ux * ux + uy * uy + uz * uz)) / 3.0;
}

// Parameters of column c: q[0..4] = (pref, u_x, u_y, u_z, theta), q[5..8] =
// eps * (du_x, du_y, du_z, dtheta) / theta, q[9] = 1 / (2 theta).
__device__ __forceinline__ void column_params(const double* V, int nx, int bc, double dx, double eps, int c,
                                              double* q, int* status)
{
    double pm[5], p0[5], pp[5];
    prim_cell(V, nx, bc, c - 1, pm);
    prim_cell(V, nx, bc, c, p0);
    prim_cell(V, nx, bc, c + 1, pp);
    const double rho = p0[0], th = p0[4];
    if (!(rho > 0.0) || !(th > 0.0)) atomicCAS(status, 0, ST_NONPHYS);
    const double tp = 2.0 * 3.14159265358979323846 * th;
    q[0] = rho / (tp * sqrt(tp));
    q[1] = p0[1];
    q[2] = p0[2];
    q[3] = p0[3];
    q[4] = th;
    for (int k = 0; k < 4; ++k) q[5 + k] = eps * (pp[1 + k] - pm[1 + k]) / (2.0 * dx) / th;
    q[9] = 0.5 / th;
}

// f at velocity (vx, vy, vz) of a column with parameters q (T arithmetic).
template <typename T>
__device__ __forceinline__ T ce_value(const T* q, T vx, T vy, T vz)
{
    const T cx = vx - q[1], cy = vy - q[2], cz = vz - q[3];
    const T c2 = cx * cx + cy * cy + cz * cz;
    const T M = q[0] * (sizeof(T) == sizeof(double) ? (T)exp((double)(-c2 * q[9])) : (T)expf((float)(-c2 * q[9])));
    // eps P(c) with the gradients already scaled by eps / theta
    const T P = cx * (cx * q[5] + cy * q[6] + cz * q[7]) - c2 * q[5] * (T)(1.0 / 3.0) +
                cx * (c2 * q[9] - (T)2.5) * q[8];
    return M * ((T)1 - P);
}

// E = 0 path: one CTA per (x cell, velocity chunk, active instance).
template <typename T>
__global__ void __launch_bounds__(LT)
k_lift_ce(const Inst* __restrict__ insts, InstState* st, const Active* __restrict__ act, int* status)
{
    const int b = act->begin + blockIdx.z;
    if (b >= act->end) return;
    const Inst& I = insts[b];
    const int c = blockIdx.x;
    if (c >= I.nx) return;
    __shared__ T q[10];
    if (threadIdx.x == 0) {
        double qd[10];
        column_params(I.Uin, I.nx, I.bc, I.dx, I.eps, c, qd, status);
        for (int k = 0; k < 10; ++k) q[k] = (T)qd[k];
    }
    __syncthreads();
    const int cur = st[b].cur, nv = I.nv;
    T* g = static_cast<T*>(I.g[cur]) + (size_t)c * I.ldv;
    for (int v = blockIdx.y * LT + threadIdx.x; v < I.nv3; v += gridDim.y * LT) {
        const int jz = v % nv, jy = (v / nv) % nv, jx = v / (nv * nv);
        const T vx = (T)(-I.L + (jx + 0.5) * I.dv), vy = (T)(-I.L + (jy + 0.5) * I.dv),
                vz = (T)(-I.L + (jz + 0.5) * I.dv);
        g[v] = ce_value<T>(q, vx, vy, vz);
    }
    if (blockIdx.y == 0) {
        T* tb = static_cast<T*>(I.tab[cur]) + (size_t)c * 3 * nv;  // the lazy Maxwellian term is zero
        for (int k = threadIdx.x; k < 3 * nv; k += LT) tb[k] = T(0);
        if (c == 0 && threadIdx.x == 0) st[b].a0 = 1.0;
    }
}

// Conserved moments (Eq. 18) of the state g of each active instance into Ucur
// (one CTA per (x cell, instance), double accumulation).
template <typename T>
__global__ void __launch_bounds__(LT)
k_lift_moments(const Inst* __restrict__ insts, const InstState* __restrict__ st, const Active* __restrict__ act)
{
    const int b = act->begin + blockIdx.y;
    if (b >= act->end) return;
    const Inst& I = insts[b];
    const int c = blockIdx.x;
    if (c >= I.nx) return;
    const int nv = I.nv;
    const T* g = static_cast<const T*>(I.g[st[b].cur]) + (size_t)c * I.ldv;
    double a[5] = {0, 0, 0, 0, 0};
    for (int v = threadIdx.x; v < I.nv3; v += LT) {
        const int jz = v % nv, jy = (v / nv) % nv, jx = v / (nv * nv);
        const double vx = -I.L + (jx + 0.5) * I.dv, vy = -I.L + (jy + 0.5) * I.dv, vz = -I.L + (jz + 0.5) * I.dv;
        const double f = (double)g[v];
        a[0] += f;
        a[1] += vx * f;
        a[2] += vy * f;
        a[3] += vz * f;
        a[4] += (vx * vx + vy * vy + vz * vz) * f;
    }
    __shared__ double red[LT / 32][5];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
#pragma unroll
        for (int o = 16; o; o >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
        if (lane == 0) red[w][k] = a[k];
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0.0;
        for (int k = 0; k < LT / 32; ++k) t += red[k][threadIdx.x];
        t *= I.dv3;
        if (threadIdx.x == 4) t *= 0.5;
        I.Ucur[(size_t)threadIdx.x * I.nx + c] = t;
    }
}

// Force path: one CTA per (velocity chunk, x cell, active instance) of the
// anisotropic grid, written into buffer 0.
template <typename T>
__global__ void __launch_bounds__(LT)
k_force_lift_ce(const FInst* __restrict__ insts, FGeom gm, const Active* __restrict__ act, int* __restrict__ cur,
                int* __restrict__ status)
{
    const int b = blockIdx.z;
    if (b < act->begin || b >= act->end) return;
    const FInst& I = insts[b];
    const int i = blockIdx.y, nvp = gm.nvp, nvp2 = nvp * nvp;
    __shared__ T q[10];
    if (threadIdx.x == 0) {
        double qd[10];
        column_params(I.Uin, I.nx, I.bc, I.dx, I.eps, i, qd, status);
        for (int k = 0; k < 10; ++k) q[k] = (T)qd[k];
        if (i == 0 && blockIdx.x == 0) cur[b] = 0;
    }
    __syncthreads();
    const T* vt = static_cast<const T*>(I.vtab);  // v_x[nvx], v_y[nvp2], v_z[nvp2]
    T* out = static_cast<T*>(I.f[0]) + (size_t)i * gm.ncol;
    for (long long e = (long long)blockIdx.x * LT + threadIdx.x; e < gm.ncol; e += (long long)gridDim.x * LT) {
        const int jx = (int)(e / nvp2), jp = (int)(e - (long long)jx * nvp2);
        out[e] = ce_value<T>(q, vt[jx], vt[gm.nvx + jp], vt[gm.nvx + nvp2 + jp]);
    }
}

}  // namespace

cudaError_t launch_lift_ce(int precision, const Inst* insts, InstState* st, const Active* active, int nx_max,
                           int n_inst_max, int with_moments, int* status, cudaStream_t s)
{
    dim3 grid(nx_max, 8, n_inst_max);
    if (precision == 0) k_lift_ce<double><<<grid, LT, 0, s>>>(insts, st, active, status);
    else k_lift_ce<float><<<grid, LT, 0, s>>>(insts, st, active, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !with_moments) return e;
    dim3 g2(nx_max, n_inst_max);
    if (precision == 0) k_lift_moments<double><<<g2, LT, 0, s>>>(insts, st, active);
    else k_lift_moments<float><<<g2, LT, 0, s>>>(insts, st, active);
    return cudaGetLastError();
}

cudaError_t launch_force_lift_ce(int precision, const FInst* insts, const FGeom& g, int nx, int n_inst,
                                 const Active* act, int* cur, int* status, cudaStream_t s)
{
    const int chunks = (int)((g.ncol + LT * 16 - 1) / (LT * 16));
    dim3 grid(chunks, nx, n_inst);
    if (precision == 0) k_force_lift_ce<double><<<grid, LT, 0, s>>>(insts, g, act, cur, status);
    else k_force_lift_ce<float><<<grid, LT, 0, s>>>(insts, g, act, cur, status);
    return cudaGetLastError();
}

}  // namespace prk
