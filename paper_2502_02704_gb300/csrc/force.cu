// Fine propagator with an exterior force E != 0 (Laidin & Rey, arXiv
// 2502.02704: Eq. (11) with the force term, the fluxes of Eq. (13), Test 3).
//
// One fine step of the IMEX scheme on an anisotropic velocity grid (nvx cells
// along v_x, nvp along v_y and v_z, all on [-L, L]):
//   f*_ij = f_ij - dt/dx (F_{i+1/2,j} - F_{i-1/2,j}) - dt/dv_x (G_{i,j+1/2} - G_{i,j-1/2})
//   F: upwind, or MUSCL with minmod slopes, in x (Eq. 13, reading R1);
//   G_{i,a+1/2} = E_i/2 (f_a + f_{a+1}) - E_max/2 (f_{a+1} - f_a), zero through
//   v_x = -L and v_x = +L (the Rusanov reading of Eq. 13's garbled viscosity);
//   (rho, u, theta)_i = P(f*_i) (Eq. 18);  f^{n+1} = a f* + b M (a = eps/(eps+dt),
//   b = dt/(eps+dt), the implicit BGK step).
//
// A thread-block cluster of C CTAs owns one x column of one instance: each CTA
// takes a contiguous 1/C of the column's velocities, keeps f* in registers,
// reduces its five moment sums, and the cluster exchanges those partials
// through distributed shared memory (every CTA adds the C partials in rank
// order, so all see the same totals).  Each CTA then builds the separable
// Maxwellian tables, relaxes its cells and writes f^{n+1}; on the last step of
// a run a second exchange gives the projection P(f^{n+1}).  f is read once
// (neighbour columns come from L2) and written once per step: one launch per
// step, the step-to-step dependency being the stream order.
//
// Storage: f[b][buf][i][j], j = (jx*nvp + jy)*nvp + jz, float (mixed
// precision, moments and Maxwellian parameters in double) or double.
#include <cooperative_groups.h>
#include <math.h>

#include "pr_kernels.h"

namespace cg = cooperative_groups;

namespace prk {

namespace {

constexpr int FT = FORCE_THREADS;
constexpr int FW = FT / 32;

template <typename T>
__device__ __forceinline__ T minmod(T a, T b)
{
    if (a * b <= T(0)) return T(0);
    return (a < T(0) ? -a : a) < (b < T(0) ? -b : b) ? a : b;
}

// x cell c of the column range (ghosts -2..nx+1) under the boundary rule:
// returns the stored column and whether v_x is mirrored (reflecting wall).
__device__ __forceinline__ int ghost_col(int c, int nx, int bc, bool* mir)
{
    *mir = false;
    if (c >= 0 && c < nx) return c;
    if (bc == 0) return ((c % nx) + nx) % nx;
    if (bc == 1) return c < 0 ? 0 : nx - 1;
    *mir = true;
    return c < 0 ? -1 - c : 2 * nx - 1 - c;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float texp(float x) { return expf(x); }
__device__ __forceinline__ double texp(double x) { return exp(x); }

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Shared-memory layout of the step kernel.
struct FShared {
    double red[FW][5];   // per-warp partial sums
    double part[2][8];   // this CTA's partials, phase 0 (f*) and 1 (f^{n+1}); read by the cluster
    double par[8];       // rho, u_x, u_y, u_z, theta, pref, ok
};

// Sum of the CTA's 5 values s[] into sh.part[phase] (FP64 over warps).
template <typename T>
__device__ __forceinline__ void cta_partials(const T (&s)[5], FShared& sh, int phase)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        T v = warp_sum_t(s[q]);
        if (lane == 0) sh.red[w][q] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double a = 0.0;
        for (int k = 0; k < FW; ++k) a += sh.red[k][threadIdx.x];
        sh.part[phase][threadIdx.x] = a;
    }
}

// Cluster totals of part[phase], added in rank order (threads 0..4).
__device__ __forceinline__ double cluster_total(cg::cluster_group& cl, FShared& sh, int phase, int C)
{
    double a = 0.0;
    for (int r = 0; r < C; ++r) {
        const FShared* rs = cl.map_shared_rank(&sh, r);
        a += rs->part[phase][threadIdx.x];
    }
    return a;
}

template <typename T, int SCHEME>
__global__ void __launch_bounds__(FT)
k_force_step(const FInst* __restrict__ insts, FGeom g, const Active* __restrict__ act, int* __restrict__ cur,
             int step, int last, int* __restrict__ status)
{
    const int b = blockIdx.z;
    if (b < act->begin || b >= act->end) return;  // uniform over the cluster
    cg::cluster_group cl = cg::this_cluster();
    const FInst& I = insts[b];
    const int i = blockIdx.y, rank = blockIdx.x, C = gridDim.x;
    const int nvx = g.nvx, nvp = g.nvp, nvp2 = nvp * nvp;
    const long long ncol = g.ncol;

    extern __shared__ __align__(16) unsigned char fsm[];
    FShared& sh = *reinterpret_cast<FShared*>(fsm);
    T* vxs = reinterpret_cast<T*>(fsm + sizeof(FShared));  // velocity tables (copied from I.vtab)
    T* vy = vxs + nvx;
    T* vz = vy + nvp2;
    T* vp2 = vz + nvp2;
    T* eyz = vp2 + nvp2;  // Maxwellian tables
    T* ex = eyz + nvp2;
    T* st = ex + nvx;     // f* of this CTA's chunk

    const T* vt = static_cast<const T*>(I.vtab);
    for (int q = threadIdx.x; q < nvx + 3 * nvp2; q += FT) vxs[q] = vt[q];

    const int c0 = rank * g.chunk;
    const int c1 = (int)min((long long)c0 + g.chunk, ncol);
    const int bufi = cur[b] ^ (step & 1);
    const T* __restrict__ fin = static_cast<const T*>(I.f[bufi]);
    T* __restrict__ fout = static_cast<T*>(I.f[bufi ^ 1]);
    const T* col0 = fin + (size_t)i * ncol;

    // neighbour columns i-2 .. i+2 under the boundary rule
    const T* colp[5];
    bool mir[5];
    bool anymir = false;
#pragma unroll
    for (int d = -2; d <= 2; ++d) {
        bool m;
        int cc = ghost_col(i + d, I.nx, I.bc, &m);
        colp[d + 2] = fin + (size_t)cc * ncol;
        mir[d + 2] = m;
        anymir |= m;
    }
    const T nu = (T)I.nu, nuv = (T)I.nuv;
    const T Ei = (T)I.E[i], Em = (T)I.Emax, half = T(0.5);

    // this thread's cells e = c0 + t + k FT, (jx, jp) advanced without division
    const int e0 = c0 + threadIdx.x;
    const int dq = FT / nvp2, dr = FT - dq * nvp2;
    int jx = e0 / nvp2, jp = e0 - jx * nvp2;

    __syncthreads();
    T s[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll 2
    for (int e = e0; e < c1; e += FT) {
        const T vx = vxs[jx];
        const int jm = anymir ? (nvx - 1 - jx) * nvp2 + jp : e;
        const T c = col0[e];
        T Fr, Fl;
        if (SCHEME == 0) {
            if (vx > T(0)) {
                Fr = vx * c;
                Fl = vx * colp[1][mir[1] ? jm : e];
            } else {
                Fr = vx * colp[3][mir[3] ? jm : e];
                Fl = vx * c;
            }
        } else {
            const T m1 = colp[1][mir[1] ? jm : e], p1 = colp[3][mir[3] ? jm : e];
            if (vx > T(0)) {
                const T m2 = colp[0][mir[0] ? jm : e];
                Fr = vx * (c + half * minmod(c - m1, p1 - c));
                Fl = vx * (m1 + half * minmod(m1 - m2, c - m1));
            } else {
                const T p2 = colp[4][mir[4] ? jm : e];
                Fr = vx * (p1 - half * minmod(p1 - c, p2 - p1));
                Fl = vx * (c - half * minmod(c - m1, p1 - c));
            }
        }
        T Gr = T(0), Gl = T(0);
        if (jx < nvx - 1) {
            const T up = col0[e + nvp2];
            Gr = half * Ei * (c + up) - half * Em * (up - c);
        }
        if (jx > 0) {
            const T dn = col0[e - nvp2];
            Gl = half * Ei * (dn + c) - half * Em * (c - dn);
        }
        const T v = c - nu * (Fr - Fl) - nuv * (Gr - Gl);
        st[e - c0] = v;
        s[0] += v;
        s[1] += vx * v;
        s[2] += vy[jp] * v;
        s[3] += vz[jp] * v;
        s[4] += (vx * vx + vp2[jp]) * v;
        jp += dr;
        jx += dq;
        if (jp >= nvp2) {
            jp -= nvp2;
            ++jx;
        }
    }

    cta_partials(s, sh, 0);
    cl.sync();
    if (threadIdx.x < 5) sh.red[0][threadIdx.x] = cluster_total(cl, sh, 0, C);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double dv3 = I.dv3;
        double rho = sh.red[0][0] * dv3;
        double ux = sh.red[0][1] * dv3 / rho, uy = sh.red[0][2] * dv3 / rho, uz = sh.red[0][3] * dv3 / rho;
        double th = (sh.red[0][4] * dv3 / rho - (ux * ux + uy * uy + uz * uz)) / 3.0;
        bool ok = rho > 0.0 && th > 0.0 && isfinite(rho) && isfinite(th);
        if (!ok && rank == 0 && I.collide) atomicCAS(status, 0, ST_NONPHYS);
        sh.par[0] = rho;
        sh.par[1] = ux;
        sh.par[2] = uy;
        sh.par[3] = uz;
        sh.par[4] = ok ? th : 1.0;
        sh.par[5] = ok ? rho * pow(2.0 * 3.14159265358979323846 * th, -1.5) : 0.0;
    }
    __syncthreads();

    const T a = (T)I.a, bb = (T)I.b;
    const bool collide = I.collide != 0;
    if (collide) {
        // separable Maxwellian M = pref ex[jx] ey[jy] ez[jz], evaluated in T
        // from the double parameters
        const T ux = (T)sh.par[1], uy = (T)sh.par[2], uz = (T)sh.par[3];
        const T inv2th = (T)(0.5 / sh.par[4]), pref = (T)sh.par[5];
        for (int q = threadIdx.x; q < nvx; q += FT) {
            T cx = vxs[q] - ux;
            ex[q] = texp(-cx * cx * inv2th);
        }
        for (int q = threadIdx.x; q < nvp2; q += FT) {
            T cy = vy[q] - uy, cz = vz[q] - uz;
            eyz[q] = pref * texp(-cy * cy * inv2th) * texp(-cz * cz * inv2th);
        }
        __syncthreads();
    }

    T* out = fout + (size_t)i * ncol;
    T s2[5] = {T(0), T(0), T(0), T(0), T(0)};
    jx = e0 / nvp2;
    jp = e0 - jx * nvp2;
#pragma unroll 4
    for (int e = e0; e < c1; e += FT) {
        T v = st[e - c0];
        if (collide) v = a * v + bb * (ex[jx] * eyz[jp]);
        out[e] = v;
        if (last) {
            const T vx = vxs[jx];
            s2[0] += v;
            s2[1] += vx * v;
            s2[2] += vy[jp] * v;
            s2[3] += vz[jp] * v;
            s2[4] += (vx * vx + vp2[jp]) * v;
        }
        jp += dr;
        jx += dq;
        if (jp >= nvp2) {
            jp -= nvp2;
            ++jx;
        }
    }
    if (last) {
        cta_partials(s2, sh, 1);
        cl.sync();
        if (threadIdx.x < 5) {
            double t = cluster_total(cl, sh, 1, C) * I.dv3;
            if (threadIdx.x == 4) t *= 0.5;  // energy = 1/2 sum |v|^2 f dv
            if (rank == 0) {
                I.Ucur[threadIdx.x * I.nx + i] = t;
                if (I.Uout) I.Uout[threadIdx.x * I.nx + i] = t;
            }
        }
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

// Lift (Eq. 17) of the conserved state Uin into buffer 0 of the active
// instances; cur <- 0.
template <typename T>
__global__ void __launch_bounds__(FT)
k_force_lift(const FInst* __restrict__ insts, FGeom g, const Active* __restrict__ act, int* __restrict__ cur,
             int* __restrict__ status)
{
    const int b = blockIdx.z;
    if (b < act->begin || b >= act->end) return;
    const FInst& I = insts[b];
    const int i = blockIdx.y, nvx = g.nvx, nvp = g.nvp, nvp2 = nvp * nvp;
    extern __shared__ __align__(16) unsigned char fsm[];
    double* par = reinterpret_cast<double*>(fsm);
    T* ex = reinterpret_cast<T*>(fsm + 8 * sizeof(double));
    T* eyz = ex + nvx;
    const T* vt = static_cast<const T*>(I.vtab);  // vx[nvx], vy[nvp2], vz[nvp2]
    if (threadIdx.x == 0) {
        const int nx = I.nx;
        double rho = I.Uin[i], ux = I.Uin[nx + i] / rho, uy = I.Uin[2 * nx + i] / rho, uz = I.Uin[3 * nx + i] / rho;
        double th = (2.0 * I.Uin[4 * nx + i] / rho - (ux * ux + uy * uy + uz * uz)) / 3.0;
        bool ok = rho > 0.0 && th > 0.0 && isfinite(rho) && isfinite(th);
        if (!ok) atomicCAS(status, 0, ST_NONPHYS);
        par[1] = ux;
        par[2] = uy;
        par[3] = uz;
        par[4] = ok ? th : 1.0;
        par[5] = ok ? rho * pow(2.0 * 3.14159265358979323846 * th, -1.5) : 0.0;
        if (i == 0 && blockIdx.x == 0) cur[b] = 0;
    }
    __syncthreads();
    const T ux = (T)par[1], uy = (T)par[2], uz = (T)par[3], inv2th = (T)(0.5 / par[4]), pref = (T)par[5];
    for (int q = threadIdx.x; q < nvx; q += FT) {
        T cx = vt[q] - ux;
        ex[q] = texp(-cx * cx * inv2th);
    }
    for (int q = threadIdx.x; q < nvp2; q += FT) {
        T cy = vt[nvx + q] - uy, cz = vt[nvx + nvp2 + q] - uz;
        eyz[q] = pref * texp(-cy * cy * inv2th) * texp(-cz * cz * inv2th);
    }
    __syncthreads();
    T* out = static_cast<T*>(I.f[0]) + (size_t)i * g.ncol;
    const int c0 = blockIdx.x * g.chunk;
    const int c1 = min((long long)c0 + g.chunk, g.ncol);
    for (int e = c0 + threadIdx.x; e < c1; e += FT) {
        int jx = e / nvp2, jp = e - jx * nvp2;
        out[e] = ex[jx] * eyz[jp];
    }
}

// Conserved moments (Eq. 18) of the current state of instances [b0, b1) into
// Ucur: one CTA per (column, instance), double accumulation.
template <typename T>
__global__ void __launch_bounds__(FT)
k_force_moments(const FInst* __restrict__ insts, FGeom g, int b0, const int* __restrict__ cur)
{
    const int b = b0 + blockIdx.y;
    const FInst& I = insts[b];
    const int i = blockIdx.x, nvp = g.nvp, nvp2 = nvp * nvp;
    const T* f = static_cast<const T*>(I.f[cur[b]]) + (size_t)i * g.ncol;
    double s[5] = {0, 0, 0, 0, 0};
    for (long long e = threadIdx.x; e < g.ncol; e += FT) {
        int jx = (int)(e / nvp2), jp = (int)(e - (long long)jx * nvp2);
        int jy = jp / nvp, jz = jp - jy * nvp;
        double vx = -I.L + (jx + 0.5) * I.dvx, vy = -I.L + (jy + 0.5) * I.dvp, vz = -I.L + (jz + 0.5) * I.dvp;
        double v = (double)f[e];
        s[0] += v;
        s[1] += vx * v;
        s[2] += vy * v;
        s[3] += vz * v;
        s[4] += (vx * vx + vy * vy + vz * vz) * v;
    }
    __shared__ double red[FW][5];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double v = warp_sum(s[q]);
        if (lane == 0) red[w][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double a = 0.0;
        for (int k = 0; k < FW; ++k) a += red[k][threadIdx.x];
        a *= I.dv3;
        if (threadIdx.x == 4) a *= 0.5;
        I.Ucur[threadIdx.x * I.nx + i] = a;
    }
}

template <typename T>
__global__ void k_force_load(const FInst* __restrict__ insts, int b, const int* __restrict__ cur, const double* src,
                             long long n)
{
    T* dst = static_cast<T*>(insts[b].f[cur[b]]);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dst[e] = (T)src[e];
}

template <typename T>
__global__ void k_force_store(const FInst* __restrict__ insts, int b, const int* __restrict__ cur, double* dst,
                              long long n)
{
    const T* src = static_cast<const T*>(insts[b].f[cur[b]]);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dst[e] = (double)src[e];
}

__global__ void k_force_advance(const Active* __restrict__ act, int* __restrict__ cur, int nsteps)
{
    int b = act->begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (b < act->end) cur[b] ^= (nsteps & 1);
}

__global__ void k_force_set_cur(int* cur, int b, int v) { cur[b] = v; }

void* pick_step(int precision, int scheme)
{
    if (precision == 0) return scheme == 0 ? reinterpret_cast<void*>(&k_force_step<double, 0>)
                                           : reinterpret_cast<void*>(&k_force_step<double, 1>);
    return scheme == 0 ? reinterpret_cast<void*>(&k_force_step<float, 0>)
                       : reinterpret_cast<void*>(&k_force_step<float, 1>);
}

}  // namespace

size_t force_step_smem(int precision, int nvx, int nvp, int chunk)
{
    size_t es = precision == 0 ? sizeof(double) : sizeof(float);
    return sizeof(FShared) + ((size_t)4 * nvp * nvp + 2 * nvx + chunk) * es;
}

size_t force_lift_smem(int precision, int nvx, int nvp)
{
    size_t es = precision == 0 ? sizeof(double) : sizeof(float);
    return 8 * sizeof(double) + ((size_t)nvp * nvp + nvx) * es;
}

cudaError_t prepare_force_kernels(int max_smem)
{
    for (int p = 0; p < 2; ++p)
        for (int sc = 0; sc < 2; ++sc) {
            const void* fn = pick_step(p, sc);
            cudaFuncAttributes fa;
            if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
                cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - (int)fa.sharedSizeBytes);
            cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        }
    const void* lifts[2] = {reinterpret_cast<const void*>(&k_force_lift<double>),
                            reinterpret_cast<const void*>(&k_force_lift<float>)};
    for (const void* fn : lifts) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - (int)fa.sharedSizeBytes);
    }
    return cudaGetLastError();
}

int force_step_occupancy(int precision, int scheme, int C, size_t smem, int* clusters)
{
    const void* fn = pick_step(precision, scheme);
    if (!fn) return -1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(FT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    *clusters = n;
    return 0;
}

cudaError_t launch_force_step(int precision, int scheme, const FInst* insts, const FGeom& g, int nx, int n_inst,
                              const Active* act, int* cur, int step, int last, int* status, size_t smem,
                              cudaStream_t s)
{
    void* fn = pick_step(precision, scheme);
    if (!fn) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g.C, nx, n_inst);
    cfg.blockDim = dim3(FT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = g.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void* args[] = {(void*)&insts, (void*)&g, (void*)&act, (void*)&cur, (void*)&step, (void*)&last, (void*)&status};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_force_lift(int precision, const FInst* insts, const FGeom& g, int nx, int n_inst,
                              const Active* act, int* cur, int* status, cudaStream_t s)
{
    dim3 grid(g.C, nx, n_inst);
    size_t smem = force_lift_smem(precision, g.nvx, g.nvp);
    if (precision == 0) k_force_lift<double><<<grid, FT, smem, s>>>(insts, g, act, cur, status);
    else k_force_lift<float><<<grid, FT, smem, s>>>(insts, g, act, cur, status);
    return cudaGetLastError();
}

cudaError_t launch_force_moments(int precision, const FInst* insts, const FGeom& g, int nx, int b0, int b1,
                                 const int* cur, cudaStream_t s)
{
    if (b1 <= b0) return cudaSuccess;
    dim3 grid(nx, b1 - b0);
    if (precision == 0) k_force_moments<double><<<grid, FT, 0, s>>>(insts, g, b0, cur);
    else k_force_moments<float><<<grid, FT, 0, s>>>(insts, g, b0, cur);
    return cudaGetLastError();
}

cudaError_t launch_force_load(int precision, const FInst* insts, int b, const int* cur, const double* src,
                              long long n, cudaStream_t s)
{
    int grid = (int)std::min<long long>((n + 255) / 256, 4096);
    if (precision == 0) k_force_load<double><<<grid, 256, 0, s>>>(insts, b, cur, src, n);
    else k_force_load<float><<<grid, 256, 0, s>>>(insts, b, cur, src, n);
    return cudaGetLastError();
}

cudaError_t launch_force_store(int precision, const FInst* insts, int b, const int* cur, double* dst, long long n,
                               cudaStream_t s)
{
    int grid = (int)std::min<long long>((n + 255) / 256, 4096);
    if (precision == 0) k_force_store<double><<<grid, 256, 0, s>>>(insts, b, cur, dst, n);
    else k_force_store<float><<<grid, 256, 0, s>>>(insts, b, cur, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_force_advance(const Active* act, int* cur, int nsteps, int n_inst, cudaStream_t s)
{
    if (!(nsteps & 1)) return cudaSuccess;
    k_force_advance<<<(n_inst + 127) / 128, 128, 0, s>>>(act, cur, nsteps);
    return cudaGetLastError();
}

cudaError_t launch_force_set_cur(int* cur, int b, int v, cudaStream_t s)
{
    k_force_set_cur<<<1, 1, 0, s>>>(cur, b, v);
    return cudaGetLastError();
}

}  // namespace prk
