// Coarse fluid propagator G and the sequential parareal correction on the
// device (Laidin & Rey, arXiv 2502.02704).
//
// G: the Euler system of Eq. (14) in conserved variables V = (rho, rho u, E),
// explicit update of Eq. (15) with the Rusanov flux of Eq. (16) read as
//   H_{i+1/2} = (h(V_i) + h(V_{i+1}))/2 - S_{i+1/2} (V_{i+1} - V_i)/2,
//   S_{i+1/2} = max(|u_x| + c) over the two cells, c = sqrt(5 theta/3) (or the
//   printed sqrt(theta)), local steps dt = min(cfl dx / max S, remaining) until
//   the coarse interval is covered (Sec. 2.2).  Ghost cells: periodic wrap,
//   outflow copy, reflecting mirror with rho u_x negated.
// With an exterior force E (Eq. 5) each local step adds dt (0, rho E_i, 0, 0,
// rho u_x E_i) evaluated on the state before the step.  With visc = eps > 0
// the model is the compressible Navier-Stokes system of Eq. (8): viscous
// fluxes with mu = rho theta and kappa = 5 rho theta / 2 added to the Rusanov
// flux, local steps also limited by dx^2 / (2 eps (5/3) max theta).
// Sweep: Algorithm 2's sequential loop U^{n,k} = G(U^{n-1,k}) + jump^n for
// n = k..N, with jump^n = PFL(U^{n-1,k-1}) - G(U^{n-1,k-1}) formed from the
// stored G results of the previous sweep, and the Eq. (10) error
// max |U^{n,k} - U^{n,k-1}| reduced in the same pass.
//
// One thread-block cluster runs the whole sweep (the loop over n is
// sequential by nature), its CTAs owning contiguous blocks of cells in their
// shared memory (or global regions when the blocks do not fit).  This file
// is compiled without floating-point contraction so that the arithmetic is
// the plain IEEE sequence of the formulas above (with rho's reciprocal times
// the momenta for the primitive variables).
#include <cooperative_groups.h>
#include <math.h>

#include "pr_kernels.h"

namespace cg = cooperative_groups;

namespace prk {

namespace {

constexpr int CT = 256;  // threads per coarse CTA at most (cells beyond loop)

struct Prim {
    double ux, uy, uz, p, th;
};

// Primitive variables of a conserved state with one reciprocal of rho (the
// quotients v/rho as products with 1/rho: within an ulp of the divisions,
// and a much shorter dependent chain on this part's FP64 pipe).
__device__ __forceinline__ Prim prim(const double* v)
{
    Prim q;
    const double rinv = 1.0 / v[0];
    q.ux = v[1] * rinv;
    q.uy = v[2] * rinv;
    q.uz = v[3] * rinv;
    q.th = (2.0 * v[4] * rinv - (q.ux * q.ux + q.uy * q.uy + q.uz * q.uz)) * (1.0 / 3.0);
    q.p = v[0] * q.th;
    return q;
}

__device__ double block_max(double v, double* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    for (int k = 0; k < nw; ++k) r = fmax(r, sh[k]);
    return r;
}

// Two maxima over the CTA in one pass (sh holds 2 doubles per warp).
__device__ void block_max2(double& a, double& b, double* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    __syncthreads();
    if (lane == 0) {
        sh[2 * warp] = a;
        sh[2 * warp + 1] = b;
    }
    __syncthreads();
    double ra = 0.0, rb = 0.0;
    for (int k = 0; k < nw; ++k) {
        ra = fmax(ra, sh[2 * k]);
        rb = fmax(rb, sh[2 * k + 1]);
    }
    a = ra;
    b = rb;
}

// Per-cell values of one substep, computed once from the state before it:
// u_x, u_y, u_z, theta, p, the Euler flux h (5) and the wave speed, stored
// [NCACHE][nx].  A face then combines two cached cells; a reflecting ghost
// (rho u_x negated) has u_x and h_0, h_2, h_3, h_4 negated, which is exactly
// what the same formulas give on the mirrored state.
constexpr int NCACHE = 11;

struct CellF {
    double v[5], ux, uy, uz, th, p, h[5], s;
};

// Region of one cluster CTA (m cells): state A[5][m], next state B[5][m],
// cell cache [NCACHE][m], then 2 doubles of the CTA's CFL maxima.  Lives in
// the CTA's shared memory, or in a global workspace (one region per CTA)
// when m cells do not fit; peers read it through distributed shared memory
// or plainly, ordered by the cluster barriers.
__host__ __device__ inline size_t region_doubles(int m) { return (size_t)(10 + NCACHE) * m + 2; }

struct Peers {
    double* base;      // this CTA's region
    double* gbase;     // global regions (when not in shared memory)
    size_t region;     // doubles per region
    int rank, m;
    bool smem;
    __device__ __forceinline__ double* of(cg::cluster_group& cl, int r) const
    {
        if (r == rank) return base;
        return smem ? cl.map_shared_rank(base, r) : gbase + (size_t)r * region;
    }
};

// Cell c of the whole domain (ghosts through the boundary rule) from the
// state at offset cur_off and the cache of its owner.
__device__ __forceinline__ void fetch(cg::cluster_group& cl, const Peers& P, int cur_off, int nx, int bc, int c,
                                      CellF& o)
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
    const int m = P.m, b0 = P.rank * m;
    int owner, li;
    if (cc >= b0 && cc < b0 + m) owner = P.rank, li = cc - b0;              // own block
    else if (cc == b0 - 1) owner = P.rank - 1, li = m - 1;                  // left neighbour block
    else if (cc == b0 + m) owner = P.rank + 1, li = 0;                      // right neighbour block
    else owner = cc / m, li = cc - owner * m;                               // a wrapped or mirrored ghost
    const double* R = P.of(cl, owner);
    const double* V = R + cur_off;
    const double* Cc = R + 10 * m;
#pragma unroll
    for (int q = 0; q < 5; ++q) o.v[q] = V[q * m + li];
    o.ux = Cc[li];
    o.uy = Cc[m + li];
    o.uz = Cc[2 * m + li];
    o.th = Cc[3 * m + li];
    o.p = Cc[4 * m + li];
#pragma unroll
    for (int q = 0; q < 5; ++q) o.h[q] = Cc[(5 + q) * m + li];
    o.s = Cc[10 * m + li];
    if (flip) {
        o.v[1] = -o.v[1];
        o.ux = -o.ux;
        o.h[0] = -o.h[0];
        o.h[2] = -o.h[2];
        o.h[3] = -o.h[3];
        o.h[4] = -o.h[4];
    }
}

// Flux through the face between cells a and b: Rusanov (Eq. 16) plus, when
// eps > 0, the viscous flux of the compressible Navier-Stokes model (Eq. 8)
// with mu = rho theta, kappa = 5 rho theta / 2, gradients (b - a)/dx (idx =
// 1/dx) and coefficients and u averaged over the face.
__device__ __forceinline__ void face_flux(const CellF& a, const CellF& b, double visc, double idx, double* H)
{
    const double S = a.s > b.s ? a.s : b.s;
#pragma unroll
    for (int q = 0; q < 5; ++q) H[q] = 0.5 * (a.h[q] + b.h[q]) - 0.5 * S * (b.v[q] - a.v[q]);
    if (visc > 0.0) {
        const double eps = visc;
        double mu = 0.5 * (a.p + b.p);
        double kappa = 2.5 * mu;
        double dux = (b.ux - a.ux) * idx, duy = (b.uy - a.uy) * idx, duz = (b.uz - a.uz) * idx, dth = (b.th - a.th) * idx;
        double ux = 0.5 * (a.ux + b.ux), uy = 0.5 * (a.uy + b.uy), uz = 0.5 * (a.uz + b.uz);
        double sxx = -eps * mu * (4.0 / 3.0) * dux, sxy = -eps * mu * duy, sxz = -eps * mu * duz;
        double qh = -eps * kappa * dth;
        H[0] += 0.0;
        H[1] += sxx;
        H[2] += sxy;
        H[3] += sxz;
        H[4] += sxx * ux + sxy * uy + sxz * uz + qh;
    }
}

// G over dT applied to this CTA's cells [c0, c1) of the state at region
// offset 0 (A), with the other CTAs of the cluster doing theirs; the result
// ends in A.  Per local step: one pass caching each own cell's primitives,
// flux and speed and its CTA's two CFL maxima, a cluster barrier, the
// cluster maxima, one pass forming each own cell's two face fluxes (peer
// cells through the owners' regions) and its update into B, a cluster
// barrier; A and B swap roles.  Every CTA takes the same local steps.
// (Forming each face once into a face array, with one more CTA barrier,
// measured no faster: the step is a chain of dependent FP64 operations.)
__device__ void coarse_G(const CoarseParams& p, cg::cluster_group& cl, const Peers& P, int C, int c0, int c1,
                         double dT, int* status, double* sh)
{
    const int nx = p.nx, m = P.m, mc = c1 - c0;
    double* R = P.base;
    double* Cc = R + 10 * m;
    double* red = R + (10 + NCACHE) * m;
    int cur_off = 0, nxt_off = 5 * m;
    const double idx = 1.0 / p.dx;
    double t = 0.0;
    while (t < dT) {
        const double* cur = R + cur_off;
        double smax = 0.0, thmax = 0.0;
        bool bad = false;
        for (int li = threadIdx.x; li < mc; li += blockDim.x) {
            double v[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) v[q] = cur[q * m + li];
            Prim pr = prim(v);
            if (!(v[0] > 0.0) || !(pr.th > 0.0)) bad = true;
            double c = p.sound == 1 ? sqrt(pr.th) : sqrt(pr.th * (5.0 / 3.0));
            double s = fabs(pr.ux) + c;
            if (s > smax) smax = s;
            if (pr.th > thmax) thmax = pr.th;
            Cc[li] = pr.ux;
            Cc[m + li] = pr.uy;
            Cc[2 * m + li] = pr.uz;
            Cc[3 * m + li] = pr.th;
            Cc[4 * m + li] = pr.p;
            Cc[5 * m + li] = v[1];
            Cc[6 * m + li] = v[1] * pr.ux + pr.p;
            Cc[7 * m + li] = v[1] * pr.uy;
            Cc[8 * m + li] = v[1] * pr.uz;
            Cc[9 * m + li] = pr.ux * (v[4] + pr.p);
            Cc[10 * m + li] = s;
        }
        if (bad) atomicCAS(status, 0, ST_NONPHYS);
        block_max2(smax, thmax, sh);
        if (threadIdx.x == 0) {
            red[0] = smax;
            red[1] = thmax;
        }
        cl.sync();  // caches, states and CTA maxima of every rank visible
        for (int r = 0; r < C; ++r) {
            const double* rr = P.of(cl, r) + (10 + NCACHE) * m;
            smax = fmax(smax, rr[0]);
            thmax = fmax(thmax, rr[1]);
        }
        if (!(smax > 0.0) || isnan(smax)) break;  // the same on every rank
        double rem = dT - t;
        double dt = p.cfl * p.dx / smax;
        if (p.visc > 0.0) {
            double dtv = p.cfl * p.dx * p.dx / (2.0 * p.visc * (5.0 / 3.0) * thmax);
            if (dtv < dt) dt = dtv;
        }
        bool last = false;
        if (dt >= rem) {
            dt = rem;
            last = true;
        }
        double* nxt = R + nxt_off;
        const double dtdx = dt / p.dx;
        for (int li = threadIdx.x; li < mc; li += blockDim.x) {
            const int i = c0 + li;
            CellF L, M, Rt;
            fetch(cl, P, cur_off, nx, p.bc, i - 1, L);
            fetch(cl, P, cur_off, nx, p.bc, i, M);
            fetch(cl, P, cur_off, nx, p.bc, i + 1, Rt);
            double Hl[5], Hr[5];
            face_flux(L, M, p.visc, idx, Hl);
            face_flux(M, Rt, p.visc, idx, Hr);
#pragma unroll
            for (int q = 0; q < 5; ++q) nxt[q * m + li] = cur[q * m + li] - dtdx * (Hr[q] - Hl[q]);
            if (p.E) {  // exterior force: forward-Euler source on the old state
                nxt[1 * m + li] += dt * cur[0 * m + li] * p.E[i];
                nxt[4 * m + li] += dt * cur[1 * m + li] * p.E[i];
            }
        }
        cl.sync();  // every rank's reads of the old states and caches are over
        const int tmp = cur_off;
        cur_off = nxt_off;
        nxt_off = tmp;
        if (last) break;
        t += dt;
    }
    if (cur_off != 0) {
        for (int li = threadIdx.x; li < mc; li += blockDim.x)
#pragma unroll
            for (int q = 0; q < 5; ++q) R[q * m + li] = R[cur_off + q * m + li];
        __syncthreads();
    }
}

__device__ __forceinline__ Peers make_peers(double* dsm, double* work, int use_smem, int m)
{
    Peers P;
    P.region = region_doubles(m);
    P.rank = (int)blockIdx.x;
    P.m = m;
    P.smem = use_smem != 0;
    P.gbase = work;
    P.base = P.smem ? dsm : work + (size_t)blockIdx.x * P.region;
    return P;
}

// One G over dT of Vin (device [5][nx]) into Vout; one cluster of C CTAs.
__global__ void __launch_bounds__(CT)
k_coarse(CoarseParams p, const double* Vin, double* Vout, double dT, double* work, int use_smem, int* status)
{
    extern __shared__ __align__(16) double dsm[];
    __shared__ double sh[2 * (CT / 32)];
    cg::cluster_group cl = cg::this_cluster();
    const int nx = p.nx, C = gridDim.x, m = (nx + C - 1) / C;
    const int c0 = (int)blockIdx.x * m, c1 = min(nx, c0 + m);
    const Peers P = make_peers(dsm, work, use_smem, m);
    for (int li = threadIdx.x; li < c1 - c0; li += blockDim.x)
#pragma unroll
        for (int q = 0; q < 5; ++q) P.base[q * m + li] = Vin[q * nx + c0 + li];
    __syncthreads();
    coarse_G(p, cl, P, C, c0, c1, dT, status, sh);
    for (int li = threadIdx.x; li < c1 - c0; li += blockDim.x)
#pragma unroll
        for (int q = 0; q < 5; ++q) Vout[q * nx + c0 + li] = P.base[q * m + li];
    cl.sync();  // no CTA leaves while another may still read its region
}

// Algorithm 2's sequential sweep over n = max(k,1)..N on one cluster of C
// CTAs, each owning a contiguous block of cells.
__global__ void __launch_bounds__(CT)
k_sweep(CoarseParams p, int N, double dT, const int* dk, double* U, const double* PFL, double* Gs, double* err,
        double* work, int use_smem, int* status, int bump, int* dk_mut)
{
    extern __shared__ __align__(16) double dsm[];
    __shared__ double sh[2 * (CT / 32)];
    cg::cluster_group cl = cg::this_cluster();
    const int nx = p.nx, sz = 5 * nx, C = gridDim.x, m = (nx + C - 1) / C;
    const int c0 = (int)blockIdx.x * m, c1 = min(nx, c0 + m), mc = c1 - c0;
    const int k = *dk;
    const Peers P = make_peers(dsm, work, use_smem, m);
    double* A = P.base;
    double emax = 0.0;
    for (int n = (k > 1 ? k : 1); n <= N; ++n) {
        for (int li = threadIdx.x; li < mc; li += blockDim.x)
#pragma unroll
            for (int q = 0; q < 5; ++q) A[q * m + li] = U[(size_t)(n - 1) * sz + q * nx + c0 + li];
        __syncthreads();
        coarse_G(p, cl, P, C, c0, c1, dT, status, sh);
        for (int li = threadIdx.x; li < mc; li += blockDim.x)
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const size_t o = (size_t)n * sz + q * nx + c0 + li;
                double gv = A[q * m + li];
                double nv = k > 0 ? gv + (PFL[o] - Gs[o]) : gv;
                double d = fabs(nv - U[o]);
                if (d > emax) emax = d;
                U[o] = nv;
                Gs[o] = gv;
            }
        __syncthreads();
    }
    // the error of the iteration: max over the cluster
    double dummy = 0.0;
    block_max2(emax, dummy, sh);
    double* red = P.base + (10 + NCACHE) * m;
    if (threadIdx.x == 0) red[0] = emax;
    cl.sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double e = 0.0;
        for (int r = 0; r < C; ++r) e = fmax(e, P.of(cl, r)[(10 + NCACHE) * m]);
        err[k] = e;
        if (bump) *dk_mut = k + 1;
    }
    cl.sync();  // no CTA leaves while another may still read its region
}

__global__ void k_set_active(const int* dk, Active* a, int first_slice, int n_inst, int N)
{
    // slices n = max(k,1)..N are active; instance b runs slice first_slice + b
    int k = *dk;
    int lo = (k > 1 ? k : 1) - first_slice;
    if (lo < 0) lo = 0;
    int hi = N - first_slice + 1;
    if (hi > n_inst) hi = n_inst;
    if (lo > hi) lo = hi;
    a->begin = lo;
    a->end = hi;
}

// CTAs of the coarse cluster: blocks of about 32 cells (one warp each; the
// local steps are chains of dependent FP64 operations, so a block's cells
// share an SM's FP64 pipe with no other warp), at most 16 CTAs, none empty
// (C = ceil(nx / m) for the block size m).
int coarse_ctas(int nx)
{
    const int C0 = nx >= 512 ? 16 : nx > 32 ? (nx + 31) / 32 : 1;
    const int m = (nx + C0 - 1) / C0;
    return (nx + m - 1) / m;
}

// Doubles of global workspace of a coarse step (one region per CTA).
size_t work_doubles(int nx)
{
    const int C = coarse_ctas(nx), m = (nx + C - 1) / C;
    return (size_t)C * region_doubles(m);
}

bool fits_smem(int nx)
{
    const int C = coarse_ctas(nx), m = (nx + C - 1) / C;
    return region_doubles(m) * sizeof(double) <= 200 * 1024;
}

template <typename... Args>
cudaError_t launch_cluster(void (*fn)(Args...), int nx, cudaStream_t s, Args... args)
{
    const int C = coarse_ctas(nx), m = (nx + C - 1) / C;
    const int use = fits_smem(nx);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(m < CT ? (m + 31) / 32 * 32 : CT, 1, 1);
    cfg.dynamicSmemBytes = use ? region_doubles(m) * sizeof(double) : 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, args...);
}

}  // namespace

void prepare_coarse_kernels(int max_smem)
{
    const void* fns[2] = {reinterpret_cast<const void*>(&k_coarse), reinterpret_cast<const void*>(&k_sweep)};
    for (const void* fn : fns) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - (int)fa.sharedSizeBytes);
        cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaGetLastError();
    }
}

cudaError_t launch_coarse(const CoarseParams& p, const double* Vin, double* Vout, double dT, double* work,
                          int* status, cudaStream_t s)
{
    return launch_cluster(k_coarse, p.nx, s, p, Vin, Vout, dT, work, (int)fits_smem(p.nx), status);
}

cudaError_t launch_sweep(const CoarseParams& p, int N, double dT, const int* dk, double* U, const double* PFL,
                         double* Gs, double* err, double* work, int* status, int bump, int* dk_mut,
                         cudaStream_t s)
{
    return launch_cluster(k_sweep, p.nx, s, p, N, dT, dk, U, PFL, Gs, err, work, (int)fits_smem(p.nx), status,
                          bump, dk_mut);
}

size_t coarse_work_doubles(int nx) { return work_doubles(nx); }

cudaError_t launch_set_active(const int* dk, Active* active, int first_slice, int n_inst, int N, cudaStream_t s)
{
    k_set_active<<<1, 1, 0, s>>>(dk, active, first_slice, n_inst, N);
    return cudaGetLastError();
}

}  // namespace prk
