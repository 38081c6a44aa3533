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
// shared memory (or global regions when the blocks do not fit).  The
// compiler may contract products and sums into fused multiply-adds (one
// rounding each, fewer instructions on this part's narrow FP64 pipe); with
// rho's reciprocal times the momenta for the primitive variables, the result
// agrees with the plain sequence of the formulas above to ~1e-15 relative.
#include <algorithm>
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
// the Euler flux h (5) and the wave speed s, then for the Navier-Stokes
// model u_x, u_y, u_z, theta and p, stored [NCACHE][m].  A face combines two
// cells; a reflecting ghost (rho u_x negated) has u_x and h_0, h_2, h_3, h_4
// negated, which is exactly what the same formulas give on the mirrored
// state.  Substeps alternate between two caches (and two slots of CFL
// maxima), so a CTA fills the next cache while its peers may still read the
// current one: one cluster barrier per substep orders everything.
constexpr int NCACHE = 11;
constexpr int NRED = 4;  // (max speed, max theta) for each of the two caches
constexpr unsigned long long SIGN = 0x8000000000000000ull;

// Region of one cluster CTA (m cells): states A[5][m] and B[5][m], caches
// K0 and K1 [NCACHE][m], the CFL maxima of K0 and K1, then the CTA's face
// fluxes [5][m+1].  Lives in the CTA's shared memory, or in a global
// workspace (one region per CTA) when m cells do not fit; peers read states
// and caches through distributed shared memory or plainly, ordered by the
// cluster barriers.
__host__ __device__ inline size_t region_doubles(int m) { return (size_t)(15 + 2 * NCACHE) * m + NRED + 5; }

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

__device__ __forceinline__ double flip_sign(double x, unsigned long long mask)
{
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)mask);
}

// x > 0 and finite (not NaN, not +inf) from the bit pattern of x, on the
// integer pipe.
__device__ __forceinline__ bool positive(long long b) { return b > 0 && b < 0x7ff0000000000000ll; }

// A guard on the local steps of one G: no physical run needs this many, and
// a run that reaches it (a degenerate state the checks let through, or a
// step too small to advance the time) stops with PR_ENONPHYS instead of
// spinning.
constexpr int MAX_LOCAL_STEPS = 1 << 24;

// The CFL maxima are taken over speeds and temperatures, non-negative in
// every physical state, where the order of the IEEE bit patterns as unsigned
// 64-bit integers is the order of the values: integer maxima keep them off
// this part's narrow FP64 pipe.  Values with the sign bit set (a negative
// theta, already flagged non-physical) count as 0; a NaN maps above every
// number and stops G.  The warp maximum of a 64-bit pattern: the maximum high
// word, then the maximum low word among the lanes holding it.
__device__ __forceinline__ unsigned long long clamp_sign(long long b) { return b < 0 ? 0ull : (unsigned long long)b; }

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x)
{
    const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(x >> 32));
    const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(x >> 32) == hi ? (unsigned)x : 0u);
    return ((unsigned long long)hi << 32) | lo;
}

// The cell beyond this CTA's block on one side (side -1: left of its first
// cell, +1: right of its last): the owner's region, the local index there and
// the mirror mask.  Interior block edges read the neighbouring rank; the
// domain ends follow the boundary rule (periodic: the opposite end; outflow:
// a copy of the end cell; reflecting: the end cell mirrored).
__device__ __forceinline__ const double* beyond_block(cg::cluster_group& cl, const Peers& P, int C, int nx, int bc,
                                                      int side, int& lj, unsigned long long& mask)
{
    const int last_lj = nx - 1 - (C - 1) * P.m;  // local index of cell nx-1 on rank C-1
    int r;
    mask = 0ull;
    if (side < 0) {
        if (P.rank > 0) r = P.rank - 1, lj = P.m - 1;
        else if (bc == 0) r = C - 1, lj = last_lj;
        else r = 0, lj = 0, mask = bc == 2 ? SIGN : 0ull;
    } else {
        if (P.rank < C - 1) r = P.rank + 1, lj = 0;
        else if (bc == 0) r = 0, lj = 0;
        else r = C - 1, lj = last_lj, mask = bc == 2 ? SIGN : 0ull;
    }
    return P.of(cl, r);
}

// G over dT applied to this CTA's cells [c0, c1) of the state at region
// offset 0 (A), with the other CTAs of the cluster doing theirs; returns the
// region offset of the result (A, or B after an odd number of local steps).
// Per local step:
//   1. one thread per own cell: primitives, flux h, speed (and the
//      Navier-Stokes primitives) into the cache, the CTA's CFL maxima;
//   2. one cluster barrier; the cluster maxima (one rank per lane), dt;
//   3. one thread per (face, component) of the block's mc + 1 faces: the
//      Rusanov flux of Eq. (16) (plus the viscous flux of Eq. (8)), the
//      cells beyond the block through their owners' regions;
//   4. one thread per (cell, component): the update of Eq. (15) into the
//      other state (plus the force source).
// Spreading steps 3 and 4 over all warps of the CTA keeps the FP64
// instructions of any one warp few: this part's FP64 pipe takes tens of
// cycles per warp instruction, and the local step is a chain of them.  A
// cluster barrier after the last local step ends every peer read before the
// caller reuses the region.  Every CTA takes the same local steps.
template <bool VISC>
__device__ int coarse_G(const CoarseParams& p, cg::cluster_group& cl, const Peers& P, int C, int c0, int c1,
                         double dT, int* status, unsigned long long* sh)
{
    const int nx = p.nx, m = P.m, mc = c1 - c0, nf = mc + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const int cell_warps = (min(mc, (int)blockDim.x) + 31) >> 5;
    // the face pass runs on every warp but the last (which takes dt) when
    // the CTA has more than one
    const int face_threads = nw > 1 ? (nw - 1) * 32 : 32;
    const int face_thread = nw > 1 && warp == nw - 1 ? 5 * nf : (int)threadIdx.x;
    double* R = P.base;
    const int red_off = (10 + 2 * NCACHE) * m;
    double* F = R + red_off + NRED;  // face fluxes [5][m + 1]
    int lL, lR;
    unsigned long long mL, mR;
    const double* RL = beyond_block(cl, P, C, nx, p.bc, -1, lL, mL);
    const double* RR = beyond_block(cl, P, C, nx, p.bc, +1, lR, mR);
    int cur_off = 0, nxt_off = 5 * m, buf = 0;
    const double idx = 1.0 / p.dx;
    double t = 0.0;
    int nloc = 0;
    while (t < dT) {
        const double* cur = R + cur_off;
        const int ko = (10 + buf * NCACHE) * m;  // this substep's cache
        double* K = R + ko;
        unsigned long long smax = 0, thmax = 0;
        bool bad = false;
        for (int li = threadIdx.x; li < mc; li += blockDim.x) {
            double v[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) v[q] = cur[q * m + li];
            Prim pr = prim(v);
            const long long rb = __double_as_longlong(v[0]), tb = __double_as_longlong(pr.th);
            if (!positive(rb) || !positive(tb)) bad = true;
            double c = p.sound == 1 ? sqrt(pr.th) : sqrt(pr.th * (5.0 / 3.0));
            double s = fabs(pr.ux) + c;
            smax = max(smax, clamp_sign(__double_as_longlong(s)));
            thmax = max(thmax, clamp_sign(tb));
            K[li] = v[1];
            K[m + li] = v[1] * pr.ux + pr.p;
            K[2 * m + li] = v[1] * pr.uy;
            K[3 * m + li] = v[1] * pr.uz;
            K[4 * m + li] = pr.ux * (v[4] + pr.p);
            K[5 * m + li] = s;
            if (VISC) {
                K[6 * m + li] = pr.ux;
                K[7 * m + li] = pr.uy;
                K[8 * m + li] = pr.uz;
                K[9 * m + li] = pr.th;
                K[10 * m + li] = pr.p;
            }
        }
        if (bad) {
            atomicCAS(status, 0, ST_NONPHYS);
            // a NaN pattern orders above every speed: the cluster maximum
            // becomes NaN on every rank and all of them stop together
            smax = 0x7ff8000000000000ull;
        }
        smax = warp_max_u64(smax);
        thmax = warp_max_u64(thmax);
        double* red = R + red_off + 2 * buf;
        if (cell_warps == 1) {  // only warp 0 holds cells
            if (threadIdx.x == 0) red[0] = __longlong_as_double(smax), red[1] = __longlong_as_double(thmax);
        } else {
            if (lane == 0) sh[2 * warp] = smax, sh[2 * warp + 1] = thmax;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned long long a = 0, b = 0;
                for (int w = 0; w < cell_warps; ++w) a = max(a, sh[2 * w]), b = max(b, sh[2 * w + 1]);
                red[0] = __longlong_as_double(a);
                red[1] = __longlong_as_double(b);
            }
        }
        cl.sync();  // caches, states and CTA maxima of every rank visible
        // 2. the last warp (the fewest face items) takes the cluster maxima
        // and dt while the others start on the faces, which need neither
        if (warp == nw - 1) {
            smax = 0;
            thmax = 0;
            if (lane < C) {
                const double* rr = P.of(cl, lane) + red_off + 2 * buf;
                smax = __double_as_longlong(rr[0]);
                thmax = __double_as_longlong(rr[1]);
            }
            smax = warp_max_u64(smax);
            thmax = warp_max_u64(thmax);
            const double sm = __longlong_as_double(smax);
            // (finite speeds: positive() rejected +inf and NaN above, a
            // degenerate step that makes no progress runs into the step cap)
            unsigned long long flags = 0;  // 1: last local step, 2: stop (degenerate state or steps)
            double dt = 0.0;
            if (!(sm > 0.0) || isnan(sm) || nloc >= MAX_LOCAL_STEPS) {
                flags = 2;
            } else {
                const double rem = dT - t;
                dt = p.cfl * p.dx / sm;
                if (VISC) {
                    double dtv = p.cfl * p.dx * p.dx / (2.0 * p.visc * (5.0 / 3.0) * __longlong_as_double(thmax));
                    if (dtv < dt) dt = dtv;
                }
                if (dt >= rem) {
                    dt = rem;
                    flags = 1;
                }
            }
            if (flags == 2 && lane == 0) atomicCAS(status, 0, ST_NONPHYS);
            if (lane == 0) sh[0] = __double_as_longlong(dt), sh[1] = flags;
        }
        // 3. face f of the block lies between its cells f - 1 and f
        for (int w = face_thread; w < 5 * nf; w += face_threads) {
            const int q = w / nf, f = w - q * nf;
            const double* Ra = f > 0 ? R : RL;
            const double* Rb = f < mc ? R : RR;
            const int ia = f > 0 ? f - 1 : lL, ib = f < mc ? f : lR;
            const unsigned long long ma = f > 0 ? 0ull : mL, mb = f < mc ? 0ull : mR;
            // mirrored: rho u_x (q = 1) of the state, every flux component but h_1
            const unsigned long long va_m = q == 1 ? ma : 0ull, ha_m = q == 1 ? 0ull : ma;
            const unsigned long long vb_m = q == 1 ? mb : 0ull, hb_m = q == 1 ? 0ull : mb;
            const double va = flip_sign(Ra[cur_off + q * m + ia], va_m);
            const double vb = flip_sign(Rb[cur_off + q * m + ib], vb_m);
            const double ha = flip_sign(Ra[ko + q * m + ia], ha_m);
            const double hb = flip_sign(Rb[ko + q * m + ib], hb_m);
            const long long sa = __double_as_longlong(Ra[ko + 5 * m + ia]);
            const long long sb = __double_as_longlong(Rb[ko + 5 * m + ib]);
            const double S = __longlong_as_double(sa > sb ? sa : sb);
            double H = 0.5 * (ha + hb) - 0.5 * S * (vb - va);
            if (VISC && q > 0) {
                const double eps = p.visc;
                const double* Ka = Ra + ko + ia;
                const double* Kb = Rb + ko + ib;
                const double mu = 0.5 * (Ka[10 * m] + Kb[10 * m]);
                const double uxa = flip_sign(Ka[6 * m], ma), uxb = flip_sign(Kb[6 * m], mb);
                const double dux = (uxb - uxa) * idx;
                const double sxx = -eps * mu * (4.0 / 3.0) * dux;
                if (q == 1) {
                    H += sxx;
                } else if (q == 2) {
                    H += -eps * mu * ((Kb[7 * m] - Ka[7 * m]) * idx);
                } else if (q == 3) {
                    H += -eps * mu * ((Kb[8 * m] - Ka[8 * m]) * idx);
                } else {
                    const double duy = (Kb[7 * m] - Ka[7 * m]) * idx, duz = (Kb[8 * m] - Ka[8 * m]) * idx;
                    const double dth = (Kb[9 * m] - Ka[9 * m]) * idx;
                    const double ux = 0.5 * (uxa + uxb), uy = 0.5 * (Ka[7 * m] + Kb[7 * m]);
                    const double uz = 0.5 * (Ka[8 * m] + Kb[8 * m]);
                    const double sxy = -eps * mu * duy, sxz = -eps * mu * duz;
                    const double qh = -eps * (2.5 * mu) * dth;
                    H += sxx * ux + sxy * uy + sxz * uz + qh;
                }
            }
            F[q * (m + 1) + f] = H;
        }
        __syncthreads();
        const double dt = __longlong_as_double(sh[0]);
        const unsigned long long flags = sh[1];
        if (flags & 2) break;  // the same on every rank
        const bool last = flags & 1;
        // 4. update of Eq. (15), forward-Euler force source on the old state
        double* nxt = R + nxt_off;
        const double dtdx = dt * idx;
        for (int w = threadIdx.x; w < 5 * mc; w += blockDim.x) {
            const int q = w / mc, li = w - q * mc;
            double u = cur[q * m + li] - dtdx * (F[q * (m + 1) + li + 1] - F[q * (m + 1) + li]);
            if (p.E && (q == 1 || q == 4)) u += dt * cur[(q == 1 ? 0 : 1) * m + li] * p.E[c0 + li];
            nxt[q * m + li] = u;
        }
        __syncthreads();  // the next local step reads nxt by cell
        const int tmp = cur_off;
        cur_off = nxt_off;
        nxt_off = tmp;
        buf ^= 1;
        if (last) break;
        t += dt;
        ++nloc;
    }
    cl.sync();  // every rank's reads of this region are over
    return cur_off;
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
template <bool VISC>
__global__ void __launch_bounds__(CT)
k_coarse(CoarseParams p, const double* Vin, double* Vout, double dT, double* work, int use_smem, int* status)
{
    extern __shared__ __align__(16) double dsm[];
    __shared__ unsigned long long sh[2 * (CT / 32)];
    cg::cluster_group cl = cg::this_cluster();
    const int nx = p.nx, C = gridDim.x, m = (nx + C - 1) / C;
    const int c0 = (int)blockIdx.x * m, c1 = min(nx, c0 + m);
    const Peers P = make_peers(dsm, work, use_smem, m);
    for (int li = threadIdx.x; li < c1 - c0; li += blockDim.x)
#pragma unroll
        for (int q = 0; q < 5; ++q) P.base[q * m + li] = Vin[q * nx + c0 + li];
    __syncthreads();
    const int off = coarse_G<VISC>(p, cl, P, C, c0, c1, dT, status, sh);
    for (int li = threadIdx.x; li < c1 - c0; li += blockDim.x)
#pragma unroll
        for (int q = 0; q < 5; ++q) Vout[q * nx + c0 + li] = P.base[off + q * m + li];
    cl.sync();  // no CTA leaves while another may still read its region
}

// Algorithm 2's sequential sweep over n = max(k,1)..N on one cluster of C
// CTAs, each owning a contiguous block of cells.
template <bool VISC>
__global__ void __launch_bounds__(CT)
k_sweep(CoarseParams p, int N, double dT, const int* dk, double* U, const double* PFL, double* Gs, double* err,
        double* work, int use_smem, int* status, int bump, int* dk_mut)
{
    extern __shared__ __align__(16) double dsm[];
    __shared__ unsigned long long sh[2 * (CT / 32)];
    cg::cluster_group cl = cg::this_cluster();
    const int nx = p.nx, sz = 5 * nx, C = gridDim.x, m = (nx + C - 1) / C;
    const int c0 = (int)blockIdx.x * m, c1 = min(nx, c0 + m), mc = c1 - c0;
    const int k = *dk;
    const Peers P = make_peers(dsm, work, use_smem, m);
    double* A = P.base;
    double emax = 0.0;
    const int n0 = k > 1 ? k : 1;
    // one cell per thread: the slice's jump and old iterate are prefetched
    // into registers while G runs (they do not depend on it)
    const bool pre = mc <= (int)blockDim.x;
    if (n0 <= N) {
        for (int li = threadIdx.x; li < mc; li += blockDim.x)
#pragma unroll
            for (int q = 0; q < 5; ++q) A[q * m + li] = U[(size_t)(n0 - 1) * sz + q * nx + c0 + li];
        __syncthreads();
    }
    for (int n = n0; n <= N; ++n) {
        double jp[5], uo[5];
        if (pre && (int)threadIdx.x < mc) {
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const size_t o = (size_t)n * sz + q * nx + c0 + threadIdx.x;
                jp[q] = k > 0 ? PFL[o] - Gs[o] : 0.0;
                uo[q] = U[o];
            }
        }
        const int off = coarse_G<VISC>(p, cl, P, C, c0, c1, dT, status, sh);
        // correction; the new iterate also stays in A as the next slice's start
        for (int li = threadIdx.x; li < mc; li += blockDim.x)
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const size_t o = (size_t)n * sz + q * nx + c0 + li;
                const double gv = P.base[off + q * m + li];
                const double jump = pre ? jp[q] : (k > 0 ? PFL[o] - Gs[o] : 0.0);
                const double nv = k > 0 ? gv + jump : gv;
                const double d = fabs(nv - (pre ? uo[q] : U[o]));
                if (d > emax) emax = d;
                U[o] = nv;
                Gs[o] = gv;
                A[q * m + li] = nv;
            }
        __syncthreads();
    }
    // the error of the iteration: max over the cluster
    double dummy = 0.0;
    block_max2(emax, dummy, reinterpret_cast<double*>(sh));
    const int red_off = (10 + 2 * NCACHE) * m;
    if (threadIdx.x == 0) P.base[red_off] = emax;
    cl.sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double e = 0.0;
        for (int r = 0; r < C; ++r) e = fmax(e, P.of(cl, r)[red_off]);
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

// CTAs of the coarse cluster: blocks of about 32 cells (the per-cell pass of
// a local step is then one warp per CTA, the face and update passes a few
// warps; more CTAs would shorten no warp's chain of FP64 instructions and
// only add participants to the cluster barrier), at most 16 CTAs, none empty
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
    // a thread per face component, and one more warp for the local step dt
    cfg.blockDim = dim3(std::min(CT, (5 * (m + 1) + 31) / 32 * 32 + 32), 1, 1);
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
    const void* fns[4] = {reinterpret_cast<const void*>(&k_coarse<false>), reinterpret_cast<const void*>(&k_coarse<true>),
                          reinterpret_cast<const void*>(&k_sweep<false>), reinterpret_cast<const void*>(&k_sweep<true>)};
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
    return launch_cluster(p.visc > 0.0 ? k_coarse<true> : k_coarse<false>, p.nx, s, p, Vin, Vout, dT, work,
                          (int)fits_smem(p.nx), status);
}

cudaError_t launch_sweep(const CoarseParams& p, int N, double dT, const int* dk, double* U, const double* PFL,
                         double* Gs, double* err, double* work, int* status, int bump, int* dk_mut,
                         cudaStream_t s)
{
    return launch_cluster(p.visc > 0.0 ? k_sweep<true> : k_sweep<false>, p.nx, s, p, N, dT, dk, U, PFL, Gs, err, work,
                          (int)fits_smem(p.nx), status, bump, dk_mut);
}

size_t coarse_work_doubles(int nx) { return work_doubles(nx); }

// Several problems iterated in lockstep (one k): instances 0..n_sl-1 run
// slices nidx[i] (ascending), the rest are independent instances.  Slices
// n >= max(k,1) run and are lifted: run = [lo, n_inst), lift = [lo, n_sl).
__global__ void k_set_active_multi(const int* dk, const int* nidx, int n_sl, int n_inst, Active* run, Active* lift)
{
    const int k = *dk, first = k > 1 ? k : 1;
    int lo = 0, hi = n_sl;  // first instance whose slice is >= first
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (nidx[mid] >= first) hi = mid;
        else lo = mid + 1;
    }
    run->begin = lo;
    run->end = n_inst;
    lift->begin = lo;
    lift->end = n_sl;
}

cudaError_t launch_set_active_multi(const int* dk, const int* nidx, int n_sl, int n_inst, Active* run, Active* lift,
                                    cudaStream_t s)
{
    k_set_active_multi<<<1, 1, 0, s>>>(dk, nidx, n_sl, n_inst, run, lift);
    return cudaGetLastError();
}

cudaError_t launch_set_active(const int* dk, Active* active, int first_slice, int n_inst, int N, cudaStream_t s)
{
    k_set_active<<<1, 1, 0, s>>>(dk, active, first_slice, n_inst, N);
    return cudaGetLastError();
}

}  // namespace prk
