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

#include <algorithm>
#include <math.h>
#include <stdint.h>

#include "maxwell_tab.h"
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

__device__ __forceinline__ double texp(double x) { return exp(x); }

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Accumulators of the cross-warp and cluster sums: double in the double
// path; in the float path a double-float pair (hi + lo, error-free FP32
// transformations: Knuth's TwoSum, Dekker's product with fmaf), which keeps
// ~44 bits without touching the double pipe, slow on this part.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const float s = a.hi + b.hi, bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    const float h = s + e;
    return {h, e - (h - s)};
}

__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    const float h = p + e;
    return {h, e - (h - p)};
}

template <typename T>
struct Acc;
template <>
struct Acc<double> {
    using A = double;
    static __device__ __forceinline__ A from(double x) { return x; }
    static __device__ __forceinline__ A add(A a, A b) { return a + b; }
    static __device__ __forceinline__ double to_double(A a) { return a; }
};
template <>
struct Acc<float> {
    using A = DF;
    static __device__ __forceinline__ A from(float x) { return {x, 0.0f}; }
    static __device__ __forceinline__ A add(A a, A b) { return df_add(a, b); }
    static __device__ __forceinline__ double to_double(A a) { return (double)a.hi + (double)a.lo; }
};

// Shared-memory layout of the step kernel (the same size for both
// accumulator types: 8 bytes each).
template <typename A>
struct FSharedT {
    A red[32][5];     // per-warp partial sums (up to 1024 threads)
    A part[2][8];     // this CTA's partials, phase 0 (f*) and 1 (f^{n+1}); read by the cluster
    A gat[16][5];     // the cluster's partials, gathered (rank, quantity)
    A tot[8];         // cluster totals (rank order)
    double par[8];    // double path: rho, u_x, u_y, u_z, theta, pref, 1/(2 theta)
    float fpar[8];    // (unused: the float path's pairs FPar replace tot once read)
};
using FShared = FSharedT<double>;
static_assert(sizeof(FSharedT<DF>) == sizeof(FSharedT<double>), "layouts differ");

// A per-instance scalar in the element type: the float copy in the float path
// (a double-to-float conversion runs on the slow double pipe of this part).
__device__ __forceinline__ float pick_t(double, float f, float*) { return f; }
__device__ __forceinline__ double pick_t(double d, float, double*) { return d; }
template <typename T>
__device__ __forceinline__ T scal(double d, float f)
{
    return pick_t(d, f, static_cast<T*>(nullptr));
}

// Sum of the CTA's 5 values s[] into sh.part[phase] (accumulators over warps).
template <typename T>
__device__ __forceinline__ void cta_partials(const T (&s)[5], FSharedT<typename Acc<T>::A>& sh, int phase)
{
    using AC = Acc<T>;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        T v = warp_sum_t(s[q]);
        if (lane == 0) sh.red[w][q] = AC::from(v);
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        typename AC::A a = AC::from(T(0));
        const int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < nw; ++k) a = AC::add(a, sh.red[k][threadIdx.x]);
        sh.part[phase][threadIdx.x] = a;
    }
}

// Copy the cluster's partials part[phase] of every rank into gat (one
// distributed-shared-memory load per thread, all in flight at once; a CTA
// of fewer than 5 C threads takes several).
template <typename A>
__device__ __forceinline__ void cluster_gather(cg::cluster_group& cl, FSharedT<A>& sh, int phase, int C)
{
    for (int t = threadIdx.x; t < 5 * C; t += blockDim.x) {
        const int r = t / 5, k = t - 5 * r;
        const FSharedT<A>* rs = cl.map_shared_rank(&sh, r);
        sh.gat[r][k] = rs->part[phase][k];
    }
}

// Sum of quantity k over the C ranks' gathered partials in a fixed pairwise
// order (depth log2 C; every CTA of the cluster adds in the same order).
template <typename T>
__device__ __forceinline__ typename Acc<T>::A rank_sum(const FSharedT<typename Acc<T>::A>& sh, int k, int C)
{
    using AC = Acc<T>;
    typename AC::A v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = r < C ? sh.gat[r][k] : AC::from(T(0));
#pragma unroll
    for (int w = 1; w < 16; w *= 2)
#pragma unroll
        for (int r = 0; r + w < 16; r += 2 * w) v[r] = AC::add(v[r], v[r + w]);
    return v[0];
}

// Reciprocal and reciprocal square root in double precision by two
// Newton-Raphson steps from a single-precision seed (each step squares the
// relative error: 2^-23 -> 2^-46 -> below double rounding).
__device__ __forceinline__ double rcp_nr(double x)
{
    double y = (double)(1.0f / (float)x);
    if (!(y != 0.0 && isfinite(y))) return 1.0 / x;  // outside the float range
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

__device__ __forceinline__ double rsqrt_nr(double x)
{
    double y = (double)rsqrtf((float)x);
    if (!(y != 0.0 && isfinite(y))) return 1.0 / sqrt(x);
    double e = fma(-x * y, y, 1.0);  // 1 - x y^2
    y = fma(0.5 * y, e, y);
    e = fma(-x * y, y, 1.0);
    return fma(0.5 * y, e, y);
}

// Maxwellian parameters from the cluster totals (one thread).  The double
// path gets tot = (rho, rho u, 2E) with 2E = sum |v|^2 f dv and writes par =
// (rho, u_x, u_y, u_z, theta, rho (2 pi theta)^(-3/2), 1/(2 theta)), the
// reciprocals by Newton steps.  The float path gets the same sums without the
// cell volume dv3 (double-float) and writes FPar: u, 1/(2 theta) and the
// prefactor rho dv3 (2 pi theta)^{-3/2} as float pairs, in pair arithmetic
// (~1e-13; theta = (rho 2E - |rho u|^2) / (3 rho^2) with the numerator, which
// cancels when |u|^2 >> theta, formed in double-float), so that the float32
// factor tables come out within about 1e-9 before their one rounding.  A
// non-positive rho or theta raises PR_ENONPHYS when report is set.
struct FPar {
    F2 u[3], i2t, pref;
};
static_assert(sizeof(FPar) == 5 * sizeof(DF), "FPar takes the place of the five double-float totals");

__device__ __forceinline__ void maxwell_params_d(const double* tot, double* par, bool report, int* status)
{
    const double r = tot[0], m1 = tot[1], m2 = tot[2], m3 = tot[3], e2 = tot[4];
    const double num = fma(r, e2, -(fma(m1, m1, fma(m2, m2, m3 * m3))));  // 3 rho^2 theta
    const bool ok = r > 0.0 && num > 0.0 && isfinite(r) && isfinite(num);
    if (!ok && report) atomicCAS(status, 0, ST_NONPHYS);
    const double ir = rcp_nr(r);
    const double th = ok ? num * (ir * ir) * (1.0 / 3.0) : 1.0;
    const double rs = ok ? rsqrt_nr(2.0 * 3.14159265358979323846 * th) : 0.0;
    par[0] = r;
    par[1] = m1 * ir;
    par[2] = m2 * ir;
    par[3] = m3 * ir;
    par[4] = th;
    par[5] = r * rs * rs * rs;
    par[6] = 0.5 * rcp_nr(th);
}

__device__ __forceinline__ void maxwell_params(FSharedT<double>& sh, double, bool report, int* status)
{
    maxwell_params_d(sh.tot, sh.par, report, status);
}

__device__ __forceinline__ void maxwell_params_f(const DF* tot, float* fpar, double dv3, bool report, int* status)
{
    const DF r = tot[0], m1 = tot[1], m2 = tot[2], m3 = tot[3], e2 = tot[4];
    const DF mm = df_add(df_mul(m1, m1), df_add(df_mul(m2, m2), df_mul(m3, m3)));
    const DF nd = df_add(df_mul(r, e2), DF{-mm.hi, -mm.lo});  // 3 rho^2 theta (sums without dv3)
    const float rf = r.hi + r.lo, num = nd.hi + nd.lo;
    const bool ok = rf > 0.0f && num > 0.0f && isfinite(rf) && isfinite(num);
    if (!ok && report) atomicCAS(status, 0, ST_NONPHYS);
    FPar P;
    if (ok) {
        const F2 R = f2_norm(r.hi, r.lo), ir = f2_rcp(R);
        P.u[0] = f2_mul(f2_norm(m1.hi, m1.lo), ir);
        P.u[1] = f2_mul(f2_norm(m2.hi, m2.lo), ir);
        P.u[2] = f2_mul(f2_norm(m3.hi, m3.lo), ir);
        const F2 th = f2_mul(f2_mul(f2_norm(nd.hi, nd.lo), f2_mul(ir, ir)), f2_of(1.0 / 3.0));
        P.i2t = f2_mul(F2{0.5f, 0.0f}, f2_rcp(th));
        const F2 tp = f2_mul(f2_of(2.0 * 3.14159265358979323846), th);
        P.pref = f2_mul(f2_mul(R, f2_of(dv3)), f2_rcp(f2_mul(tp, f2_sqrt(tp))));
    } else {
        P.u[0] = P.u[1] = P.u[2] = F2{0.0f, 0.0f};
        P.i2t = F2{0.5f, 0.0f};
        P.pref = F2{0.0f, 0.0f};
    }
    *reinterpret_cast<FPar*>(fpar) = P;
}

__device__ __forceinline__ void maxwell_params(FSharedT<DF>& sh, double dv3, bool report, int* status)
{
    maxwell_params_f(sh.tot, reinterpret_cast<float*>(sh.tot), dv3, report, status);  // FPar over tot
}

// exp(-(v - u)^2 / (2 theta)) times m, from the float-pair node v, mean u and
// 1/(2 theta): the exponent in pair arithmetic, exp_neg_pair for the rest.
__device__ __forceinline__ float gauss_f2(F2 v, F2 u, F2 i2t, F2 m)
{
    float ch, cl;
    two_sum(v.h, -u.h, ch, cl);
    cl += v.l - u.l;
    const F2 c = f2_norm(ch, cl);
    const F2 x = f2_mul(f2_mul(c, c), i2t);
    return exp_neg_pair(x.h, x.l, m.h, m.l);
}

__device__ __forceinline__ void cluster_arrive()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

// Arrival without ordering: for a CTA whose remote reads have all returned.
__device__ __forceinline__ void cluster_arrive_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ long long gtimer()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait (bounded by limit_ns) until the phase of the mbarrier with the given
// parity completes; false on time-out.  Each try suspends the thread for up
// to 100 us unless the phase completes first.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, long long limit_ns, uint32_t parity = 0)
{
    const long long t0 = gtimer();
    for (int it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity), "r"(100000)
            : "memory");
        if (done) return true;
        if ((it & 63) == 63 && gtimer() - t0 > limit_ns) return false;
    }
}

// One contiguous run of v_x rows [a, b) of a (possibly ghost) x column, to be
// placed at rows dst0.. of a shared-memory buffer.  Mirrored columns (a
// reflecting wall reverses v_x) hold row r at stored row nvx-1-r.
struct Seg {
    const void* col;  // stored column base
    int a, b;         // ghost-column rows
    int dst0;         // buffer row of ghost row a
    bool mir;
};

// Bulk copies of the non-mirrored segments (thread 0; completion on the
// mbarrier, which thread 0 initialises here), when rows are 16-byte multiples.
template <typename T>
__device__ __forceinline__ void stage_bulk(const Seg* segs, int nseg, T* const* dst, int nvp2, uint32_t mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    uint32_t bytes = 0;
    for (int k = 0; k < nseg; ++k)
        if (!segs[k].mir && segs[k].b > segs[k].a) bytes += (uint32_t)(segs[k].b - segs[k].a) * nvp2 * sizeof(T);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
    for (int k = 0; k < nseg; ++k) {
        const Seg& q = segs[k];
        if (q.mir || q.b <= q.a) continue;
        const T* src = static_cast<const T*>(q.col) + (size_t)q.a * nvp2;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_addr(dst[k] + (size_t)q.dst0 * nvp2)),
            "l"(src), "r"((uint32_t)(q.b - q.a) * nvp2 * (uint32_t)sizeof(T)), "r"(mbar)
            : "memory");
    }
}

// The other segments (mirrored, or all when rows are not 16-byte multiples),
// copied by all threads of the CTA element by element (a __syncthreads follows).
template <typename T>
__device__ __forceinline__ void stage_threads(const Seg* segs, int nseg, T* const* dst, int nvx, int nvp2, bool bulk)
{
    for (int k = 0; k < nseg; ++k) {
        const Seg& q = segs[k];
        if (bulk && !q.mir) continue;
        const T* col = static_cast<const T*>(q.col);
        const int n = (q.b - q.a) * nvp2;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const int r = q.a + e / nvp2, j = e - (e / nvp2) * nvp2;
            dst[k][(size_t)(q.dst0 + r - q.a) * nvp2 + j] = col[(size_t)(q.mir ? nvx - 1 - r : r) * nvp2 + j];
        }
    }
}

// VEC consecutive values of one shared-memory or global row (16 bytes when
// VEC * sizeof(T) == 16).
template <typename T, int V>
struct alignas(sizeof(T) * V) Pack {
    T x[V];
};

template <typename T, int V>
__device__ __forceinline__ Pack<T, V> ldv(const T* p)
{
    return *reinterpret_cast<const Pack<T, V>*>(p);
}

template <typename T, int V>
__device__ __forceinline__ void stv(T* p, const Pack<T, V>& v)
{
    *reinterpret_cast<Pack<T, V>*>(p) = v;
}

// Thread layout of the step kernel: Lr = nvp^2 / VEC threads cover a v_x row
// (thread q owns the VEC consecutive (v_y, v_z) cells q*VEC ..), G groups of
// Lr threads split the CTA's rows into contiguous runs.
template <typename T, int SCHEME, int VEC>
__global__ void __launch_bounds__(VEC == 1 ? 1024 : 512, 1)
k_force_step(const FInst* __restrict__ insts, FGeom g, const Active* __restrict__ act, int* __restrict__ cur,
             int step, int last, int* __restrict__ status, long long wait_ns, int poison)
{
    const int b = blockIdx.z;
    if (b < act->begin || b >= act->end) return;  // uniform over the cluster
    cg::cluster_group cl = cg::this_cluster();
    const FInst& I = insts[b];
    const int i = blockIdx.y, rank = blockIdx.x, C = gridDim.x;
    const int nvx = g.nvx, nvp2 = g.nvp * g.nvp;
    const long long ncol = g.ncol;
    const int R = g.rows;
    const int r0 = rank * R, r1 = min(r0 + R, nvx), nr = r1 - r0;

    extern __shared__ __align__(16) unsigned char fsm[];
    using AC = Acc<T>;
    FSharedT<typename AC::A>& sh = *reinterpret_cast<FSharedT<typename AC::A>*>(fsm);
    unsigned long long* mbar_p = reinterpret_cast<unsigned long long*>(fsm + sizeof(FShared));
    T* vxs = reinterpret_cast<T*>(fsm + sizeof(FShared) + 16);  // v_x nodes
    T* ex = vxs + nvx;                                           // Maxwellian factors: ex[nvx], ey[nvp], ez[nvp]
    T* cen = reinterpret_cast<T*>(fsm + g.buf_off);              // rows r0-1 .. r1 of column i
    T* nb = cen + (size_t)(R + 2) * nvp2;                        // NB x R rows of neighbour columns; f* into nb
    const uint32_t mbar = smem_addr(mbar_p);

    const int Lr = nvp2 / VEC;                       // threads per row
    const int G = g.groups;                          // row groups
    const int q = threadIdx.x % Lr, grp = threadIdx.x / Lr;
    const int jp = q * VEC;
    const int Rg = (nr + G - 1) / G;
    const int ra = r0 + grp * Rg, rb = min(ra + Rg, r1);
    const bool active = grp < G && ra < rb;
    const bool bulk = g.bulk != 0;
    const int bufi = cur[b] ^ (step & 1);
    const T* __restrict__ fin = static_cast<const T*>(I.f[bufi]);
    T* __restrict__ fout = static_cast<T*>(I.f[bufi ^ 1]);

    // segments: own column rows r0-1..r1 (clipped), then the neighbour rows each
    // v_x row needs: upwind: i-1 where v_x > 0, i+1 where v_x < 0; MUSCL: i-1
    // and i+1 everywhere plus i-2 / i+2 where v_x > 0 / < 0.  hpos: first row
    // with v_x > 0.
    const int hpos = I.hpos;
    const int pa = max(r0, hpos), na = min(r1, hpos);
    Seg segs[5];
    T* dst[5];
    int nseg = 0;
    auto col = [&](int d, bool* m) { return static_cast<const void*>(fin + (size_t)ghost_col(i + d, I.nx, I.bc, m) * ncol); };
    {
        bool m;
        const void* c0 = col(0, &m);
        int a = max(r0 - 1, 0), e = min(r1 + 1, nvx);
        segs[nseg] = {c0, a, e, a - (r0 - 1), false};
        dst[nseg++] = cen;
    }
    if (SCHEME == 0) {
        bool mm, mp;
        const void* cm = col(-1, &mm);
        const void* cp = col(1, &mp);
        segs[nseg] = {cm, pa, r1, pa - r0, mm};
        dst[nseg++] = nb;
        segs[nseg] = {cp, r0, na, 0, mp};
        dst[nseg++] = nb;
    } else {
        bool mm, mp, mm2, mp2;
        const void* cm = col(-1, &mm);
        const void* cp = col(1, &mp);
        const void* cm2 = col(-2, &mm2);
        const void* cp2 = col(2, &mp2);
        segs[nseg] = {cm, r0, r1, 0, mm};
        dst[nseg++] = nb;
        segs[nseg] = {cp, r0, r1, 0, mp};
        dst[nseg++] = nb + (size_t)R * nvp2;
        segs[nseg] = {cm2, pa, r1, pa - r0, mm2};
        dst[nseg++] = nb + (size_t)2 * R * nvp2;
        segs[nseg] = {cp2, r0, na, 0, mp2};
        dst[nseg++] = nb + (size_t)2 * R * nvp2;
    }
    // the bulk copies go out first; the tables load while they are in flight.
    // poison (failure-detection check): a second mbarrier expects 16 bytes
    // that no copy delivers, so the wait on it runs out
    const uint32_t mbar2 = mbar + 8;
    if (bulk && threadIdx.x == 0) {
        stage_bulk<T>(segs, nseg, dst, nvp2, mbar);
        if (poison) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar2), "r"(1) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar2), "r"(16) : "memory");
        }
    }
    stage_threads<T>(segs, nseg, dst, nvx, nvp2, bulk);
    const T* vt = static_cast<const T*>(I.vtab);
    for (int k = threadIdx.x; k < nvx; k += blockDim.x) vxs[k] = vt[k];
    T vy[VEC], vz[VEC], vp2[VEC];
    int jy[VEC], jz[VEC];
    {
        int y = jp / g.nvp, z = jp - (jp / g.nvp) * g.nvp;  // one division; the lanes step on
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
            vy[l] = active ? vt[nvx + jp + l] : T(0);
            vz[l] = active ? vt[nvx + nvp2 + jp + l] : T(0);
            vp2[l] = active ? vt[nvx + 2 * nvp2 + jp + l] : T(0);
            jy[l] = y;
            jz[l] = z;
            if (++z == g.nvp) {
                z = 0;
                ++y;
            }
        }
    }
    __syncthreads();  // mbarrier initialised; thread-staged rows visible
    if (bulk && poison && !mbar_wait(mbar2, wait_ns)) atomicCAS(status, 0, ST_TIMEOUT);
    if (bulk && !mbar_wait(mbar, wait_ns)) {
        atomicCAS(status, 0, ST_TIMEOUT);
        mbar_wait(mbar, wait_ns);  // let copies in flight land before the buffers are reused
    }

    const T nu = scal<T>(I.nu, I.fnu), nuv = scal<T>(I.nuv, I.fnuv);
    const T hE = T(0.5) * scal<T>(I.E[i], I.Ef[i]), hEm = T(0.5) * scal<T>(I.Emax, I.fEmax), half = T(0.5);

    // pass 1: f* of this thread's rows (written over the first neighbour
    // buffer, each element by the thread that read it), with the sums
    // sum f* per lane and sum v_x f*, sum v_x^2 f* over the lanes
    T S0[VEC], S1 = T(0), S4 = T(0);
#pragma unroll
    for (int l = 0; l < VEC; ++l) S0[l] = T(0);
    if (active) {
        T* nb1 = nb;
        const T* nb2 = nb + (size_t)R * nvp2;
        const T* nb3 = nb + (size_t)2 * R * nvp2;
        Pack<T, VEC> dn, c;
#pragma unroll
        for (int l = 0; l < VEC; ++l) dn.x[l] = T(0);
        if (ra > 0) dn = ldv<T, VEC>(cen + (size_t)(ra - r0) * nvp2 + jp);
        c = ldv<T, VEC>(cen + (size_t)(ra - r0 + 1) * nvp2 + jp);
#pragma unroll 2
        for (int r = ra; r < rb; ++r) {
            const size_t o = (size_t)(r - r0) * nvp2 + jp;
            Pack<T, VEC> up;
            if (r < nvx - 1) up = ldv<T, VEC>(cen + o + 2 * (size_t)nvp2);
            else {
#pragma unroll
                for (int l = 0; l < VEC; ++l) up.x[l] = T(0);
            }
            const T vx = vxs[r];
            const bool pos = vx > T(0);
            const Pack<T, VEC> x1 = ldv<T, VEC>(nb1 + o);
            Pack<T, VEC> x2, x3;
            if (SCHEME == 1) {
                x2 = ldv<T, VEC>(nb2 + o);
                x3 = ldv<T, VEC>(nb3 + o);
            }
            const bool interior = r > 0 && r < nvx - 1;
            Pack<T, VEC> out;
            T vsum = T(0);
#pragma unroll
            for (int l = 0; l < VEC; ++l) {
                const T cc = c.x[l], u = up.x[l], d = dn.x[l];
                T Fd;  // F_{i+1/2} - F_{i-1/2}
                if (SCHEME == 0) {
                    Fd = vx * (pos ? cc - x1.x[l] : x1.x[l] - cc);
                } else {
                    const T m1 = x1.x[l], p1 = x2.x[l], far = x3.x[l];
                    if (pos) Fd = vx * ((cc + half * minmod(cc - m1, p1 - cc)) - (m1 + half * minmod(m1 - far, cc - m1)));
                    else Fd = vx * ((p1 - half * minmod(p1 - cc, far - p1)) - (cc - half * minmod(cc - m1, p1 - cc)));
                }
                T Gd;  // G_{j+1/2} - G_{j-1/2}, zero flux through the ends of the box
                if (interior) Gd = hE * (u - d) - hEm * ((u + d) - (cc + cc));
                else {
                    const T Gr = r < nvx - 1 ? hE * (cc + u) - hEm * (u - cc) : T(0);
                    const T Gl = r > 0 ? hE * (d + cc) - hEm * (cc - d) : T(0);
                    Gd = Gr - Gl;
                }
                const T v = cc - nu * Fd - nuv * Gd;
                out.x[l] = v;
                S0[l] += v;
                vsum += v;
            }
            stv<T, VEC>(nb1 + o, out);
            S1 += vx * vsum;
            S4 += (vx * vx) * vsum;
            dn = c;
            c = up;
        }
    }
    {
        T s[5] = {T(0), S1, T(0), T(0), S4};
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
            s[0] += S0[l];
            s[2] += vy[l] * S0[l];
            s[3] += vz[l] * S0[l];
            s[4] += vp2[l] * S0[l];
        }
        cta_partials(s, sh, 0);
    }
    cl.sync();
    cluster_gather(cl, sh, 0, C);
    __syncthreads();
    if (threadIdx.x < 5) {
        // the same order in every CTA; the double path scales by dv3 here
        const typename AC::A t = rank_sum<T>(sh, threadIdx.x, C);
        if constexpr (sizeof(T) == sizeof(double)) sh.tot[threadIdx.x] = t * I.dv3;
        else sh.tot[threadIdx.x] = t;
    }
    cluster_arrive_relaxed();  // the peers' partials are read (the matching wait is at the end)
    __syncthreads();
    if (threadIdx.x == 0) maxwell_params(sh, I.dv3, I.collide && rank == 0, status);
    __syncthreads();

    const T a = scal<T>(I.a, I.fa), bb = scal<T>(I.b, I.fb);
    const bool collide = I.collide != 0;
    T myz[VEC];  // b pref ey[jy] ez[jz] per lane
#pragma unroll
    for (int l = 0; l < VEC; ++l) myz[l] = T(0);
    if (collide) {
        // separable Maxwellian b M = (b pref ex[jx]) ey[jy] ez[jz]: in float64
        // from the double parameters; in float32 each factor within ~1e-9 of
        // its exact value before one rounding (the exponent in pair
        // arithmetic from the pair parameters and nodes), b pref folded into
        // ex with the same single rounding
        T* ey = ex + nvx;
        T* ez = ey + g.nvp;
        const int nvp = g.nvp;
        if constexpr (sizeof(T) == sizeof(float)) {
            const FPar& P = *reinterpret_cast<const FPar*>(sh.tot);
            const F2 m = f2_mul(F2{(float)bb, 0.0f}, P.pref), one{1.0f, 0.0f};
            const F2* vp = reinterpret_cast<const F2*>(I.vpair);
            for (int k = threadIdx.x; k < nvx + 2 * nvp; k += blockDim.x) {
                if (k < nvx) {
                    ex[k] = gauss_f2(vp[k], P.u[0], P.i2t, m);
                } else {
                    const int j = k - nvx < nvp ? k - nvx : k - nvx - nvp;
                    ex[k] = gauss_f2(vp[nvx + j], P.u[k - nvx < nvp ? 1 : 2], P.i2t, one);
                }
            }
            __syncthreads();
#pragma unroll
            for (int l = 0; l < VEC; ++l) myz[l] = ey[jy[l]] * ez[jz[l]];
        } else {
            const T ux = sh.par[1], uy = sh.par[2], uz = sh.par[3], inv2th = sh.par[6];
            for (int k = threadIdx.x; k < nvx + 2 * nvp; k += blockDim.x) {
                if (k < nvx) {
                    const T cx = vxs[k] - ux;
                    ex[k] = texp(-cx * cx * inv2th);
                } else {
                    const int j = k - nvx < nvp ? k - nvx : k - nvx - nvp;
                    const T v = vt[nvx + j * nvp];  // v_y node j (v_y table, jz = 0)
                    const T cc = v - (k - nvx < nvp ? uy : uz);
                    ex[k] = texp(-cc * cc * inv2th);
                }
            }
            __syncthreads();
            const T pb = bb * sh.par[5];
#pragma unroll
            for (int l = 0; l < VEC; ++l) myz[l] = pb * (ey[jy[l]] * ez[jz[l]]);
        }
    }

    // pass 2: relax and store; on the last step also the sums of f^{n+1}
    T P0[VEC], P1 = T(0), P4 = T(0);
#pragma unroll
    for (int l = 0; l < VEC; ++l) P0[l] = T(0);
    if (active) {
        T* out = fout + (size_t)i * ncol + jp;
#pragma unroll 4
        for (int r = ra; r < rb; ++r) {
            Pack<T, VEC> v = ldv<T, VEC>(nb + (size_t)(r - r0) * nvp2 + jp);
            if (collide) {
                const T e = ex[r];
#pragma unroll
                for (int l = 0; l < VEC; ++l) v.x[l] = a * v.x[l] + e * myz[l];
            }
            stv<T, VEC>(out + (size_t)r * nvp2, v);
            if (last) {
                const T vx = vxs[r];
                T vsum = T(0);
#pragma unroll
                for (int l = 0; l < VEC; ++l) {
                    P0[l] += v.x[l];
                    vsum += v.x[l];
                }
                P1 += vx * vsum;
                P4 += (vx * vx) * vsum;
            }
        }
    }
    if (last) {
        T s[5] = {T(0), P1, T(0), T(0), P4};
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
            s[0] += P0[l];
            s[2] += vy[l] * P0[l];
            s[3] += vz[l] * P0[l];
            s[4] += vp2[l] * P0[l];
        }
        cta_partials(s, sh, 1);
        cluster_wait();  // completes the barrier arrived at after the first exchange
        cl.sync();       // every CTA's phase-1 partials are written
        cluster_gather(cl, sh, 1, C);
        __syncthreads();
        if (rank == 0 && threadIdx.x < 5) {
            double t = AC::to_double(rank_sum<T>(sh, threadIdx.x, C)) * I.dv3;
            if (threadIdx.x == 4) t *= 0.5;  // energy = 1/2 sum |v|^2 f dv
            I.Ucur[threadIdx.x * I.nx + i] = t;
            if (I.Uout) I.Uout[threadIdx.x * I.nx + i] = t;
        }
        cluster_arrive();
    }
    cluster_wait();  // no CTA leaves while another may still read its shared memory
}

// ---- fused single-pass step (upwind; float or double): one CTA walks S columns ----
//
// With upwind x fluxes the sums of phi f* over a column (phi = 1, v, |v|^2)
// are linear in sums of f^n over columns c-1, c, c+1 (summation by parts):
//   P_phi(f*_c) = M_phi(c) - nu (A+_phi(c) - A+_phi(c-1) + A-_phi(c+1) - A-_phi(c)) - nuv Q_phi(c),
// M_phi = sum phi f, A+-_phi = sum over v_x > 0 / v_x <= 0 of v_x phi f; the
// v_x Rusanov fluxes telescope (zero flux through +-L), so Q vanishes for
// phi = 1, v_y, v_z and, for phi = v_x, |v|^2, needs only M_1, M_v_x and the
// densities rho_0, rho_{nvx-1} of the first and last v_x rows:
//   Q_vx   = -dv_x [E (M_1 - (rho_0 + rho_last)/2) - E_max (rho_last - rho_0)/2]
//   Q_|v|2 = -dv_x [E (2 M_vx - L (rho_last - rho_0)) - E_max (L (rho_0 + rho_last) - dv_x M_1)].
// A reflecting wall's ghost column (v_x mirrored) has A+- = s A-+ of its
// edge column, s = -1 for the even weights (1, v_y, v_z, |v|^2), +1 for v_x.
// Each step therefore writes, next to f^{n+1}, these 17 sums of f^{n+1} per
// (column, CTA) — the partials — and the next step knows every column's
// Maxwellian before it reads f: one pass per cell (transport, relaxation,
// store, sums), no exchange between CTAs and no f* kept anywhere.  A CTA owns
// v_x rows [r0, r0+R) of the columns [i0, i0+S) of one instance: at the start
// of its walk it adds the partials of columns i0-1 .. i0+S over the C CTAs of
// a column in a fixed order and builds the parameters and factor tables of
// all S columns while the first bulk copies land; then, per column, three
// column slots rotate in shared memory as in a pipelined ring (rows with
// v_x > 0 read columns c-1 and c, the others c and c+1; a CTA's rows never
// straddle v_x = 0), the next column's copy in flight during the pass.
constexpr int NQ = 17;  // per (column, CTA): M[5], A+[5], A-[5], rho_0, rho_{nvx-1}

// The partials and the moments of f* are accumulated in FuOps<T>::A: a
// double-float pair in the float path (44 bits without the double pipe),
// double in the double path; both 8 bytes, so one layout serves both.
template <typename T>
struct FuOps;
template <>
struct FuOps<float> {
    using A = DF;
    using T2 = float2;
    static __device__ __forceinline__ A from(float x) { return DF{x, 0.0f}; }
    static __device__ __forceinline__ A add(A a, A b) { return df_add(a, b); }
    static __device__ __forceinline__ A sub(A a, A b) { return df_add(a, DF{-b.hi, -b.lo}); }
    static __device__ __forceinline__ A scale(A a, float s) { return df_mul(a, DF{s, 0.0f}); }
    static __device__ __forceinline__ float val(A a) { return a.hi + a.lo; }
    static __device__ __forceinline__ double dval(A a) { return (double)a.hi + (double)a.lo; }
    static __device__ __forceinline__ A ldcg(const A* p)
    {
        const float2 x = __ldcg(reinterpret_cast<const float2*>(p));
        return DF{x.x, x.y};
    }
};
template <>
struct FuOps<double> {
    using A = double;
    using T2 = double2;
    static __device__ __forceinline__ A from(double x) { return x; }
    static __device__ __forceinline__ A add(A a, A b) { return a + b; }
    static __device__ __forceinline__ A sub(A a, A b) { return a - b; }
    static __device__ __forceinline__ A scale(A a, double s) { return a * s; }
    static __device__ __forceinline__ double val(A a) { return a; }
    static __device__ __forceinline__ double dval(A a) { return a; }
    static __device__ __forceinline__ A ldcg(const A* p) { return __ldcg(p); }
};

__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }

constexpr int MB_CHECK = 5;     // mbarrier of the failure-detection check
constexpr int MU_SLOTS = 5;     // column slots of the MUSCL walk (upwind: 3)

struct FuShared {
    DF red[2][8][12];            // per-warp sums (<= 256 threads), by column parity (8-byte A)
    unsigned long long mbar[6];  // column slots 0..4; MB_CHECK: failure-detection check
};

// Byte offsets of the walk's tables after FuShared (host and device); es is
// the element size of f (4 or 8).  A MUSCL walk of S columns computes S + 2
// (its neighbours on both sides too) and keeps five column slots.
struct FuLayout {
    size_t rs, tot, par, vxe, eyz, slots, total;
};

__host__ __device__ inline size_t fu_al16(size_t x) { return (x + 15) / 16 * 16; }

__host__ __device__ inline FuLayout fu_layout(int nvp, int R, int S, int es, int scheme = 0)
{
    FuLayout L;
    const int Wc = scheme ? S + 2 : S;                 // computed columns
    const int nslot = scheme ? MU_SLOTS : 3;
    size_t o = fu_al16(sizeof(FuShared));
    L.rs = o;                                          // A [(Wc+2)][NQ]: rank sums of the computed columns and one each side
    o = fu_al16(o + (size_t)(Wc + 2) * NQ * 8);
    L.tot = o;                                         // A [Wc][5]: P(f*) of each column
    o = fu_al16(o + (size_t)Wc * 5 * 8);
    L.par = o;                                         // T [Wc][8]: Maxwellian parameters (double path)
    o = fu_al16(o + (size_t)Wc * 8 * es);
    L.vxe = o;                                         // T2 [Wc][R]: (v_x, b pref ex) of the CTA's rows
    o = fu_al16(o + (size_t)Wc * R * 2 * es);
    L.eyz = o;                                         // T [Wc][2 nvp]: ey, ez
    o += (size_t)Wc * 2 * nvp * es;
    o = (o + 127) / 128 * 128;
    L.slots = o;                                       // T [nslot][R+2][nvp^2]
    o += (size_t)nslot * (R + 2) * nvp * nvp * es;
    L.total = o;
    return L;
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Sum over the C ranks (stride NQ) in the pairwise order of rank_sum, read
// past L1 (written by other CTAs of the same launch in the persistent run).
template <typename T>
__device__ __forceinline__ typename FuOps<T>::A part_rank_sum(const typename FuOps<T>::A* __restrict__ p, int C)
{
    using O = FuOps<T>;
    typename O::A v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = r < C ? O::ldcg(p + (size_t)r * NQ) : O::from(T(0));
#pragma unroll
    for (int w = 1; w < 16; w *= 2)
#pragma unroll
        for (int r = 0; r + w < 16; r += 2 * w) v[r] = O::add(v[r], v[r + w]);
    return v[0];
}

// Maxwellian parameters of a column from its P(f*) sums (without dv3): the
// float path's double-float function, or the double path's.
__device__ __forceinline__ void fu_params(DF* tot, float*, const FInst& I, bool report, int* status)
{
    maxwell_params_f(tot, reinterpret_cast<float*>(tot), I.dv3, report, status);  // FPar over tot
}
__device__ __forceinline__ void fu_params(const double* tot, double* par, const FInst& I, bool report, int* status)
{
    double t[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) t[k] = tot[k] * I.dv3;
    maxwell_params_d(t, par, report, status);
}

// Packed float32 pairs (two (v_y, v_z) lanes per instruction; IEEE
// round-to-nearest in each lane, so each lane's value is the scalar
// operation's): lanes 2p, 2p+1 of a row, and a - b as b (-1) + a (exact
// product, one rounding).
__device__ __forceinline__ float2 f2at(const float* x, int p) { return make_float2(x[2 * p], x[2 * p + 1]); }
__device__ __forceinline__ void f2put(float* x, int p, float2 v)
{
    x[2 * p] = v.x;
    x[2 * p + 1] = v.y;
}
__device__ __forceinline__ float2 splat(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

// Per-thread sums of f^{n+1} over the thread's rows: per lane sum f and
// sum v_x f; per row (vs = the row's lane sum) sum v_x vs, v_x^2 vs, v_x^3 vs
// and the first / last row's vs.
template <typename T, int VEC>
struct FuAcc {
    T S0[VEC], Tx[VEC], R1, R2, R3, e0, en;
};

template <typename T, int VEC>
__device__ __forceinline__ void fu_clear(FuAcc<T, VEC>& s)
{
#pragma unroll
    for (int l = 0; l < VEC; ++l) s.S0[l] = s.Tx[l] = T(0);
    s.R1 = s.R2 = s.R3 = s.e0 = s.en = T(0);
}

// Row sums without the end-row densities (rows inside the box).
template <typename T, int VEC>
__device__ __forceinline__ T fu_row_in(FuAcc<T, VEC>& s, const Pack<T, VEC>& v, T vx)
{
    T vs = T(0);
#pragma unroll
    for (int l = 0; l < VEC; ++l) {
        s.S0[l] += v.x[l];
        s.Tx[l] = tfma(vx, v.x[l], s.Tx[l]);
        vs += v.x[l];
    }
    const T vx2 = vx * vx;
    s.R1 = tfma(vx, vs, s.R1);
    s.R2 = tfma(vx2, vs, s.R2);
    s.R3 = tfma(vx2 * vx, vs, s.R3);
    return vs;
}

template <typename T, int VEC>
__device__ __forceinline__ void fu_row(FuAcc<T, VEC>& s, const Pack<T, VEC>& v, T vx, int r, int nvx)
{
    const T vs = fu_row_in(s, v, vx);
    if (r == 0) s.e0 = vs;
    if (r == nvx - 1) s.en = vs;
}

// One exchange of the transposed butterfly over lane bit w: lanes with the
// bit clear keep values 0..n-1 and send n..2n-1 (the others the reverse); each
// keeps the sum of its half with its partner's.
template <int n, typename T>
__device__ __forceinline__ void fu_xchg(T (&x)[16], int lane, int w)
{
    const bool up = (lane & w) != 0;
#pragma unroll
    for (int j = 0; j < n; ++j) {
        const T send = up ? x[j] : x[j + n];
        const T keep = up ? x[j + n] : x[j];
        x[j] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
}

// CTA sums of the accumulators into the 17 partials of one column at dst
// (threads < NQ write): M from every row; A into A+ (rows with v_x > 0) or A-
// (the other CTAs); the end-row densities from the CTAs holding those rows.
// S0, R1, R2: sum f, sum v_x vs, sum v_x^2 vs; Tx, RA2, RA3: sum v_x g,
// sum v_x^2 gs, sum v_x^3 gs of the values g the half sums A take (f for
// upwind fluxes, f +- s/2 for MUSCL).
template <typename T, int VEC>
__device__ __forceinline__ void fu_reduce_sums(const T (&S0)[VEC], const T (&Tx)[VEC], T R1, T R2, T RA2, T RA3,
                                               T e0, T en, const T (&vy)[VEC], const T (&vz)[VEC],
                                               const T (&vp2)[VEC], typename FuOps<T>::A (*red)[12], bool posc,
                                               bool has0, bool hasn, typename FuOps<T>::A* __restrict__ dst)
{
    using O = FuOps<T>;
    T val[12];
    val[0] = val[2] = val[3] = val[4] = val[5] = val[7] = val[8] = val[9] = T(0);
#pragma unroll
    for (int l = 0; l < VEC; ++l) {
        val[0] += S0[l];
        val[2] += vy[l] * S0[l];
        val[3] += vz[l] * S0[l];
        val[4] += vp2[l] * S0[l];
        val[5] += Tx[l];
        val[7] += vy[l] * Tx[l];
        val[8] += vz[l] * Tx[l];
        val[9] += vp2[l] * Tx[l];
    }
    val[1] = R1;
    val[4] += R2;
    val[6] = RA2;
    val[9] += RA3;
    val[10] = e0;
    val[11] = en;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // transposed butterfly: each exchange halves the values a lane keeps, so
    // 8 + 4 + 2 + 1 + 1 shuffles leave lanes 2q, 2q+1 with the warp sum of
    // value q (12..15 are padding)
    T x[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) x[q] = q < 12 ? val[q] : T(0);
    fu_xchg<8>(x, lane, 16);
    fu_xchg<4>(x, lane, 8);
    fu_xchg<2>(x, lane, 4);
    fu_xchg<1>(x, lane, 2);
    x[0] += __shfl_xor_sync(0xffffffffu, x[0], 1);
    if (!(lane & 1) && lane < 24) red[w][lane >> 1] = O::from(x[0]);
    __syncthreads();
    if (threadIdx.x < NQ) {
        const int q = threadIdx.x;
        int src;
        if (q < 5) src = q;
        else if (q < 10) src = posc ? q : -1;
        else if (q < 15) src = posc ? -1 : q - 5;
        else src = q == 15 ? (has0 ? 10 : -1) : (hasn ? 11 : -1);
        typename O::A a = O::from(T(0));
        if (src >= 0) {
            const int nw = (blockDim.x + 31) >> 5;
            for (int k = 0; k < nw; ++k) a = O::add(a, red[k][src]);
        }
        dst[q] = a;
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void fu_reduce(const FuAcc<T, VEC>& s, const T (&vy)[VEC], const T (&vz)[VEC],
                                          const T (&vp2)[VEC], typename FuOps<T>::A (*red)[12], bool posc,
                                          bool has0, bool hasn, typename FuOps<T>::A* __restrict__ dst)
{
    fu_reduce_sums(s.S0, s.Tx, s.R1, s.R2, s.R2, s.R3, s.e0, s.en, vy, vz, vp2, red, posc, has0, hasn, dst);
}

// Uniform per-column constants of the pass.
template <typename T>
struct FuCol {
    T nu, gE, gM;   // dt/dx; dt/dv_x E/2 and dt/dv_x E_max/2
    T a;            // f^{n+1} = a f* + ex ey ez (b M folded into the tables); 1 without collisions
    T hE, hEm;      // E/2, E_max/2 (box-end rows)
    T nuv;
};

// One column's pass over the thread's rows [ra, rb): f* (upwind x flux
// against the neighbour slot, v_x Rusanov flux, combined on interior rows),
// f^{n+1} stored with 16-byte stores, its sums accumulated.  POS: the rows
// take the x flux from column c-1 (v_x > 0); BND: the CTA holds a box-end
// row (zero v_x flux through +-L); NVPC: nvp when > 0.
template <bool POS, bool BND, int NVPC, typename T, int VEC>
__device__ __forceinline__ void fu_pass(const T* __restrict__ cen, const T* __restrict__ nb, T* __restrict__ out,
                                        const typename FuOps<T>::T2* __restrict__ vxe, int ra, int rb, int r0,
                                        int nvx, int nvp2_rt, const FuCol<T>& k, const T (&myz)[VEC],
                                        FuAcc<T, VEC>& acc)
{
    const int nvp2 = NVPC > 0 ? NVPC * NVPC : nvp2_rt;
    Pack<T, VEC> dnv, cv;
#pragma unroll
    for (int l = 0; l < VEC; ++l) dnv.x[l] = T(0);
    if (!BND || ra > 0) dnv = ldv<T, VEC>(cen + (size_t)(ra - r0) * nvp2);
    cv = ldv<T, VEC>(cen + (size_t)(ra - r0 + 1) * nvp2);
    const T* cp = cen + (size_t)(ra - r0 + 2) * nvp2;  // row r+1
    const T* np = nb + (size_t)(ra - r0 + 1) * nvp2;   // neighbour row r
    T* op = out + (size_t)ra * nvp2;
#pragma unroll 4
    for (int r = ra; r < rb; ++r) {
        Pack<T, VEC> up;
        if (!BND || r < nvx - 1) up = ldv<T, VEC>(cp);
        else {
#pragma unroll
            for (int l = 0; l < VEC; ++l) up.x[l] = T(0);
        }
        const typename FuOps<T>::T2 ve = vxe[r - r0];
        const T vx = ve.x, nvx_ = k.nu * ve.x;
        const Pack<T, VEC> x1 = ldv<T, VEC>(np);
        Pack<T, VEC> v;
        if (!BND || (r > 0 && r < nvx - 1)) {
            if constexpr (sizeof(T) == sizeof(float)) {
                // lane pairs: the same operations, two lanes per instruction
#pragma unroll
                for (int p = 0; p < VEC / 2; ++p) {
                    const float2 cc = f2at(cv.x, p), u = f2at(up.x, p), d = f2at(dnv.x, p), xl = f2at(x1.x, p);
                    float2 fs = __ffma2_rn(splat(-nvx_), POS ? psub(cc, xl) : psub(xl, cc), cc);
                    fs = __ffma2_rn(splat(-k.gE), psub(u, d), fs);
                    fs = __ffma2_rn(splat(k.gM), __ffma2_rn(splat(-2.0f), cc, __fadd2_rn(u, d)), fs);
                    f2put(v.x, p, __ffma2_rn(splat(k.a), fs, __fmul2_rn(splat(ve.y), f2at(myz, p))));
                }
            } else {
#pragma unroll
                for (int l = 0; l < VEC; ++l) {
                    const T cc = cv.x[l], u = up.x[l], d = dnv.x[l];
                    T fs = tfma(-nvx_, POS ? cc - x1.x[l] : x1.x[l] - cc, cc);
                    fs = tfma(-k.gE, u - d, fs);
                    fs = tfma(k.gM, tfma(T(-2), cc, u + d), fs);
                    v.x[l] = tfma(k.a, fs, ve.y * myz[l]);
                }
            }
        } else {
#pragma unroll
            for (int l = 0; l < VEC; ++l) {
                const T cc = cv.x[l], u = up.x[l], d = dnv.x[l];
                const T Gr = r < nvx - 1 ? k.hE * (cc + u) - k.hEm * (u - cc) : T(0);
                const T Gl = r > 0 ? k.hE * (d + cc) - k.hEm * (cc - d) : T(0);
                T fs = tfma(-nvx_, POS ? cc - x1.x[l] : x1.x[l] - cc, cc);
                fs = tfma(-k.nuv, Gr - Gl, fs);
                v.x[l] = tfma(k.a, fs, ve.y * myz[l]);
            }
        }
        stv<T, VEC>(op, v);
        if (BND) fu_row(acc, v, vx, r, nvx);
        else fu_row_in(acc, v, vx);
        dnv = cv;
        cv = up;
        cp += nvp2;
        np += nvp2;
        op += nvp2;
    }
}

// mbarriers of the three column slots (and the failure-detection check's)
// at the start of the CTA's shared memory; thread 0 initialises, all wait.
__device__ __forceinline__ void fu_init_mbar(unsigned char* fsm, int poison)
{
    FuShared& sh = *reinterpret_cast<FuShared*>(fsm);
    const uint32_t mbar0 = smem_addr(&sh.mbar[0]);
    if (threadIdx.x == 0) {
        for (int k = 0; k <= MB_CHECK; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar0 + 8u * k), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (poison)  // 16 bytes that no copy delivers: the wait on it runs out
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar0 + 8u * MB_CHECK),
                         "r"(16)
                         : "memory");
    }
    __syncthreads();
}

// One walk of the fused step: columns [wk S, wk S + S) of instance b, the v_x
// rows of CTA `rank` of C, step `step` of the run (state buffer
// cur[b] ^ (step & 1)).  The slot mbarriers are initialised by the caller;
// `phase` carries their parities from one walk to the next (every copy a walk
// issues, it also waits for).  Ends after the last column's partials are
// written by threads < 17 (no barrier after them).
template <typename T, int NVPC>
__device__ __forceinline__ void fused_walk(const FInst* __restrict__ insts, const FGeom& g, const int* __restrict__ cur,
                                           int b, int wk, int rank, int C, int step, int* __restrict__ status,
                                           long long wait_ns, uint32_t& phase, unsigned char* fsm)
{
    using O = FuOps<T>;
    using A = typename O::A;
    using T2 = typename O::T2;
    constexpr int VEC = 16 / (int)sizeof(T);
    const FInst& I = insts[b];
    const int S = g.march, nx = I.nx, bc = I.bc;
    const int i0 = wk * S, i1 = min(i0 + S, nx), W = i1 - i0;
    const int nvx = g.nvx, nvp = NVPC > 0 ? NVPC : g.nvp, nvp2 = nvp * nvp;
    const long long ncol = g.ncol;
    const int R = g.rows;
    const int r0 = rank * R, r1 = min(r0 + R, nvx), nr = r1 - r0;
    const bool posc = r0 >= I.hpos;  // all rows of this CTA have v_x > 0 (else all <= 0)
    const int dn = posc ? -1 : 1;
    const size_t slot_elems = (size_t)(R + 2) * nvp2;

    FuShared& sh = *reinterpret_cast<FuShared*>(fsm);
    A (*red)[8][12] = reinterpret_cast<A (*)[8][12]>(&sh.red[0][0][0]);
    const FuLayout lay = fu_layout(nvp, R, S, (int)sizeof(T));
    A* rs = reinterpret_cast<A*>(fsm + lay.rs);
    A* tot = reinterpret_cast<A*>(fsm + lay.tot);
    T* par = reinterpret_cast<T*>(fsm + lay.par);
    T2* vxe = reinterpret_cast<T2*>(fsm + lay.vxe);
    T* eyz = reinterpret_cast<T*>(fsm + lay.eyz);
    T* slots = reinterpret_cast<T*>(fsm + lay.slots);
    const uint32_t mbar0 = smem_addr(&sh.mbar[0]);

    const int Lr = nvp2 / VEC, G = g.groups;
    const int q = threadIdx.x % Lr, grp = threadIdx.x / Lr;
    const int jp = q * VEC;
    const int Rg = (nr + G - 1) / G;
    const int ra = r0 + grp * Rg, rb = min(ra + Rg, r1);
    const bool active = grp < G && ra < rb;
    const int bufi = cur[b] ^ (step & 1);
    const T* __restrict__ fin = static_cast<const T*>(I.f[bufi]);
    T* __restrict__ fout = static_cast<T*>(I.f[bufi ^ 1]);
    const A* __restrict__ pin = static_cast<const A*>(I.part[bufi]);
    A* __restrict__ pout = static_cast<A*>(I.part[bufi ^ 1]);
    const int ha = max(r0 - 1, 0), hb = min(r1 + 1, nvx);

    const int cfirst = posc ? i0 - 1 : i0, clast = posc ? i1 - 1 : i1;
    auto slot_of = [&](int c) { return (c - i0 + 3) % 3; };
    // column c (a ghost through the boundary rule) into its slot: one bulk
    // copy by thread 0, or, for a mirrored ghost (only ever a neighbour),
    // rows r0..r1-1 copied by all threads; true if the slot waits on its mbarrier
    auto load = [&](int c) -> bool {
        bool mir;
        const int sc = ghost_col(c, nx, bc, &mir);
        T* dst = slots + (size_t)slot_of(c) * slot_elems;
        const T* col = fin + (size_t)sc * ncol;
        if (!mir) {
            if (threadIdx.x == 0) {
                const uint32_t mb = mbar0 + 8u * (uint32_t)slot_of(c);
                const uint32_t bytes = (uint32_t)(hb - ha) * nvp2 * (uint32_t)sizeof(T);
                fence_proxy_async();
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_addr(dst + (size_t)(ha - (r0 - 1)) * nvp2)),
                    "l"(col + (size_t)ha * nvp2), "r"(bytes), "r"(mb)
                    : "memory");
            }
            return true;
        }
        for (int e = threadIdx.x; e < nr * nvp2; e += blockDim.x) {
            const int r = r0 + e / nvp2, j = e - (e / nvp2) * nvp2;
            dst[(size_t)(r - r0 + 1) * nvp2 + j] = __ldcg(col + (size_t)(nvx - 1 - r) * nvp2 + j);
        }
        fence_proxy_async();  // a later bulk copy into this slot comes after these stores
        return false;
    };

    uint32_t pend = 0;
    for (int c = cfirst; c < cfirst + 3 && c <= clast; ++c)
        if (load(c)) pend |= 1u << slot_of(c);

    // the walk's Maxwellians, while the copies land: rank sums of the
    // partials of columns i0-1 .. i1 (ghosts raw), then P(f*) per column
    const T* vt = static_cast<const T*>(I.vtab);
    for (int t = threadIdx.x; t < (W + 2) * NQ; t += blockDim.x) {
        const int j = t / NQ, qq = t - j * NQ;
        bool mir;
        const int src = ghost_col(i0 - 1 + j, nx, bc, &mir);
        rs[t] = part_rank_sum<T>(pin + (size_t)src * C * NQ + qq, C);
    }
    __syncthreads();
    const T nu = scal<T>(I.nu, I.fnu), nuv = scal<T>(I.nuv, I.fnuv), Emax = scal<T>(I.Emax, I.fEmax);
    for (int t5 = threadIdx.x; t5 < W * 5; t5 += blockDim.x) {
        const int j = t5 / 5, k = t5 - 5 * j, c = i0 + j;
        const A* Mc = rs + (size_t)(j + 1) * NQ;
        const A* Lc = rs + (size_t)j * NQ;
        const A* Rc = rs + (size_t)(j + 2) * NQ;
        const T sk = k == 1 ? T(1) : T(-1);
        const bool mirL = bc == 2 && c == 0, mirR = bc == 2 && c == nx - 1;
        const A Apl = mirL ? O::scale(Lc[10 + k], sk) : Lc[5 + k];  // A+ of column c-1
        const A Amr = mirR ? O::scale(Rc[5 + k], sk) : Rc[10 + k];  // A- of column c+1
        const A fl = O::add(O::sub(Mc[5 + k], Apl), O::sub(Amr, Mc[10 + k]));
        A t = O::sub(Mc[k], O::scale(fl, nu));
        if (k == 1 || k == 4) {
            const T dvx = (T)I.dvx, Lb = (T)I.L, E = scal<T>(I.E[c], I.Ef[c]);
            const T M0 = O::val(Mc[0]), M1 = O::val(Mc[1]);
            const T e0 = O::val(Mc[15]), en = O::val(Mc[16]);
            const T Q = k == 1 ? -dvx * (E * (M0 - T(0.5) * (e0 + en)) - Emax * T(0.5) * (en - e0))
                               : -dvx * (E * (T(2) * M1 - Lb * (en - e0)) - Emax * (Lb * (e0 + en) - dvx * M0));
            t = O::sub(t, O::from(nuv * Q));
        }
        tot[j * 5 + k] = t;
    }
    __syncthreads();
    // (float path: each column's parameter pairs FPar replace its five
    // double-float totals, read first; double path: par [8] per column)
    for (int j = threadIdx.x; j < W; j += blockDim.x) fu_params(tot + j * 5, par + j * 8, I, I.collide && rank == 0, status);
    __syncthreads();
    // per column: (v_x, b pref ex) of the rows and ey, ez (float32: each
    // factor from the pair parameters within ~1e-9 before its rounding, as in
    // the clustered step); zero tables without collisions
    const bool collide = I.collide != 0;
    const T bb = scal<T>(I.b, I.fb);
    for (int t = threadIdx.x; t < W * (nr + 2 * nvp); t += blockDim.x) {
        const int j = t / (nr + 2 * nvp), k = t - j * (nr + 2 * nvp);
        const T* pj = par + j * 8;
        if (k < nr) {
            const T vx = vt[r0 + k];
            T2 e;
            e.x = vx;
            if constexpr (sizeof(T) == sizeof(float)) {
                const FPar& P = *reinterpret_cast<const FPar*>(tot + j * 5);
                const F2* vp = reinterpret_cast<const F2*>(I.vpair);
                e.y = collide ? gauss_f2(vp[r0 + k], P.u[0], P.i2t, f2_mul(F2{(float)bb, 0.0f}, P.pref)) : T(0);
            } else {
                const T cx = vx - pj[1];
                e.y = collide ? bb * pj[5] * texp(-cx * cx * pj[6]) : T(0);
            }
            vxe[j * R + k] = e;
        } else {
            const int m = k - nr < nvp ? k - nr : k - nr - nvp;
            T val;
            if constexpr (sizeof(T) == sizeof(float)) {
                const FPar& P = *reinterpret_cast<const FPar*>(tot + j * 5);
                const F2* vp = reinterpret_cast<const F2*>(I.vpair);
                val = gauss_f2(vp[nvx + m], P.u[k - nr < nvp ? 1 : 2], P.i2t, F2{1.0f, 0.0f});
            } else {
                const T cc = vt[nvx + m * nvp] - (k - nr < nvp ? pj[2] : pj[3]);
                val = texp(-cc * cc * pj[6]);
            }
            eyz[j * 2 * nvp + (k - nr)] = collide ? val : T(0);
        }
    }
    T vy[VEC], vz[VEC], vp2[VEC];
    int jy[VEC], jz[VEC];
    {
        int y = jp / nvp, z = jp - (jp / nvp) * nvp;
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
            vy[l] = active ? vt[nvx + jp + l] : T(0);
            vz[l] = active ? vt[nvx + nvp2 + jp + l] : T(0);
            vp2[l] = active ? vt[nvx + 2 * nvp2 + jp + l] : T(0);
            jy[l] = y;
            jz[l] = z;
            if (++z == nvp) {
                z = 0;
                ++y;
            }
        }
    }
    FuCol<T> kc;
    kc.nu = nu;
    kc.nuv = nuv;
    kc.hEm = T(0.5) * Emax;
    kc.gM = nuv * kc.hEm;
    kc.a = collide ? scal<T>(I.a, I.fa) : T(1);
    const bool has0 = r0 == 0, hasn = r1 == nvx, bnd = has0 || hasn;
    __syncthreads();  // tables and thread-staged slots visible

    for (int c = i0; c < i1; ++c) {
        const int j = c - i0;
        const int sc = slot_of(c), sn = slot_of(c + dn);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int s = k == 0 ? sc : sn;
            if (pend & (1u << s)) {
                const uint32_t mb = mbar0 + 8u * (uint32_t)s, ph = (phase >> s) & 1u;
                if (!mbar_wait(mb, wait_ns, ph)) {
                    atomicCAS(status, 0, ST_TIMEOUT);
                    mbar_wait(mb, wait_ns, ph);  // let the copy land before the slot is reused
                }
                pend &= ~(1u << s);
                phase ^= 1u << s;
            }
        }
        const T* cen = slots + (size_t)sc * slot_elems + jp;
        const T* nb = slots + (size_t)sn * slot_elems + jp;
        kc.hE = T(0.5) * scal<T>(I.E[c], I.Ef[c]);
        kc.gE = nuv * kc.hE;
        T myz[VEC];
        {
            const T* ey = eyz + j * 2 * nvp;
#pragma unroll
            for (int l = 0; l < VEC; ++l) myz[l] = ey[jy[l]] * ey[nvp + jz[l]];
        }
        FuAcc<T, VEC> acc;
        fu_clear(acc);
        if (active) {
            T* out = fout + (size_t)c * ncol + jp;
            const T2* ve = vxe + j * R;
            if (posc) {
                if (bnd) fu_pass<true, true, NVPC>(cen, nb, out, ve, ra, rb, r0, nvx, nvp2, kc, myz, acc);
                else fu_pass<true, false, NVPC>(cen, nb, out, ve, ra, rb, r0, nvx, nvp2, kc, myz, acc);
            } else {
                if (bnd) fu_pass<false, true, NVPC>(cen, nb, out, ve, ra, rb, r0, nvx, nvp2, kc, myz, acc);
                else fu_pass<false, false, NVPC>(cen, nb, out, ve, ra, rb, r0, nvx, nvp2, kc, myz, acc);
            }
        }
        // the 17 sums of f^{n+1} of this column; the reduction's barrier ends
        // every read of this column's slots
        fu_reduce(acc, vy, vz, vp2, red[c & 1], posc, has0, hasn, pout + ((size_t)c * C + rank) * NQ);
        {
            const int nc = posc ? c + 2 : c + 3;
            if (nc <= clast && load(nc)) pend |= 1u << slot_of(nc);
        }
    }
}

// ---- fused single-pass step with MUSCL-minmod x fluxes ----
//
// The interface value on the upwind side of face c+1/2 is f_c + s_c/2
// (v_x > 0) or f_{c+1} - s_{c+1}/2 (v_x <= 0), s_c = minmod(f_c - f_{c-1},
// f_{c+1} - f_c), so the column-sum identity of the upwind step holds with
// A+ and A- taken of f + s/2 and f - s/2 (v_x Rusanov fluxes unchanged).  The
// 17 partials keep their layout; the slope of f^{n+1} in column c needs
// f^{n+1} of columns c-1 and c+1, so a walk also computes (without storing
// them) the column on each side of its own, keeps each lane's last two
// outputs in registers, and writes the sums of column c-1 once column c is
// computed.  The transport of column c reads f^n of columns c-2 .. c+1
// (v_x > 0) or c-1 .. c+2 (v_x <= 0): five column slots rotate, four in use
// and the next copy in flight.  Periodic and outflow boundaries: an outflow
// edge column's slope is zero (its ghost repeats it), so a wall's outside
// neighbour is not computed; a reflecting wall keeps the clustered step.

// Branch-free minmod: the value of smaller magnitude when a and b have the
// same sign, else 0 (equal to minmod() for every finite pair).
__device__ __forceinline__ float mm2(float a, float b) { return fminf(fmaxf(b, fminf(a, 0.0f)), fmaxf(a, 0.0f)); }
// float64: the same selection on the IEEE bit patterns with integer
// operations (equal sign bits: the smaller magnitude, else 0), off this
// part's reduced-rate FP64 pipe
__device__ __forceinline__ double mm2(double a, double b)
{
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    const long long ma = ia & 0x7fffffffffffffffLL, mb = ib & 0x7fffffffffffffffLL;
    return (ia ^ ib) >= 0 ? __longlong_as_double(ma < mb ? ia : ib) : 0.0;
}
__device__ __forceinline__ float mmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float mmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double mmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ double mmax(double a, double b) { return fmax(a, b); }

// The limiter per lane of a packed pair.
__device__ __forceinline__ float2 pmm2(float2 a, float2 b) { return make_float2(mm2(a.x, b.x), mm2(a.y, b.y)); }

// Sums of one column of f^{n+1} (values h of its rows) with the limited
// half-sum values g = h +- s/2 (sign + for rows with v_x > 0).
template <typename T, int VEC>
struct FuAccM {
    T S0[VEC], Tx[VEC], R1, R2, RA2, RA3, e0, en;
};

template <typename T, int VEC>
__device__ __forceinline__ void fu_clear(FuAccM<T, VEC>& s)
{
#pragma unroll
    for (int l = 0; l < VEC; ++l) s.S0[l] = s.Tx[l] = T(0);
    s.R1 = s.R2 = s.RA2 = s.RA3 = s.e0 = s.en = T(0);
}

// One row of a column's sums: h its values, g the limited values.
template <bool BND, typename T, int VEC>
__device__ __forceinline__ void fu_row_m(FuAccM<T, VEC>& s, const T (&h)[VEC], const T (&g)[VEC], T vx, int r,
                                         int nvx)
{
    T vs = T(0), gs = T(0);
    if constexpr (sizeof(T) == sizeof(float)) {
        // in lane pairs; the row sums add the pair's two lanes last
        float2 vs2 = f2at(h, 0), gs2 = f2at(g, 0);
#pragma unroll
        for (int p = 0; p < VEC / 2; ++p) {
            f2put(s.S0, p, __fadd2_rn(f2at(s.S0, p), f2at(h, p)));
            f2put(s.Tx, p, __ffma2_rn(splat(vx), f2at(g, p), f2at(s.Tx, p)));
            if (p > 0) {
                vs2 = __fadd2_rn(vs2, f2at(h, p));
                gs2 = __fadd2_rn(gs2, f2at(g, p));
            }
        }
        vs = vs2.x + vs2.y;
        gs = gs2.x + gs2.y;
    } else {
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
            s.S0[l] += h[l];
            s.Tx[l] = tfma(vx, g[l], s.Tx[l]);
            vs += h[l];
            gs += g[l];
        }
    }
    const T vx2 = vx * vx;
    s.R1 = tfma(vx, vs, s.R1);
    s.R2 = tfma(vx2, vs, s.R2);
    s.RA2 = tfma(vx2, gs, s.RA2);
    s.RA3 = tfma(vx2 * vx, gs, s.RA3);
    if (BND) {
        if (r == 0) s.e0 = vs;
        if (r == nvx - 1) s.en = vs;
    }
}

// One computed column's pass over the thread's rows [ra, rb) (at most RG):
// f* from the limited x fluxes and the v_x Rusanov flux, f^{n+1} = a f* + b M
// stored when `out` is set.  cen: this column's slot with its row halo; x1,
// xf: the upwind neighbour and the one beyond it; xd: the downwind
// neighbour; sgn = +1 for rows with v_x > 0, -1 otherwise.  With the
// differences e = f_c - f_x1, d1 = f_xd - f_c, d2 = f_x1 - f_xf the flux
// difference over v_x is sgn (e + (minmod(e, d1) - minmod(e, d2)) / 2) for
// either sign (minmod is odd), so one formula serves both.  With `sums`, the
// sums of the previous computed column h1 (slope from dd = h1 - its own
// predecessor and this column's f^{n+1} - h1); then dd <- f^{n+1} - h1 (0 when
// `dup`: the first column next to an outflow wall) and h1 <- f^{n+1}.
template <bool BND, int NVPC, int RG, typename T, int VEC>
__device__ __forceinline__ void fu_pass_m(const T* __restrict__ cen, const T* __restrict__ x1s,
                                          const T* __restrict__ xfs, const T* __restrict__ xds, T* __restrict__ out,
                                          const typename FuOps<T>::T2* __restrict__ vxe, int ra, int rb, int r0,
                                          int nvx, int nvp2_rt, const FuCol<T>& k, T sgn, const T (&myz)[VEC],
                                          bool sums, bool dup, T (&h1)[RG][VEC], T (&dd)[RG][VEC],
                                          FuAccM<T, VEC>& acc)
{
    const int nvp2 = NVPC > 0 ? NVPC * NVPC : nvp2_rt;
    const T nus = sgn * k.nu, hs = T(0.5) * sgn;
    Pack<T, VEC> dnv, cv;
#pragma unroll
    for (int l = 0; l < VEC; ++l) dnv.x[l] = T(0);
    if (!BND || ra > 0) dnv = ldv<T, VEC>(cen + (size_t)(ra - r0) * nvp2);
    cv = ldv<T, VEC>(cen + (size_t)(ra - r0 + 1) * nvp2);
    const size_t o = (size_t)(ra - r0 + 1) * nvp2;  // row ra in a slot
#pragma unroll
    for (int i = 0; i < RG; ++i) {
        const int r = ra + i;
        if (r < rb) {
            Pack<T, VEC> up;
            if (!BND || r < nvx - 1) up = ldv<T, VEC>(cen + o + (size_t)(i + 1) * nvp2);
            else {
#pragma unroll
                for (int l = 0; l < VEC; ++l) up.x[l] = T(0);
            }
            const typename FuOps<T>::T2 ve = vxe[r - r0];
            const T vx = ve.x, nvx_ = nus * ve.x;
            const Pack<T, VEC> a1 = ldv<T, VEC>(x1s + o + (size_t)i * nvp2);
            const Pack<T, VEC> af = ldv<T, VEC>(xfs + o + (size_t)i * nvp2);
            const Pack<T, VEC> ad = ldv<T, VEC>(xds + o + (size_t)i * nvp2);
            T v[VEC], dn[VEC];
            if constexpr (sizeof(T) == sizeof(float)) {
                // lane pairs: the same operations, two lanes per instruction
                // (the limiters, scalar, as clamps: minmod(e, x) = x clamped
                // to [min(e, 0), max(e, 0)])
                const bool inner = !BND || (r > 0 && r < nvx - 1);
#pragma unroll
                for (int p = 0; p < VEC / 2; ++p) {
                    const float2 cc = f2at(cv.x, p), u = f2at(up.x, p), d = f2at(dnv.x, p), a1p = f2at(a1.x, p);
                    const float2 e = psub(cc, a1p), d1 = psub(f2at(ad.x, p), cc), d2 = psub(a1p, f2at(af.x, p));
                    const float lx = mmin(e.x, 0.0f), hx = mmax(e.x, 0.0f), ly = mmin(e.y, 0.0f), hy = mmax(e.y, 0.0f);
                    const float2 c1 = make_float2(mmin(mmax(d1.x, lx), hx), mmin(mmax(d1.y, ly), hy));
                    const float2 c2 = make_float2(mmin(mmax(d2.x, lx), hx), mmin(mmax(d2.y, ly), hy));
                    float2 fs = __ffma2_rn(splat(-nvx_), __ffma2_rn(splat(0.5f), psub(c1, c2), e), cc);
                    if (inner) {
                        fs = __ffma2_rn(splat(-k.gE), psub(u, d), fs);
                        fs = __ffma2_rn(splat(k.gM), __ffma2_rn(splat(-2.0f), cc, __fadd2_rn(u, d)), fs);
                    } else {
                        float fl[2] = {fs.x, fs.y};
                        const float cl[2] = {cc.x, cc.y}, ul[2] = {u.x, u.y}, dl[2] = {d.x, d.y};
#pragma unroll
                        for (int l = 0; l < 2; ++l) {
                            const float Gr = r < nvx - 1 ? k.hE * (cl[l] + ul[l]) - k.hEm * (ul[l] - cl[l]) : 0.0f;
                            const float Gl = r > 0 ? k.hE * (dl[l] + cl[l]) - k.hEm * (cl[l] - dl[l]) : 0.0f;
                            fl[l] = tfma(-k.nuv, Gr - Gl, fl[l]);
                        }
                        fs = make_float2(fl[0], fl[1]);
                    }
                    const float2 vp = __ffma2_rn(splat(k.a), fs, __fmul2_rn(splat(ve.y), f2at(myz, p)));
                    f2put(v, p, vp);
                    f2put(dn, p, psub(vp, f2at(h1[i], p)));
                }
            } else {
#pragma unroll
                for (int l = 0; l < VEC; ++l) {
                    const T cc = cv.x[l], u = up.x[l], d = dnv.x[l];
                    const T e = cc - a1.x[l], d1 = ad.x[l] - cc, d2 = a1.x[l] - af.x[l];
                    const T D = tfma(T(0.5), mm2(e, d1) - mm2(e, d2), e);
                    T fs = tfma(-nvx_, D, cc);
                    if (!BND || (r > 0 && r < nvx - 1)) {
                        fs = tfma(-k.gE, u - d, fs);
                        fs = tfma(k.gM, tfma(T(-2), cc, u + d), fs);
                    } else {
                        const T Gr = r < nvx - 1 ? k.hE * (cc + u) - k.hEm * (u - cc) : T(0);
                        const T Gl = r > 0 ? k.hE * (d + cc) - k.hEm * (cc - d) : T(0);
                        fs = tfma(-k.nuv, Gr - Gl, fs);
                    }
                    v[l] = tfma(k.a, fs, ve.y * myz[l]);
                    dn[l] = v[l] - h1[i][l];
                }
            }
            if (out) {
                Pack<T, VEC> pv;
#pragma unroll
                for (int l = 0; l < VEC; ++l) pv.x[l] = v[l];
                stv<T, VEC>(out + (size_t)r * nvp2, pv);
            }
            if (sums) {
                T g[VEC];
                if constexpr (sizeof(T) == sizeof(float)) {
#pragma unroll
                    for (int p = 0; p < VEC / 2; ++p)
                        f2put(g, p, __ffma2_rn(splat(hs), pmm2(f2at(dd[i], p), f2at(dn, p)), f2at(h1[i], p)));
                } else {
#pragma unroll
                    for (int l = 0; l < VEC; ++l) g[l] = tfma(hs, mm2(dd[i][l], dn[l]), h1[i][l]);
                }
                fu_row_m<BND>(acc, h1[i], g, vx, r, nvx);
            }
#pragma unroll
            for (int l = 0; l < VEC; ++l) {
                dd[i][l] = dn[l];
                h1[i][l] = v[l];
            }
            dnv = cv;
            cv = up;
        }
    }
    if (dup)
#pragma unroll
        for (int i = 0; i < RG; ++i)
#pragma unroll
            for (int l = 0; l < VEC; ++l) dd[i][l] = T(0);
}

// Sums of the last computed column h1 next to an outflow wall (slope zero).
template <bool BND, int RG, typename T, int VEC>
__device__ __forceinline__ void fu_sums_edge(const typename FuOps<T>::T2* __restrict__ vxe, int ra, int rb, int r0,
                                             int nvx, const T (&h1)[RG][VEC], FuAccM<T, VEC>& acc)
{
#pragma unroll
    for (int i = 0; i < RG; ++i) {
        const int r = ra + i;
        if (r < rb) fu_row_m<BND>(acc, h1[i], h1[i], vxe[r - r0].x, r, nvx);
    }
}

// One MUSCL walk: columns [wk S, wk S + S) of instance b, as fused_walk
// (same arguments, partials and completion rule).
template <typename T, int NVPC, int RG>
__device__ __forceinline__ void fused_walk_m(const FInst* __restrict__ insts, const FGeom& g,
                                             const int* __restrict__ cur, int b, int wk, int rank, int C, int step,
                                             int* __restrict__ status, long long wait_ns, uint32_t& phase,
                                             unsigned char* fsm)
{
    using O = FuOps<T>;
    using A = typename O::A;
    using T2 = typename O::T2;
    constexpr int VEC = 16 / (int)sizeof(T);
    const FInst& I = insts[b];
    const int S = g.march, nx = I.nx, bc = I.bc;
    const int i0 = wk * S, i1 = min(i0 + S, nx);
    const int nvx = g.nvx, nvp = NVPC > 0 ? NVPC : g.nvp, nvp2 = nvp * nvp;
    const long long ncol = g.ncol;
    const int R = g.rows;
    const int r0 = rank * R, r1 = min(r0 + R, nvx), nr = r1 - r0;
    const bool posc = r0 >= I.hpos;  // all rows of this CTA have v_x > 0 (else all <= 0)
    const size_t slot_elems = (size_t)(R + 2) * nvp2;
    // computed columns cs..ce: the walk's own and its neighbours, except
    // outside an outflow wall
    const bool wallL = bc != 0 && i0 == 0, wallR = bc != 0 && i1 == nx;
    const int cs = wallL ? i0 : i0 - 1, ce = wallR ? i1 - 1 : i1, Wc = ce - cs + 1;
    const int back = posc ? 2 : 1;  // column c reads columns c-back .. c-back+3
    const int L0 = cs - back, Lend = ce - back + 3;

    FuShared& sh = *reinterpret_cast<FuShared*>(fsm);
    A (*red)[8][12] = reinterpret_cast<A (*)[8][12]>(&sh.red[0][0][0]);
    const FuLayout lay = fu_layout(nvp, R, S, (int)sizeof(T), 1);
    A* rs = reinterpret_cast<A*>(fsm + lay.rs);
    A* tot = reinterpret_cast<A*>(fsm + lay.tot);
    T* par = reinterpret_cast<T*>(fsm + lay.par);
    T2* vxe = reinterpret_cast<T2*>(fsm + lay.vxe);
    T* eyz = reinterpret_cast<T*>(fsm + lay.eyz);
    T* slots = reinterpret_cast<T*>(fsm + lay.slots);
    const uint32_t mbar0 = smem_addr(&sh.mbar[0]);

    const int Lr = nvp2 / VEC, G = g.groups;
    const int q = threadIdx.x % Lr, grp = threadIdx.x / Lr;
    const int jp = q * VEC;
    const int Rg = (nr + G - 1) / G;
    const int ra = r0 + grp * Rg, rb = min(ra + Rg, r1);
    const bool active = grp < G && ra < rb;
    const int bufi = cur[b] ^ (step & 1);
    const T* __restrict__ fin = static_cast<const T*>(I.f[bufi]);
    T* __restrict__ fout = static_cast<T*>(I.f[bufi ^ 1]);
    const A* __restrict__ pin = static_cast<const A*>(I.part[bufi]);
    A* __restrict__ pout = static_cast<A*>(I.part[bufi ^ 1]);
    const int ha = max(r0 - 1, 0), hb = min(r1 + 1, nvx);

    auto slot_of = [&](int c) { return (c - L0) % MU_SLOTS; };
    // column c (through the boundary rule: periodic wrap or outflow repeat)
    // into its slot with one bulk copy by thread 0
    auto load = [&](int c) {
        bool mir;
        const int sc = ghost_col(c, nx, bc, &mir);
        if (threadIdx.x == 0) {
            T* dst = slots + (size_t)slot_of(c) * slot_elems;
            const T* col = fin + (size_t)sc * ncol;
            const uint32_t mb = mbar0 + 8u * (uint32_t)slot_of(c);
            const uint32_t bytes = (uint32_t)(hb - ha) * nvp2 * (uint32_t)sizeof(T);
            fence_proxy_async();
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_addr(dst + (size_t)(ha - (r0 - 1)) * nvp2)),
                "l"(col + (size_t)ha * nvp2), "r"(bytes), "r"(mb)
                : "memory");
        }
    };

    uint32_t pend = 0;
    for (int c = L0; c < L0 + MU_SLOTS && c <= Lend; ++c) {
        load(c);
        pend |= 1u << slot_of(c);
    }

    // the Maxwellians of the computed columns, while the copies land: rank
    // sums of the partials of columns cs-1 .. ce+1, then P(f*) per column
    const T* vt = static_cast<const T*>(I.vtab);
    for (int t = threadIdx.x; t < (Wc + 2) * NQ; t += blockDim.x) {
        const int j = t / NQ, qq = t - j * NQ;
        bool mir;
        const int src = ghost_col(cs - 1 + j, nx, bc, &mir);
        rs[t] = part_rank_sum<T>(pin + (size_t)src * C * NQ + qq, C);
    }
    __syncthreads();
    const T nu = scal<T>(I.nu, I.fnu), nuv = scal<T>(I.nuv, I.fnuv), Emax = scal<T>(I.Emax, I.fEmax);
    for (int t5 = threadIdx.x; t5 < Wc * 5; t5 += blockDim.x) {
        const int j = t5 / 5, k = t5 - 5 * j;
        bool mir;
        const int c = ghost_col(cs + j, nx, bc, &mir);
        const A* Mc = rs + (size_t)(j + 1) * NQ;
        const A* Lc = rs + (size_t)j * NQ;
        const A* Rc = rs + (size_t)(j + 2) * NQ;
        const A fl = O::add(O::sub(Mc[5 + k], Lc[5 + k]), O::sub(Rc[10 + k], Mc[10 + k]));
        A t = O::sub(Mc[k], O::scale(fl, nu));
        if (k == 1 || k == 4) {
            const T dvx = (T)I.dvx, Lb = (T)I.L, E = scal<T>(I.E[c], I.Ef[c]);
            const T M0 = O::val(Mc[0]), M1 = O::val(Mc[1]);
            const T e0 = O::val(Mc[15]), en = O::val(Mc[16]);
            const T Q = k == 1 ? -dvx * (E * (M0 - T(0.5) * (e0 + en)) - Emax * T(0.5) * (en - e0))
                               : -dvx * (E * (T(2) * M1 - Lb * (en - e0)) - Emax * (Lb * (e0 + en) - dvx * M0));
            t = O::sub(t, O::from(nuv * Q));
        }
        tot[j * 5 + k] = t;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < Wc; j += blockDim.x) {
        const int c = cs + j;
        fu_params(tot + j * 5, par + j * 8, I, I.collide && rank == 0 && c >= i0 && c < i1, status);
    }
    __syncthreads();
    const bool collide = I.collide != 0;
    const T bb = scal<T>(I.b, I.fb);
    for (int t = threadIdx.x; t < Wc * (nr + 2 * nvp); t += blockDim.x) {
        const int j = t / (nr + 2 * nvp), k = t - j * (nr + 2 * nvp);
        const T* pj = par + j * 8;
        if (k < nr) {
            const T vx = vt[r0 + k];
            T2 e;
            e.x = vx;
            if constexpr (sizeof(T) == sizeof(float)) {
                const FPar& P = *reinterpret_cast<const FPar*>(tot + j * 5);
                const F2* vp = reinterpret_cast<const F2*>(I.vpair);
                e.y = collide ? gauss_f2(vp[r0 + k], P.u[0], P.i2t, f2_mul(F2{(float)bb, 0.0f}, P.pref)) : T(0);
            } else {
                const T cx = vx - pj[1];
                e.y = collide ? bb * pj[5] * texp(-cx * cx * pj[6]) : T(0);
            }
            vxe[j * R + k] = e;
        } else {
            const int m = k - nr < nvp ? k - nr : k - nr - nvp;
            T val;
            if constexpr (sizeof(T) == sizeof(float)) {
                const FPar& P = *reinterpret_cast<const FPar*>(tot + j * 5);
                const F2* vp = reinterpret_cast<const F2*>(I.vpair);
                val = gauss_f2(vp[nvx + m], P.u[k - nr < nvp ? 1 : 2], P.i2t, F2{1.0f, 0.0f});
            } else {
                const T cc = vt[nvx + m * nvp] - (k - nr < nvp ? pj[2] : pj[3]);
                val = texp(-cc * cc * pj[6]);
            }
            eyz[j * 2 * nvp + (k - nr)] = collide ? val : T(0);
        }
    }
    T vy[VEC], vz[VEC], vp2[VEC];
    int jy[VEC], jz[VEC];
    {
        int y = jp / nvp, z = jp - (jp / nvp) * nvp;
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
            vy[l] = active ? vt[nvx + jp + l] : T(0);
            vz[l] = active ? vt[nvx + nvp2 + jp + l] : T(0);
            vp2[l] = active ? vt[nvx + 2 * nvp2 + jp + l] : T(0);
            jy[l] = y;
            jz[l] = z;
            if (++z == nvp) {
                z = 0;
                ++y;
            }
        }
    }
    FuCol<T> kc;
    kc.nu = nu;
    kc.nuv = nuv;
    kc.hEm = T(0.5) * Emax;
    kc.gM = nuv * kc.hEm;
    kc.a = collide ? scal<T>(I.a, I.fa) : T(1);
    const bool has0 = r0 == 0, hasn = r1 == nvx, bnd = has0 || hasn;
    T h1[RG][VEC], dd[RG][VEC];
#pragma unroll
    for (int i = 0; i < RG; ++i)
#pragma unroll
        for (int l = 0; l < VEC; ++l) h1[i][l] = dd[i][l] = T(0);
    const T sgn = posc ? T(1) : T(-1);
    __syncthreads();  // tables visible

    for (int c = cs; c <= ce; ++c) {
        const int j = c - cs;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int s = slot_of(c - back + k);
            if (pend & (1u << s)) {
                const uint32_t mb = mbar0 + 8u * (uint32_t)s, ph = (phase >> s) & 1u;
                if (!mbar_wait(mb, wait_ns, ph)) {
                    atomicCAS(status, 0, ST_TIMEOUT);
                    mbar_wait(mb, wait_ns, ph);  // let the copy land before the slot is reused
                }
                pend &= ~(1u << s);
                phase ^= 1u << s;
            }
        }
        const int dn = posc ? -1 : 1;  // the upwind side
        const T* cen = slots + (size_t)slot_of(c) * slot_elems + jp;
        const T* x1s = slots + (size_t)slot_of(c + dn) * slot_elems + jp;
        const T* xfs = slots + (size_t)slot_of(c + 2 * dn) * slot_elems + jp;
        const T* xds = slots + (size_t)slot_of(c - dn) * slot_elems + jp;
        bool mir;
        const int ec = ghost_col(c, nx, bc, &mir);
        kc.hE = T(0.5) * scal<T>(I.E[ec], I.Ef[ec]);
        kc.gE = nuv * kc.hE;
        T myz[VEC];
        {
            const T* ey = eyz + j * 2 * nvp;
#pragma unroll
            for (int l = 0; l < VEC; ++l) myz[l] = ey[jy[l]] * ey[nvp + jz[l]];
        }
        const bool own = c >= i0 && c < i1, sums = c - 1 >= i0 && c - 1 < i1, dup = c == cs && wallL;
        FuAccM<T, VEC> acc;
        fu_clear(acc);
        if (active) {
            T* out = own ? fout + (size_t)c * ncol + jp : nullptr;
            const T2* ve = vxe + j * R;
            if (bnd)
                fu_pass_m<true, NVPC, RG>(cen, x1s, xfs, xds, out, ve, ra, rb, r0, nvx, nvp2, kc, sgn, myz, sums, dup,
                                          h1, dd, acc);
            else
                fu_pass_m<false, NVPC, RG>(cen, x1s, xfs, xds, out, ve, ra, rb, r0, nvx, nvp2, kc, sgn, myz, sums,
                                           dup, h1, dd, acc);
        }
        // the 17 sums of column c-1; the barrier ends every read of column
        // c-back's slot, which the next copy overwrites
        if (sums)
            fu_reduce_sums(acc.S0, acc.Tx, acc.R1, acc.R2, acc.RA2, acc.RA3, acc.e0, acc.en, vy, vz, vp2,
                           red[(c - 1) & 1], posc, has0, hasn, pout + ((size_t)(c - 1) * C + rank) * NQ);
        else
            __syncthreads();
        {
            const int nc = c - back + MU_SLOTS;
            if (nc <= Lend) {
                load(nc);
                pend |= 1u << slot_of(nc);
            }
        }
    }
    if (wallR) {  // the last column's sums: its outside neighbour repeats it
        FuAccM<T, VEC> acc;
        fu_clear(acc);
        if (active) {
            const T2* ve = vxe + (ce - cs) * R;
            if (bnd) fu_sums_edge<true>(ve, ra, rb, r0, nvx, h1, acc);
            else fu_sums_edge<false>(ve, ra, rb, r0, nvx, h1, acc);
        }
        fu_reduce_sums(acc.S0, acc.Tx, acc.R1, acc.R2, acc.RA2, acc.RA3, acc.e0, acc.en, vy, vz, vp2,
                       red[(i1 - 1) & 1], posc, has0, hasn, pout + ((size_t)(i1 - 1) * C + rank) * NQ);
    }
}

// Walk of either scheme: MU = 0 upwind, MU > 0 MUSCL with at most MU v_x
// rows per thread.
template <typename T, int NVPC, int MU>
__device__ __forceinline__ void fused_walk_any(const FInst* __restrict__ insts, const FGeom& g,
                                               const int* __restrict__ cur, int b, int wk, int rank, int C, int step,
                                               int* __restrict__ status, long long wait_ns, uint32_t& phase,
                                               unsigned char* fsm)
{
    if constexpr (MU > 0) fused_walk_m<T, NVPC, MU>(insts, g, cur, b, wk, rank, C, step, status, wait_ns, phase, fsm);
    else fused_walk<T, NVPC>(insts, g, cur, b, wk, rank, C, step, status, wait_ns, phase, fsm);
}

// Resident CTAs per SM the fused kernels are built for.
template <typename T, int MU>
constexpr int fu_min_blocks()
{
    return MU > 0 ? (sizeof(T) == 4 ? 2 : 1) : (sizeof(T) == 4 ? 3 : 2);
}

// MUSCL rows per thread of the instantiated kernels (float: 4 lanes of 4
// rows, double: 2 lanes of 8 rows; 32 registers of outputs either way).
constexpr int MU_ROWS_F = 4, MU_ROWS_D = 8;

// One launch per step: CTA (rank, walk, instance).
template <typename T, int NVPC, int MU>
__global__ void __launch_bounds__(256, fu_min_blocks<T, MU>())
k_force_fused(const FInst* __restrict__ insts, FGeom g, const Active* __restrict__ act, int* __restrict__ cur,
              int step, int* __restrict__ status, long long wait_ns, int poison)
{
    const int b = blockIdx.z;
    if (b < act->begin || b >= act->end) return;
    extern __shared__ __align__(16) unsigned char fsm[];
    fu_init_mbar(fsm, poison);
    if (poison) {
        const uint32_t mb = smem_addr(&reinterpret_cast<FuShared*>(fsm)->mbar[MB_CHECK]);
        if (!mbar_wait(mb, wait_ns)) atomicCAS(status, 0, ST_TIMEOUT);
    }
    uint32_t phase = 0;
    fused_walk_any<T, NVPC, MU>(insts, g, cur, b, blockIdx.y, blockIdx.x, gridDim.x, step, status, wait_ns, phase,
                                fsm);
}

// Wait (bounded by limit_ns) until the counter reaches target; acquire
// ordering, so the writes published before the count are visible.
__device__ __forceinline__ bool wait_count(const int* p, int target, long long limit_ns)
{
    const long long t0 = gtimer();
    for (int it = 0;; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        if (v >= target) return true;
        if ((it & 15) == 15 && gtimer() - t0 > limit_ns) return false;
        __nanosleep(64);
    }
}

// All steps of a run in one persistent launch.  Work items (step, instance,
// walk, CTA row block) are taken by ticket in that order; an item of step
// k > 0 waits until every CTA of its walk and of the walks holding its two
// neighbour columns has finished step k-1 (done[walk] >= C k): their f^k and
// partials are then written, and their reads of the buffer this item
// overwrites are over.  (A MUSCL walk reads up to three columns past its
// ends; every walk then has at least three columns, so those are still the
// neighbour walks'.)  An item only waits on smaller tickets, taken by
// running CTAs, so the lowest unfinished ticket never waits.  sync: [0]
// ticket, [1 + b walks + w] done counts (zeroed before the launch).
// poison (failure-detection check): the waits of step 1 ask for a count no
// walk reaches, so they run out after wait_ns.
template <typename T, int NVPC, int MU>
__global__ void __launch_bounds__(256, fu_min_blocks<T, MU>())
k_force_fused_run(const FInst* __restrict__ insts, FGeom g, const Active* __restrict__ act, int* __restrict__ cur,
                  int nsteps, int* __restrict__ sync, int* __restrict__ status, long long wait_ns, int poison)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ int s_t;
    fu_init_mbar(fsm, 0);
    const int b0 = act->begin, nact = act->end - act->begin;
    const int nx0 = nact > 0 ? insts[b0].nx : 1;  // the instances share nx
    const int C = g.C, walks = (nx0 + g.march - 1) / g.march;
    const int per_walk_set = walks * C;
    const long long per_step = (long long)nact * per_walk_set, total = per_step * nsteps;
    int* done = sync + 1;
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(sync, 1);
        __syncthreads();
        const long long t = s_t;
        if (t >= total) break;
        const int k = (int)(t / per_step);
        const int rem = (int)(t - (long long)k * per_step);
        const int bl = rem / per_walk_set, rem2 = rem - bl * per_walk_set;
        const int wk = rem2 / C, rank = rem2 - wk * C;
        const int b = b0 + bl;
        if (k > 0 && threadIdx.x == 0) {
            const FInst& I = insts[b];
            const int nx = I.nx, S = g.march;
            bool m;
            const int wl = ghost_col(wk * S - 1, nx, I.bc, &m) / S;
            const int wr = ghost_col(min(wk * S + S, nx), nx, I.bc, &m) / S;
            const int* d = done + (size_t)bl * walks;
            const int target = C * k + (poison && k == 1 ? 1 << 28 : 0);
            bool ok = wait_count(d + wk, target, wait_ns);
            ok = ok && wait_count(d + wl, target, wait_ns);
            ok = ok && wait_count(d + wr, target, wait_ns);
            if (!ok) atomicCAS(status, 0, ST_TIMEOUT);
            asm volatile("fence.proxy.async.global;" ::: "memory");  // the bulk copies read what others wrote
        }
        __syncthreads();
        fused_walk_any<T, NVPC, MU>(insts, g, cur, b, wk, rank, C, k, status, wait_ns, phase, fsm);
        __syncthreads();  // every store of this walk issued
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + (size_t)bl * walks + wk, 1);
        }
    }
}

// Partials (the 17 column sums of the fused step) of the current state of
// the active instances: one CTA per (rank, column, instance), rows read
// straight from memory with 16-byte loads.
template <typename T, bool MUSCL>
__global__ void __launch_bounds__(256)
k_force_sums(const FInst* __restrict__ insts, FGeom g, const Active* __restrict__ act, const int* __restrict__ cur)
{
    using O = FuOps<T>;
    constexpr int VEC = 16 / (int)sizeof(T);
    const int b = blockIdx.z;
    if (b < act->begin || b >= act->end) return;
    const FInst& I = insts[b];
    const int i = blockIdx.y, rank = blockIdx.x, C = gridDim.x;
    const int nvx = g.nvx, nvp = g.nvp, nvp2 = nvp * nvp;
    const int R = g.rows, r0 = rank * R, r1 = min(r0 + R, nvx), nr = r1 - r0;
    const int Lr = nvp2 / VEC, G = g.groups;
    const int q = threadIdx.x % Lr, grp = threadIdx.x / Lr, jp = q * VEC;
    const int Rg = (nr + G - 1) / G;
    const int ra = r0 + grp * Rg, rb = min(ra + Rg, r1);
    const bool active = grp < G && ra < rb;
    __shared__ typename O::A red[8][12];
    const int bi = cur[b];
    const T* f = static_cast<const T*>(I.f[bi]) + (size_t)i * g.ncol + jp;
    const T* vt = static_cast<const T*>(I.vtab);
    T vy[VEC], vz[VEC], vp2[VEC];
#pragma unroll
    for (int l = 0; l < VEC; ++l) {
        vy[l] = active ? vt[nvx + jp + l] : T(0);
        vz[l] = active ? vt[nvx + nvp2 + jp + l] : T(0);
        vp2[l] = active ? vt[nvx + 2 * nvp2 + jp + l] : T(0);
    }
    typename O::A* dst = static_cast<typename O::A*>(I.part[bi]) + ((size_t)i * C + rank) * NQ;
    const bool posc = r0 >= I.hpos;
    if constexpr (MUSCL) {
        // the half sums of f +- s/2, s the minmod slope from the neighbour
        // columns (periodic wrap or outflow repeat)
        bool mir;
        const T* fl = static_cast<const T*>(I.f[bi]) + (size_t)ghost_col(i - 1, I.nx, I.bc, &mir) * g.ncol + jp;
        const T* fr = static_cast<const T*>(I.f[bi]) + (size_t)ghost_col(i + 1, I.nx, I.bc, &mir) * g.ncol + jp;
        FuAccM<T, VEC> acc;
        fu_clear(acc);
        if (active)
            for (int r = ra; r < rb; ++r) {
                const Pack<T, VEC> c = ldv<T, VEC>(f + (size_t)r * nvp2);
                const Pack<T, VEC> a = ldv<T, VEC>(fl + (size_t)r * nvp2);
                const Pack<T, VEC> d = ldv<T, VEC>(fr + (size_t)r * nvp2);
                T h[VEC], gv[VEC];
#pragma unroll
                for (int l = 0; l < VEC; ++l) {
                    h[l] = c.x[l];
                    gv[l] = tfma(posc ? T(0.5) : T(-0.5), mm2(c.x[l] - a.x[l], d.x[l] - c.x[l]), c.x[l]);
                }
                fu_row_m<true>(acc, h, gv, vt[r], r, nvx);
            }
        fu_reduce_sums(acc.S0, acc.Tx, acc.R1, acc.R2, acc.RA2, acc.RA3, acc.e0, acc.en, vy, vz, vp2, red, posc,
                       r0 == 0, r1 == nvx, dst);
    } else {
        FuAcc<T, VEC> acc;
        fu_clear(acc);
        if (active)
            for (int r = ra; r < rb; ++r) fu_row(acc, ldv<T, VEC>(f + (size_t)r * nvp2), vt[r], r, nvx);
        fu_reduce(acc, vy, vz, vp2, red, posc, r0 == 0, r1 == nvx, dst);
    }
}

// Conserved moments (Eq. 18) of the current state from its partials, into
// Ucur and Uout: one thread per (moment, column) of each active instance.
template <typename T>
__global__ void k_force_finalize(const FInst* __restrict__ insts, FGeom g, const Active* __restrict__ act,
                                 const int* __restrict__ cur, int nx)
{
    using O = FuOps<T>;
    const int b = act->begin + blockIdx.y;
    if (b >= act->end) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 5 * nx) return;
    const FInst& I = insts[b];
    const int k = t / nx, i = t - k * nx;
    const typename O::A s =
        part_rank_sum<T>(static_cast<const typename O::A*>(I.part[cur[b]]) + (size_t)i * g.C * NQ + k, g.C);
    double u = O::dval(s) * I.dv3;
    if (k == 4) u *= 0.5;  // energy = 1/2 sum |v|^2 f dv
    I.Ucur[k * nx + i] = u;
    if (I.Uout) I.Uout[k * nx + i] = u;
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
    if constexpr (sizeof(T) == sizeof(float)) {
        // factors within ~1e-9 before their one rounding, the prefactor
        // folded into ex (float pairs from the float64 parameters)
        const F2 u0 = f2_of(par[1]), u1 = f2_of(par[2]), u2 = f2_of(par[3]);
        const F2 i2t = f2_of(0.5 / par[4]), pref = f2_of(par[5]), one{1.0f, 0.0f};
        const F2* vp = reinterpret_cast<const F2*>(I.vpair);
        for (int q = threadIdx.x; q < nvx; q += FT) ex[q] = gauss_f2(vp[q], u0, i2t, pref);
        for (int q = threadIdx.x; q < nvp2; q += FT) {
            const int jy = q / nvp, jz = q - jy * nvp;
            eyz[q] = gauss_f2(vp[nvx + jy], u1, i2t, one) * gauss_f2(vp[nvx + jz], u2, i2t, one);
        }
    } else {
        const T ux = (T)par[1], uy = (T)par[2], uz = (T)par[3], inv2th = (T)(0.5 / par[4]), pref = (T)par[5];
        for (int q = threadIdx.x; q < nvx; q += FT) {
            T cx = vt[q] - ux;
            ex[q] = texp(-cx * cx * inv2th);
        }
        for (int q = threadIdx.x; q < nvp2; q += FT) {
            T cy = vt[nvx + q] - uy, cz = vt[nvx + nvp2 + q] - uz;
            eyz[q] = pref * texp(-cy * cy * inv2th) * texp(-cz * cz * inv2th);
        }
    }
    __syncthreads();
    T* out = static_cast<T*>(I.f[0]) + (size_t)i * g.ncol;
    const int c0 = blockIdx.x * g.rows * nvp2;
    const int c1 = (int)min((long long)c0 + (long long)g.rows * nvp2, g.ncol);
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

void* pick_step(int precision, int scheme, int vec)
{
    if (precision == 0) {
        if (vec == 2) return scheme == 0 ? reinterpret_cast<void*>(&k_force_step<double, 0, 2>)
                                         : reinterpret_cast<void*>(&k_force_step<double, 1, 2>);
        if (vec == 1) return scheme == 0 ? reinterpret_cast<void*>(&k_force_step<double, 0, 1>)
                                         : reinterpret_cast<void*>(&k_force_step<double, 1, 1>);
        return nullptr;
    }
    if (vec == 4) return scheme == 0 ? reinterpret_cast<void*>(&k_force_step<float, 0, 4>)
                                     : reinterpret_cast<void*>(&k_force_step<float, 1, 4>);
    if (vec == 1) return scheme == 0 ? reinterpret_cast<void*>(&k_force_step<float, 0, 1>)
                                     : reinterpret_cast<void*>(&k_force_step<float, 1, 1>);
    return nullptr;
}

}  // namespace

size_t force_fused_smem(int precision, int scheme, int nvp, int rows, int walk)
{
    return fu_layout(nvp, rows, walk, precision == 0 ? 8 : 4, scheme).total;
}

int force_fused_muscl_rows(int precision) { return precision == 0 ? MU_ROWS_D : MU_ROWS_F; }

bool force_fused_fits(int precision, int scheme, const FGeom& g)
{
    if (!(g.bulk && g.vec == (precision == 0 ? 2 : 4) && g.threads <= 256 && g.C <= 16)) return false;
    if (scheme == 0) return true;
    const int nr = std::min(g.rows, g.nvx), G = std::max(g.groups, 1);
    return scheme == 1 && (nr + G - 1) / G <= force_fused_muscl_rows(precision);
}

int force_partials_per_column(const FGeom& g) { return g.C * NQ; }

size_t force_step_buf_off(int precision, int nvx, int nvp)
{
    size_t es = precision == 0 ? sizeof(double) : sizeof(float);
    size_t off = sizeof(FShared) + 16 + (2 * (size_t)nvx + 2 * (size_t)nvp) * es;  // v_x nodes, ex, ey, ez
    return (off + 127) / 128 * 128;
}

size_t force_step_smem(int precision, int scheme, int nvx, int nvp, int rows)
{
    size_t es = precision == 0 ? sizeof(double) : sizeof(float);
    size_t nbuf = (size_t)(rows + 2) + (size_t)(scheme == 0 ? 1 : 3) * rows;
    return force_step_buf_off(precision, nvx, nvp) + nbuf * nvp * nvp * es;
}

// Row groups and threads for VEC values per thread: at most max_threads
// threads (at least one row of threads), a multiple of 32.
void force_step_layout(int nvp, int vec, int rows, int max_threads, int* groups, int* threads)
{
    const int Lr = nvp * nvp / vec;
    int G = std::max(1, std::min(rows, max_threads / std::max(Lr, 1)));
    *groups = G;
    *threads = (Lr * G + 31) / 32 * 32;
}

size_t force_lift_smem(int precision, int nvx, int nvp)
{
    size_t es = precision == 0 ? sizeof(double) : sizeof(float);
    return 8 * sizeof(double) + ((size_t)nvp * nvp + nvx) * es;
}

cudaError_t prepare_force_kernels(int max_smem)
{
    const int vecs[2][2] = {{1, 2}, {1, 4}};
    for (int p = 0; p < 2; ++p)
        for (int sc = 0; sc < 2; ++sc)
            for (int vi = 0; vi < 2; ++vi) {
                const void* fn = pick_step(p, sc, vecs[p][vi]);
                cudaFuncAttributes fa;
                if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
                    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         max_smem - (int)fa.sharedSizeBytes);
                cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            }
    for (const void* fn : {reinterpret_cast<const void*>(&k_force_fused<float, 0, 0>),
                           reinterpret_cast<const void*>(&k_force_fused<float, 16, 0>),
                           reinterpret_cast<const void*>(&k_force_fused_run<float, 0, 0>),
                           reinterpret_cast<const void*>(&k_force_fused_run<float, 16, 0>),
                           reinterpret_cast<const void*>(&k_force_fused<double, 0, 0>),
                           reinterpret_cast<const void*>(&k_force_fused<double, 16, 0>),
                           reinterpret_cast<const void*>(&k_force_fused_run<double, 0, 0>),
                           reinterpret_cast<const void*>(&k_force_fused_run<double, 16, 0>),
                           reinterpret_cast<const void*>(&k_force_fused<float, 0, MU_ROWS_F>),
                           reinterpret_cast<const void*>(&k_force_fused<float, 16, MU_ROWS_F>),
                           reinterpret_cast<const void*>(&k_force_fused_run<float, 0, MU_ROWS_F>),
                           reinterpret_cast<const void*>(&k_force_fused_run<float, 16, MU_ROWS_F>),
                           reinterpret_cast<const void*>(&k_force_fused<double, 0, MU_ROWS_D>),
                           reinterpret_cast<const void*>(&k_force_fused<double, 16, MU_ROWS_D>),
                           reinterpret_cast<const void*>(&k_force_fused_run<double, 0, MU_ROWS_D>),
                           reinterpret_cast<const void*>(&k_force_fused_run<double, 16, MU_ROWS_D>)}) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - (int)fa.sharedSizeBytes);
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

int force_fused_occupancy(int precision, int scheme, int threads, size_t smem, int* per_sm)
{
    int n = 0;
    const void* fn = precision == 0 ? (scheme ? reinterpret_cast<const void*>(&k_force_fused_run<double, 0, MU_ROWS_D>)
                                              : reinterpret_cast<const void*>(&k_force_fused_run<double, 0, 0>))
                                    : (scheme ? reinterpret_cast<const void*>(&k_force_fused_run<float, 0, MU_ROWS_F>)
                                              : reinterpret_cast<const void*>(&k_force_fused_run<float, 0, 0>));
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    *per_sm = n;
    return 0;
}

int force_step_occupancy(int precision, int scheme, int vec, int C, int threads, size_t smem, int* clusters)
{
    const void* fn = pick_step(precision, scheme, vec);
    if (!fn) return -1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
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
                              cudaStream_t s, long long wait_ns, int poison)
{
    if (g.march > 0) {
        dim3 grid(g.C, (nx + g.march - 1) / g.march, n_inst);
        const bool n16 = g.nvp == 16, mu = g.scheme != 0;
#define FU_STEP(T, N, M) k_force_fused<T, N, M><<<grid, g.threads, smem, s>>>(insts, g, act, cur, step, status, wait_ns, poison)
        if (precision == 0) {
            if (mu) n16 ? FU_STEP(double, 16, MU_ROWS_D) : FU_STEP(double, 0, MU_ROWS_D);
            else n16 ? FU_STEP(double, 16, 0) : FU_STEP(double, 0, 0);
        } else {
            if (mu) n16 ? FU_STEP(float, 16, MU_ROWS_F) : FU_STEP(float, 0, MU_ROWS_F);
            else n16 ? FU_STEP(float, 16, 0) : FU_STEP(float, 0, 0);
        }
#undef FU_STEP
        return cudaGetLastError();
    }
    void* fn = pick_step(precision, scheme, g.vec);
    if (!fn) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g.C, nx, n_inst);
    cfg.blockDim = dim3(g.threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = g.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void* args[] = {(void*)&insts, (void*)&g,      (void*)&act,     (void*)&cur,   (void*)&step,
                    (void*)&last,  (void*)&status, (void*)&wait_ns, (void*)&poison};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_force_fused_run(int precision, const FInst* insts, const FGeom& g, int n_inst, const Active* act,
                                   int* cur, int nsteps, int* sync, int sync_words, int* status, size_t smem,
                                   cudaStream_t s, int ctas, long long wait_ns, int poison)
{
    cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(int) * (size_t)sync_words, s);
    if (e != cudaSuccess || nsteps <= 0) return e;
    const bool n16 = g.nvp == 16, mu = g.scheme != 0;
#define FU_RUN(T, N, M) \
    k_force_fused_run<T, N, M><<<ctas, g.threads, smem, s>>>(insts, g, act, cur, nsteps, sync, status, wait_ns, poison)
    if (precision == 0) {
        if (mu) n16 ? FU_RUN(double, 16, MU_ROWS_D) : FU_RUN(double, 0, MU_ROWS_D);
        else n16 ? FU_RUN(double, 16, 0) : FU_RUN(double, 0, 0);
    } else {
        if (mu) n16 ? FU_RUN(float, 16, MU_ROWS_F) : FU_RUN(float, 0, MU_ROWS_F);
        else n16 ? FU_RUN(float, 16, 0) : FU_RUN(float, 0, 0);
    }
#undef FU_RUN
    return cudaGetLastError();
}

cudaError_t launch_force_sums(int precision, const FInst* insts, const FGeom& g, int nx, int n_inst,
                              const Active* act, const int* cur, cudaStream_t s)
{
    const dim3 grid(g.C, nx, n_inst);
    if (precision == 0) {
        if (g.scheme) k_force_sums<double, true><<<grid, g.threads, 0, s>>>(insts, g, act, cur);
        else k_force_sums<double, false><<<grid, g.threads, 0, s>>>(insts, g, act, cur);
    } else {
        if (g.scheme) k_force_sums<float, true><<<grid, g.threads, 0, s>>>(insts, g, act, cur);
        else k_force_sums<float, false><<<grid, g.threads, 0, s>>>(insts, g, act, cur);
    }
    return cudaGetLastError();
}

cudaError_t launch_force_finalize(int precision, const FInst* insts, const FGeom& g, int nx, int n_inst,
                                  const Active* act, const int* cur, cudaStream_t s)
{
    dim3 grid((5 * nx + 127) / 128, n_inst);
    if (precision == 0) k_force_finalize<double><<<grid, 128, 0, s>>>(insts, g, act, cur, nx);
    else k_force_finalize<float><<<grid, 128, 0, s>>>(insts, g, act, cur, nx);
    return cudaGetLastError();
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
