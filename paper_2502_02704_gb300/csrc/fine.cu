// Fine kinetic propagator of the kinetic-fluid parareal method (Laidin & Rey,
// arXiv 2502.02704): one fused pass per fine step of the IMEX scheme of
// Eqs. (11)-(13) -- x-transport (upwind, or minmod-limited MUSCL slopes as the
// flux limiter of Sec. 3.1), the velocity moments of the transported f (Eq. 18,
// explicit by conservation), the local Maxwellian (Eq. 4) and the implicit BGK
// relaxation f^{n+1} = (eps f* + dt M)/(eps + dt) (Eq. 7 with tau = 1).
//
// Storage form.  The state after a step is kept as the transported values f*
// (array g) plus, per x cell, the separable factors of b*M:
//     f^{n+1}_ij = a g_ij + T0_i[jx] T1_i[jy] T2_i[jz],  a = eps/(eps+dt), b = dt/(eps+dt)
// with T0 = b rho (2 pi theta)^{-3/2} exp(-(v_x-u_x)^2/(2 theta)), T1, T2 the
// y/z Gaussians.  This is the same f^{n+1} as the paper's scheme; it is
// reconstructed on the fly where the next step reads it, so each step reads g
// once and writes g once and the all-velocity dependency of the moments is
// resolved at the step boundary instead of inside the pass.  The lifting of
// Eq. (17) is the same form with a = 0 (f = M), so a slice's first step reads
// no f at all; the projection of Eq. (18) of the final state is a P(g) + P(M),
// with P(M) from 1-D sums of the factor tables.
//
// Work decomposition.  A work item is (step, instance, x tile of tx cells,
// v chunk of 1024 velocities); within a step, instances in order, tiles in
// zigzag order, chunks innermost.  Each thread owns 4 consecutive v_z nodes (one
// 16-byte vector in float32) and marches along x with a register window of
// 2H+1 cells (H = 1 upwind, 2 MUSCL), so every cell of its strip is loaded
// once (halo cells of the tile twice).  Per x cell the 5 moment sums
// (rho, rho u, |v|^2 f) are reduced across the warp by shuffles, across warps
// in float64 shared memory, and written as a per-chunk partial; the last chunk
// CTA of a tile to finish (arrival counter) sums the partials in a fixed order
// and writes the factor tables of the next state.  One persistent launch runs
// all steps of all active instances: CTAs take tickets in step order and an
// item of step s waits only until the tiles its stencil touches have finished
// step s-1 (bounded spin on a flag; a time-out aborts the launch with a status
// code).  Tickets are taken only by running CTAs and an item waits only on
// smaller tickets, so the lowest unfinished ticket never waits.
#include <cooperative_groups.h>
#include <math.h>

#include "maxwell_tab.h"
#include "pr_kernels.h"

namespace cg = cooperative_groups;

namespace prk {

namespace {

constexpr double PI = 3.14159265358979323846;

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_status(const int* p) { return *(volatile const int*)p; }

// ---- 4-wide vector access (16 bytes in float32, 2 x 16 bytes in float64) ----
__device__ __forceinline__ void st4(float* p, const float (&v)[4])
{
    __stcg(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4])
{
    __stcg(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
    __stcg(reinterpret_cast<double2*>(p + 2), make_double2(v[2], v[3]));
}
__device__ __forceinline__ void lds4(const float* p, float (&o)[4])
{
    float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void lds4(const double* p, double (&o)[4])
{
    double2 a = *reinterpret_cast<const double2*>(p);
    double2 b = *reinterpret_cast<const double2*>(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

__device__ __forceinline__ float exp_neg(float, double arg) { return expf(-(float)arg); }
__device__ __forceinline__ double exp_neg(double, double arg) { return exp(-arg); }

// Boundary mapping of an x cell index c (ghosts -2..nx+1) to a stored cell and
// whether v_x is reversed (specular wall).  Periodic wraps, outflow copies the
// boundary cell (zero gradient), reflecting mirrors the cell.
__device__ __forceinline__ int map_col(int c, int nx, int bc, bool& flip)
{
    flip = false;
    if (c >= 0 && c < nx) return c;
    if (bc == 0) return ((c % nx) + nx) % nx;
    if (bc == 1) return c < 0 ? 0 : nx - 1;
    flip = true;
    return c < 0 ? -1 - c : 2 * nx - 1 - c;
}

template <typename T>
__device__ __forceinline__ T minmod(T a, T b)
{
    if (a * b <= T(0)) return T(0);
    return fabs(a) < fabs(b) ? a : b;
}

// minmod without branches: the argument of smaller magnitude when both have
// the same sign, else 0 -- b clamped to the interval between 0 and a (four
// min/max operations, no addition).
__device__ __forceinline__ float minmod2(float a, float b)
{
    return fminf(fmaxf(b, fminf(a, 0.f)), fmaxf(a, 0.f));
}
// float64: the same selection on the IEEE bit patterns with integer
// operations only (sign bits equal -> the smaller magnitude, else 0), which
// keeps the limiter off this GPU's reduced-rate FP64 pipe.
__device__ __forceinline__ double minmod2(double a, double b)
{
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    const long long ma = ia & 0x7fffffffffffffffLL, mb = ib & 0x7fffffffffffffffLL;
    const long long r = ma < mb ? ia : ib;
    return (ia ^ ib) >= 0 ? __longlong_as_double(r) : 0.0;
}
// Packed float32 pairs: the limiter per lane, and a - b as one fused
// multiply-add b (-1) + a (exact product, one rounding: the value of the
// scalar subtraction).
__device__ __forceinline__ float2 minmod2(float2 a, float2 b)
{
    return make_float2(minmod2(a.x, b.x), minmod2(a.y, b.y));
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

// Upwind interface value at the face between f0 and f1 (neighbours fm, f2):
// from the left (f0 side) when v_x > 0, from the right otherwise (Eq. 13 with
// the upwind sign); MUSCL adds half the minmod slope of the upwind cell.
template <typename T, int H>
__device__ __forceinline__ T face_value(T fm, T f0, T f1, T f2, bool pos)
{
    if (H == 1) return pos ? f0 : f1;
    T d0 = f0 - fm, d1 = f1 - f0, d2 = f2 - f1;
    T ua = pos ? d0 : d1, ub = pos ? d1 : d2;
    T base = pos ? f0 : f1;
    T sg = pos ? T(0.5) : T(-0.5);
    return base + sg * minmod(ua, ub);
}

// Shared-memory layout helpers.
__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Factor tables of the Maxwellians of ncols x cells.  float64: par[i*8 + 0..4]
// = (u_x, u_y, u_z, theta, weight*rho*(2 pi theta)^{-3/2}), the tables
// evaluated in float64.  float32: tp[i] holds the same parameters as float
// pairs in grid units (tabpar_from_sums) and each entry is evaluated to about
// 1e-9 before its one rounding (tab_entry, float32 pipes only: this GPU's
// FP64 pipe is ~1/64 of their rate).  Grid coordinates k_j = j + 1/2 - nv/2
// are exact, so the tables keep the grid's mirror symmetry.
template <typename T, int NT>
__device__ void write_tables(const Inst& I, int c0, int ncols, const double* par, const TabPar* tp, T* tout, T* tb)
{
    const int tid = threadIdx.x;
    const int nv = I.nv, tw = 3 * nv;
    if (sizeof(T) == 4) {
        for (int idx = tid; idx < ncols * tw; idx += NT) {
            int i = idx / tw, rem = idx - i * tw, d = rem / nv, j = rem - d * nv;
            const float val = tab_entry(tp[i], d, node_k(j, nv));
            tb[idx] = (T)val;
            tout[(size_t)(c0 + i) * tw + rem] = (T)val;
        }
    } else {
        for (int idx = tid; idx < ncols * tw; idx += NT) {
            int i = idx / tw, rem = idx - i * tw, d = rem / nv, j = rem - d * nv;
            double vj = -I.L + (j + 0.5) * I.dv;
            double u = par[i * 8 + d], th = par[i * 8 + 3];
            double dvu = vj - u;
            T val = exp_neg(T(0), dvu * dvu / (2.0 * th));
            if (d == 0) val = (T)(par[i * 8 + 4] * (double)val);
            tb[idx] = val;
            tout[(size_t)(c0 + i) * tw + rem] = val;
        }
    }
}

// Conserved moments (Eq. 18) of f = wg g + M_tab for ncols x cells, from the
// g sums in grid units mom[i*5 + 0..4] = (g, k_x g, k_y g, k_z g, |k|^2 g),
// v = k dv (no dv^3), and the 1-D sums of the tables tb (separable M):
// written to Ucur (and Uout).
template <typename T, int NT>
__device__ void project_columns(const Inst& I, int c0, int ncols, const double* mom, double wg, const T* tb,
                                double* Uout)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nv = I.nv;
    for (int i = warp; i < ncols; i += NT / 32) {
        double gs[3][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) gs[d][0] = gs[d][1] = gs[d][2] = 0.0;
        for (int j = lane; j < nv; j += 32) {
            double vj = -I.L + (j + 0.5) * I.dv;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                double t = (double)tb[(i * 3 + d) * nv + j];
                gs[d][0] += t;
                gs[d][1] += vj * t;
                gs[d][2] += vj * vj * t;
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int o = 16; o; o >>= 1) gs[d][m] += __shfl_xor_sync(0xffffffffu, gs[d][m], o);
        if (lane == 0) {
            const double dv3 = I.dv3;
            double x0 = gs[0][0], y0 = gs[1][0], z0 = gs[2][0];
            double V[5];
            V[0] = dv3 * x0 * y0 * z0;
            V[1] = dv3 * gs[0][1] * y0 * z0;
            V[2] = dv3 * x0 * gs[1][1] * z0;
            V[3] = dv3 * x0 * y0 * gs[2][1];
            V[4] = 0.5 * dv3 * (gs[0][2] * y0 * z0 + x0 * gs[1][2] * z0 + x0 * y0 * gs[2][2]);
            if (wg != 0.0) {
                const double w1 = wg * dv3 * I.dv;
                V[0] += wg * mom[i * 5 + 0] * dv3;
                V[1] += w1 * mom[i * 5 + 1];
                V[2] += w1 * mom[i * 5 + 2];
                V[3] += w1 * mom[i * 5 + 3];
                V[4] += 0.5 * w1 * I.dv * mom[i * 5 + 4];
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                I.Ucur[(size_t)q * I.nx + c0 + i] = V[q];
                if (Uout) Uout[(size_t)q * I.nx + c0 + i] = V[q];
            }
        }
    }
}

// Maxwellian parameters from moment sums in grid units s = (f, k f, |k|^2 f
// summed, v = k dv, no dv^3): u = dv s_{1..3}/s_0, theta = dv^2 (s_4/s_0 -
// |s_{1..3}/s_0|^2)/3 (= Eq. 18's 3 rho theta), rho = s_0 dv^3.
__device__ __forceinline__ void prim_from_sums(const double* s, double dv, double dv3, double weight, double* par,
                                               int* status)
{
    double rho = s[0] * dv3;
    double is0 = 1.0 / s[0];
    double kx = s[1] * is0, ky = s[2] * is0, kz = s[3] * is0;
    double th = dv * dv * (s[4] * is0 - (kx * kx + ky * ky + kz * kz)) / 3.0;
    if (!(rho > 0.0) || !(th > 0.0)) atomicCAS(status, 0, ST_NONPHYS);
    double tp = 2.0 * PI * th;
    par[0] = kx * dv;
    par[1] = ky * dv;
    par[2] = kz * dv;
    par[3] = th;
    par[4] = weight * rho / (tp * sqrt(tp));
}

// The same Maxwellian as float pairs in grid units, for the float32 tables:
// u_d/dv = s_d/s_0, tau = s_4/s_0 - |u/dv|^2 = 3 theta/dv^2, so the exponent
// (k_j - u_d/dv)^2 dv^2/(2 theta) has w = 3/(2 tau) and the prefactor
// weight rho (2 pi theta)^{-3/2} = weight s_0 (2 pi tau/3)^{-3/2}: dv drops
// out.  Parameters in float64 (Eq. 18's moments and the Maxwellian of Eq. 4),
// then split into pairs.
__device__ __forceinline__ TabPar tabpar_from_sums(const double* s, double weight, int* status)
{
    TabPar P;
    // rho, u, theta (as rho dv^3-free sums, u/dv and tau) in float64
    const double is0 = 1.0 / s[0];
    const double k[3] = {s[1] * is0, s[2] * is0, s[3] * is0};
    const double tau = s[4] * is0 - (k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    if (!(s[0] > 0.0) || !(tau > 0.0)) atomicCAS(status, 0, ST_NONPHYS);
#pragma unroll
    for (int d = 0; d < 3; ++d) split_pair(k[d], P.uh[d], P.ul[d]);
    // the table weights from them in pair arithmetic (no float64 division or
    // root on the step's critical path)
    const F2 t2 = f2_of(tau);
    const F2 w = f2_mul(F2{1.5f, 0.0f}, f2_rcp(t2));
    const F2 tq = f2_mul(f2_of(2.0 * PI / 3.0), t2);
    const F2 pref = f2_mul(f2_of(weight * s[0]), f2_rcp(f2_mul(tq, f2_sqrt(tq))));
    P.wh = w.h, P.wl = w.l;
    P.ph = pref.h, P.pl = pref.l;
    return P;
}

// Grid-unit sums (f, k f, |k|^2 f without dv^3) of the conserved state V
// (rho, rho u, E) of cell c (the lift source).
__device__ __forceinline__ void sums_from_state(const double* V, int nx, int c, double dv, double dv3, double* s)
{
    const double id3 = 1.0 / dv3, id4 = id3 / dv;
    s[0] = V[c] * id3;
    s[1] = V[nx + c] * id4;
    s[2] = V[2 * nx + c] * id4;
    s[3] = V[3 * nx + c] * id4;
    s[4] = 2.0 * V[4 * nx + c] * (id4 / dv);
}

// Last CTA of a tile: sum the chunk partials of step s (fixed order, one
// thread per (x cell, moment)), build the Maxwellian of the new state and its
// tables; at the last step of the launch also the projected moments; release.
template <typename T, int NT>
__device__ void finalize_tile(const Inst& I, int s, int nsteps, int xt, int c0, int ncols, int pout,
                              unsigned char* smem, int* status)
{
    const int tid = threadIdx.x;
    double* mom = reinterpret_cast<double*>(smem);  // [MAX_TX][5]
    double* par = mom + MAX_TX * 5;                  // [MAX_TX][8]
    TabPar* tp = reinterpret_cast<TabPar*>(par);     // float32: the pairs in place of par
    T* tb = reinterpret_cast<T*>(par + MAX_TX * 8);   // [MAX_TX][3][nv]
    const int n_vc = I.n_vc;
    for (int idx = tid; idx < ncols * 5; idx += NT) {
        const int i = idx / 5, q = idx - i * 5;
        const double* p = I.part + (size_t)(c0 + i) * n_vc * 5 + q;
        double acc = 0.0;
        for (int v = 0; v < n_vc; ++v) acc += __ldcg(p + v * 5);
        mom[idx] = acc;
    }
    __syncthreads();
    if (sizeof(T) == sizeof(double) && I.trace_m)  // the recorded step's moment sums
        for (int idx = tid; idx < ncols * 5; idx += NT) I.trace_m[((size_t)(s - 1) * I.nx + c0) * 5 + idx] = mom[idx];
    for (int i = tid; i < ncols; i += NT) {
        if (sizeof(T) == 4) tp[i] = tabpar_from_sums(mom + i * 5, I.b, status);
        else prim_from_sums(mom + i * 5, I.dv, I.dv3, I.b, par + i * 8, status);
    }
    __syncthreads();
    T* tout = reinterpret_cast<T*>(I.tab[pout]);
    write_tables<T, NT>(I, c0, ncols, par, tp, tout, tb);
    if (s == nsteps) {
        __syncthreads();
        project_columns<T, NT>(I, c0, ncols, mom, I.a, tb, I.Uout);
    }
    // release the tile: the barrier orders the CTA's table writes before
    // thread 0's release store of the completion flag
    __syncthreads();
    if (tid == 0) {
        I.arrive[xt] = 0u;
        st_release(I.done + xt, (unsigned)s);
    }
}

// Wait until every tile in deps[xt] has finalised step `target`.  Called by
// warp 0: lane k spins on dependency k, so the flags are polled in parallel.
__device__ bool wait_tiles(const Inst& I, int xt, unsigned target, int* status, int lane,
                           unsigned long long limit_ns)
{
    bool ok = true;
    if (lane < MAXDEP) {
        const int tile = I.deps[xt * MAXDEP + lane];
        if (tile >= 0) {
            const unsigned* p = I.done + tile;
            const unsigned long long t0 = gtimer();
            unsigned ns = 32;
            while (ld_acquire(p) < target) {
                if (ld_status(status) != 0) {
                    ok = false;
                    break;
                }
                if (gtimer() - t0 > limit_ns) {
                    atomicCAS(status, 0, ST_TIMEOUT);
                    ok = false;
                    break;
                }
                __nanosleep(ns);
                if (ns < 128) ns <<= 1;
            }
        }
    }
    return __all_sync(0xffffffffu, ok);
}

// Per-thread asynchronous prefetch of its own 16-byte pieces of g into a ring of
// RING column slots in shared memory (cp.async, L2 only).  Each thread reads back
// only what it copied, so no barrier is needed; one commit group per column.
template <typename T>
struct Ring {
    static constexpr int SLOTS = sizeof(T) == 4 ? 8 : 4;
};

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Sum five per-lane values over the warp with 8 shuffles (transposed butterfly):
// afterwards lanes 0-3 hold the total of r0, 4-7 of r1, 8-15 of r2, 16-23 of r3,
// 24-31 of r4.  Fixed order, deterministic.
template <typename T>
__device__ __forceinline__ T warp_sum5(const T (&r)[5], int lane)
{
    const unsigned F = 0xffffffffu;
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    // level 16: lanes 0-15 keep (r0, r1, r2), lanes 16-31 keep (r3, r4)
    T y1 = __shfl_xor_sync(F, h16 ? r[0] : r[3], 16);
    T y2 = __shfl_xor_sync(F, h16 ? r[1] : r[4], 16);
    T y3 = __shfl_xor_sync(F, h16 ? r[2] : T(0), 16);
    T a = (h16 ? r[3] : r[0]) + y1;
    T b = (h16 ? r[4] : r[1]) + y2;
    T c = h16 ? T(0) : r[2] + y3;
    // level 8: 0-7 keep (a, b) = (r0, r1); 8-15 keep c = r2; 16-23 keep a = r3; 24-31 keep b = r4
    T x4 = !h16 ? (h8 ? a : c) : (h8 ? a : b);
    T y4 = __shfl_xor_sync(F, x4, 8);
    T y5 = __shfl_xor_sync(F, b, 8);
    T p, q = T(0);
    if (!h16) {
        if (!h8) { p = a + y4; q = b + y5; }
        else p = c + y4;
    } else {
        p = (h8 ? b : a) + y4;
    }
    // level 4: lanes 0-3 keep p (r0), 4-7 keep q (r1); the others keep p
    const bool grp01 = !h16 && !h8;
    T x6 = grp01 ? (h4 ? p : q) : p;
    T y6 = __shfl_xor_sync(F, x6, 4);
    p = (grp01 && h4) ? q + y6 : p + y6;
    p += __shfl_xor_sync(F, p, 2);
    p += __shfl_xor_sync(F, p, 1);
    return p;
}

// One work item: transport + moments for x cells [c0, c1) and one v chunk of
// CHUNK velocities, V consecutive v_z nodes per thread (V = 4 or 8, same row).
template <typename T, int H, int V>
__device__ void fine_item(const Inst& I, const InstState& S, int s, int nsteps, int xt, int vc,
                          unsigned char* smem, int* status, unsigned long long* ticket, long long* s_next)
{
    constexpr int NT = CHUNK / V, NW = NT / 32, NV4 = V / 4;
    constexpr int RING = Ring<T>::SLOTS;
    constexpr int CPY = V * (int)sizeof(T) / 16;  // 16-byte copies per thread and column
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = I.nx, nv = I.nv, ldv = I.ldv, bc = I.bc, tw = 3 * nv;
    const int c0 = xt * I.tx, c1 = min(nx, c0 + I.tx), ncols = c1 - c0;
    const int ne = ncols + 2 * H;
    // odd tiles march right to left (the mirror image: v_x and the upwind side
    // reversed, the same f* bit for bit), so two neighbouring tiles reach
    // their shared halo columns together and the second read finds them in L2
    const bool rev = (xt & 1) != 0;
    const int cbase = rev ? c1 - 1 + H : c0 - H, cdir = rev ? -1 : 1;
    const int pin = (S.cur + s - 1) & 1, pout = (S.cur + s) & 1;
    const T* __restrict__ gin = reinterpret_cast<const T*>(I.g[pin]);
    T* __restrict__ gout = reinterpret_cast<T*>(I.g[pout]);
    const T* __restrict__ tin = reinterpret_cast<const T*>(I.tab[pin]);
    const double wgd = (s == 1) ? S.a0 : I.a;
    const T wg = (T)wgd;
    const bool use_g = wgd != 0.0;

    T* ring = reinterpret_cast<T*>(smem);  // [RING][NT][V]
    T* stab = ring + RING * NT * V;         // [ne][3][nv]
    T* red = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(stab) +
                                  align16((size_t)ne * tw * sizeof(T)));  // [tx][NW][5] warp totals

    const int v0 = vc * CHUNK + tid * V;
    const bool act = v0 < I.nv3;
    int jx = 0, jy = 0, jz = 0;
    if (act) {
        jz = v0 % nv;
        int q = v0 / nv;
        jy = q % nv;
        jx = q / nv;
    }
    const int jxf = nv - 1 - jx;
    const int v0f = (jxf * nv + jy) * nv + jz;
    const bool load = use_g && act;
    T* const myslot = ring + tid * V;

    // prefetch of extended column e of g into ring slot e % RING (one commit group each)
    auto issue = [&](int e) {
        if (load && e < ne) {
            bool fl;
            int cc = map_col(cbase + cdir * e, nx, bc, fl);
            const T* src = gin + (size_t)cc * ldv + (fl ? v0f : v0);
            T* dst = myslot + (e % RING) * (NT * V);
#pragma unroll
            for (int k = 0; k < CPY; ++k) cp_async16(dst + k * (16 / sizeof(T)), src + k * (16 / sizeof(T)));
        }
        cp_async_commit();
    };
    // factor tables of the ne extended columns: 16-byte asynchronous copies
    // (first commit group), overlapped with the prefetch of g below
    {
        constexpr int PER = 16 / (int)sizeof(T);
        const int rowv = tw / PER;
        for (int idx = tid; idx < ne * rowv; idx += NT) {
            int e = idx / rowv, k = idx - e * rowv;
            bool fl;
            int cc = map_col(cbase + cdir * e, nx, bc, fl);
            cp_async16(stab + e * tw + k * PER, tin + (size_t)cc * tw + k * PER);
        }
        cp_async_commit();
    }
#pragma unroll
    for (int e = 0; e < RING; ++e) issue(e);
    cp_async_wait<RING>();
    __syncthreads();

    const double vxd = -I.L + (jx + 0.5) * I.dv;
    const bool pos = (vxd > 0.0) != rev;
    const T cour = rev ? -(T)(I.nu * vxd) : (T)(I.nu * vxd);
    // moment weights in grid units, v = k dv with k = j + 1/2 - nv/2 (half
    // integers, exact in float32, so no weight carries a rounding error into
    // the sums): node q of this thread has k_z = kz0 + q, so sum k_z f =
    // kz0 s0 + t1 and sum k_z^2 f = kz0^2 s0 + 2 kz0 t1 + t2 with t1 = sum q f_q,
    // t2 = sum q^2 f_q; dv and dv^2 are applied in float64 after the reduction
    const T kx = T(0.5) * T(2 * jx + 1 - nv), ky = T(0.5) * T(2 * jy + 1 - nv);
    const T kz0 = T(0.5) * T(2 * jz + 1 - nv), kz1 = T(2 * jz + 1 - nv);
    const T kk0 = kx * kx + ky * ky + kz0 * kz0;

    // value of the current state at extended column e for this thread's V velocities
    auto recon = [&](int e, T (&o)[V]) {
        bool fl;
        map_col(cbase + cdir * e, nx, bc, fl);
        int jxx = fl ? jxf : jx;
        const T* tb = stab + e * tw;
        T txy = tb[jxx] * tb[nv + jy];
        T tz[V];
#pragma unroll
        for (int k = 0; k < NV4; ++k) lds4(tb + 2 * nv + jz + 4 * k, *reinterpret_cast<T(*)[4]>(tz + 4 * k));
        cp_async_wait<RING - 1>();
        if (load) {
            T gv[V];
            const T* sl = myslot + (e % RING) * (NT * V);
#pragma unroll
            for (int k = 0; k < NV4; ++k) lds4(sl + 4 * k, *reinterpret_cast<T(*)[4]>(gv + 4 * k));
#pragma unroll
            for (int q = 0; q < V; ++q) o[q] = wg * gv[q] + txy * tz[q];
        } else {
#pragma unroll
            for (int q = 0; q < V; ++q) o[q] = txy * tz[q];
        }
        issue(e + RING);
    };

    const int qsel = lane < 4 ? 0 : lane < 8 ? 1 : lane < 16 ? 2 : lane < 24 ? 3 : 4;
    const bool writer = lane == 0 || lane == 4 || lane == 8 || lane == 16 || lane == 24;
    T* outp = gout + (size_t)(rev ? c1 - 1 : c0) * ldv + v0;
    const long long ostep = rev ? -(long long)ldv : (long long)ldv;
    if constexpr (sizeof(T) == sizeof(float)) {
        // float32: the arithmetic on pairs of v_z nodes with the packed
        // two-lane instructions (add, multiply, fused multiply-add, IEEE
        // round-to-nearest in each lane): half the issue slots of scalar code
        constexpr int V2 = V / 2;
        const float2 wg2 = make_float2(wg, wg), h2 = make_float2(0.5f, 0.5f), mh2 = make_float2(-0.5f, -0.5f);
        const float2 mc2 = make_float2(-cour, -cour);
        auto recon2 = [&](int e, float2 (&o)[V2]) {
            bool fl;
            map_col(cbase + cdir * e, nx, bc, fl);
            const int jxx = fl ? jxf : jx;
            const float* tb = stab + e * tw;
            const float txy = tb[jxx] * tb[nv + jy];
            const float2 t2 = make_float2(txy, txy);
            float2 tz[V2];
#pragma unroll
            for (int k = 0; k < NV4; ++k) {
                const float4 z = *reinterpret_cast<const float4*>(tb + 2 * nv + jz + 4 * k);
                tz[2 * k] = make_float2(z.x, z.y);
                tz[2 * k + 1] = make_float2(z.z, z.w);
            }
            cp_async_wait<RING - 1>();
            if (load) {
                const float* sl = myslot + (e % RING) * (NT * V);
#pragma unroll
                for (int k = 0; k < NV4; ++k) {
                    const float4 gv = *reinterpret_cast<const float4*>(sl + 4 * k);
                    o[2 * k] = __ffma2_rn(wg2, make_float2(gv.x, gv.y), __fmul2_rn(t2, tz[2 * k]));
                    o[2 * k + 1] = __ffma2_rn(wg2, make_float2(gv.z, gv.w), __fmul2_rn(t2, tz[2 * k + 1]));
                }
            } else {
#pragma unroll
                for (int k = 0; k < V2; ++k) o[k] = __fmul2_rn(t2, tz[k]);
            }
            issue(e + RING);
        };
        // Output cell i: fs = f_i - cour (face_{i+1/2} - face_{i-1/2}), sp =
        // face_{i-1/2}.  Upwind from the left (pos): face_{i+1/2} = f_i (+ half
        // the minmod of f_i - f_{i-1} and f_{i+1} - f_i); from the right:
        // f_{i+1} (- half the minmod of f_{i+1} - f_i and f_{i+2} - f_{i+1}).
        // A thread's side is fixed, so each side carries only the state it
        // needs: fc = f_i, sp, and fb = f_i - f_{i-1} (pos, MUSCL) or f_{i+1}.
        float2 fc[V2], fb[V2], sp[V2];
        if (H == 2) {
            float2 f0[V2], f1[V2];
            recon2(0, f0);
            recon2(1, f1);
            recon2(2, fc);
            if (pos) {
#pragma unroll
                for (int k = 0; k < V2; ++k) {
                    fb[k] = sub2(fc[k], f1[k]);
                    sp[k] = __ffma2_rn(h2, minmod2(sub2(f1[k], f0[k]), fb[k]), f1[k]);
                }
            } else {
                recon2(3, fb);
#pragma unroll
                for (int k = 0; k < V2; ++k)
                    sp[k] = __ffma2_rn(mh2, minmod2(sub2(fc[k], f1[k]), sub2(fb[k], fc[k])), fc[k]);
            }
        } else {
            float2 f0[V2];
            recon2(0, f0);
            recon2(1, fc);
#pragma unroll
            for (int k = 0; k < V2; ++k) sp[k] = pos ? f0[k] : fc[k];
        }
        // extended column read for output cell i: f_{i+1} (pos or upwind) or f_{i+2}
        const int E0 = H == 2 ? (pos ? 3 : 4) : 2;
        for (int i = 0; i < ncols; ++i, outp += ostep) {
            const int li = rev ? ncols - 1 - i : i;  // the column within the tile
            float2 fs[V2], fx[V2];
            recon2(i + E0, fx);
            if (H == 2) {
                if (pos) {
#pragma unroll
                    for (int k = 0; k < V2; ++k) {
                        const float2 dp = sub2(fx[k], fc[k]);
                        const float2 face = __ffma2_rn(h2, minmod2(fb[k], dp), fc[k]);
                        fs[k] = __ffma2_rn(mc2, sub2(face, sp[k]), fc[k]);
                        sp[k] = face;
                        fb[k] = dp;
                        fc[k] = fx[k];
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < V2; ++k) {
                        const float2 face = __ffma2_rn(mh2, minmod2(sub2(fb[k], fc[k]), sub2(fx[k], fb[k])), fb[k]);
                        fs[k] = __ffma2_rn(mc2, sub2(face, sp[k]), fc[k]);
                        sp[k] = face;
                        fc[k] = fb[k];
                        fb[k] = fx[k];
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < V2; ++k) {
                    const float2 face = pos ? fc[k] : fx[k];
                    fs[k] = __ffma2_rn(mc2, sub2(face, sp[k]), fc[k]);
                    sp[k] = face;
                    fc[k] = fx[k];
                }
            }
            T r[5];
            if (act) {
#pragma unroll
                for (int k = 0; k < NV4; ++k)
                    __stcg(reinterpret_cast<float4*>(outp + 4 * k),
                           make_float4(fs[2 * k].x, fs[2 * k].y, fs[2 * k + 1].x, fs[2 * k + 1].y));
                // node q of pair k is 2k + lane: sum f, sum q f, sum q^2 f in
                // pairs, the two lanes added last; explicit fused operations
                // so that every build rounds the column sums alike
                float2 a0 = fs[0];
                float2 a1 = __fmul2_rn(make_float2(0.0f, 1.0f), fs[0]);
                float2 a2 = a1;
#pragma unroll
                for (int k = 1; k < V2; ++k) {
                    const float q0 = (float)(2 * k), q1 = (float)(2 * k + 1);
                    a0 = __fadd2_rn(a0, fs[k]);
                    a1 = __ffma2_rn(make_float2(q0, q1), fs[k], a1);
                    a2 = __ffma2_rn(make_float2(q0 * q0, q1 * q1), fs[k], a2);
                }
                const float s0 = a0.x + a0.y, t1 = a1.x + a1.y, t2 = a2.x + a2.y;
                r[0] = s0;
                r[1] = kx * s0;
                r[2] = ky * s0;
                r[3] = fmaf(kz0, s0, t1);
                r[4] = fmaf(kk0, s0, fmaf(kz1, t1, t2));
            } else {
#pragma unroll
                for (int q = 0; q < 5; ++q) r[q] = T(0);
            }
            T tot = warp_sum5(r, lane);
            if (writer) red[(li * NW + warp) * 5 + qsel] = tot;
        }
    } else {
        // March along x.  State before output cell i: fc = f_i, fn = f_{i+1},
        // dm = f_i - f_{i-1}, dp = f_{i+1} - f_i (MUSCL), sp = face value at i-1/2.
        T fc[V], fn[V], dm[V], dp[V], sp[V];
        if (H == 2) {
            T f0[V], f1[V];
            recon(0, f0);
            recon(1, f1);
            recon(2, fc);
            recon(3, fn);
    #pragma unroll
            for (int q = 0; q < V; ++q) {
                T d0 = f1[q] - f0[q];
                dm[q] = fc[q] - f1[q];
                dp[q] = fn[q] - fc[q];
                sp[q] = pos ? f1[q] + T(0.5) * minmod2(d0, dm[q]) : fc[q] - T(0.5) * minmod2(dm[q], dp[q]);
            }
        } else {
            T f0[V];
            recon(0, f0);
            recon(1, fc);
    #pragma unroll
            for (int q = 0; q < V; ++q) sp[q] = pos ? f0[q] : fc[q];
        }

        // float64 steps two x cells per loop body (the window rotation becomes
        // register renaming: +2 % measured); float32 one (unrolling spills there)
        constexpr int XUNROLL = sizeof(T) == 8 ? 2 : 1;
    #pragma unroll XUNROLL
        for (int i = 0; i < ncols; ++i, outp += ostep) {
            const int li = rev ? ncols - 1 - i : i;  // the column within the tile
            T fs[V];
            if (H == 2) {
                T fnn[V];
                recon(i + 4, fnn);
                if (pos) {
    #pragma unroll
                    for (int q = 0; q < V; ++q) {
                        T dpp = fnn[q] - fn[q];
                        T face = fc[q] + T(0.5) * minmod2(dm[q], dp[q]);
                        fs[q] = fc[q] - cour * (face - sp[q]);
                        sp[q] = face;
                        fc[q] = fn[q];
                        fn[q] = fnn[q];
                        dm[q] = dp[q];
                        dp[q] = dpp;
                    }
                } else {
    #pragma unroll
                    for (int q = 0; q < V; ++q) {
                        T dpp = fnn[q] - fn[q];
                        T face = fn[q] - T(0.5) * minmod2(dp[q], dpp);
                        fs[q] = fc[q] - cour * (face - sp[q]);
                        sp[q] = face;
                        fc[q] = fn[q];
                        fn[q] = fnn[q];
                        dm[q] = dp[q];
                        dp[q] = dpp;
                    }
                }
            } else {
                recon(i + 2, fn);
    #pragma unroll
                for (int q = 0; q < V; ++q) {
                    T face = pos ? fc[q] : fn[q];
                    fs[q] = fc[q] - cour * (face - sp[q]);
                    sp[q] = face;
                    fc[q] = fn[q];
                }
            }
            T r[5];
            if (act) {
    #pragma unroll
                for (int k = 0; k < NV4; ++k) st4(outp + 4 * k, *reinterpret_cast<T(*)[4]>(fs + 4 * k));
                if constexpr (sizeof(T) == sizeof(double)) {
                    // the reverse sweep of the gradient records every step's f*
                    if (I.trace) {
                        double* tp = I.trace + ((size_t)(s - 1) * nx + c0 + li) * ldv + v0;
    #pragma unroll
                        for (int k = 0; k < NV4; ++k) st4(tp + 4 * k, *reinterpret_cast<T(*)[4]>(fs + 4 * k));
                    }
                }
                // the q = 0 terms of t1, t2 vanish (started at q = 1: the same
                // bits for finite values, two operations fewer per column)
                T s0 = fs[0], t1 = T(0), t2 = T(0);
    #pragma unroll
                for (int q = 1; q < V; ++q) {
                    s0 += fs[q];
                    t1 += T(q) * fs[q];
                    t2 += T(q * q) * fs[q];
                }
                r[0] = s0;
                r[1] = kx * s0;
                r[2] = ky * s0;
                r[3] = kz0 * s0 + t1;
                r[4] = kk0 * s0 + kz1 * t1 + t2;
            } else {
    #pragma unroll
                for (int q = 0; q < 5; ++q) r[q] = T(0);
            }
            T tot = warp_sum5(r, lane);
            if (writer) red[(li * NW + warp) * 5 + qsel] = tot;
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    for (int idx = tid; idx < ncols * 5; idx += NT) {
        int i = idx / 5, q = idx - i * 5;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < NW; ++k) acc += (double)red[(i * NW + k) * 5 + q];
        I.part[((size_t)(c0 + i) * I.n_vc + vc) * 5 + q] = acc;
    }
    // Arrival: the barrier orders every thread's stores (f* and partials)
    // before thread 0's gpu-scope fence and counter increment (cumulative
    // release); the last arriver fences again before its CTA reads the
    // other chunks' partials (acquire), then finalises the tile.
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        unsigned prev = atomicAdd(I.arrive + xt, 1u);
        s_last = prev == (unsigned)(I.n_vc - 1);
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last) finalize_tile<T, NT>(I, s, nsteps, xt, c0, ncols, pout, smem, status);
    // Claim the CTA's next ticket only now: claiming earlier (to hide the
    // atomic's latency) lengthens the window between claim and start, and the
    // next-step items then wait on unfinished neighbours more often (measured
    // slower on the 3 x 512 x 32^3 workload).
    if (tid == 0) *s_next = (long long)atomicAdd(ticket, 1ULL);
    __syncthreads();
}

// Resident CTAs per SM the register budget is sized for: float32 with 8
// velocities per thread (128 threads): 4; float32 with 4 (256 threads): 3;
// float64 (256 or 128 threads): 2.
template <typename T, int V>
struct MinBlocks {
    static constexpr int value = sizeof(T) == 4 ? (V == 8 ? 4 : 3) : 2;
};

template <typename T, int SCHEME, int V>
__global__ void __launch_bounds__(CHUNK / V, MinBlocks<T, V>::value)
k_fine_run(const Inst* __restrict__ insts, const InstState* __restrict__ st,
           const long long* __restrict__ prefix, const Active* __restrict__ active, int nsteps,
           unsigned long long* ticket, int* status, long long wait_ns, int poison)
{
    constexpr int H = SCHEME == 1 ? 2 : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_t;
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    const int ib = active->begin, ie = active->end;
    if (ib >= ie || nsteps <= 0) return;
    const long long base = prefix[ib];
    const long long W = prefix[ie] - base;
    const long long total = W * nsteps;
    // Tickets are claimed in increasing order by each CTA (the first one here,
    // the following ones at the end of each item).
    if (tid == 0) s_t = (long long)atomicAdd(ticket, 1ULL);
    __syncthreads();
    for (;;) {
        const long long t = s_t;
        if (t >= total || ld_status(status) != 0) break;
        const int s = (int)(t / W) + 1;
        const long long r = base + t % W;
        int lo = ib, hi = ie - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= r) lo = mid;
            else hi = mid - 1;
        }
        const Inst& I = insts[lo];
        const int loc = (int)(r - prefix[lo]);
        // tiles in zigzag order 0, n-1, 1, n-2, ...: every tile's neighbours
        // (the periodic wrap included) come at most two tiles apart, so the
        // items of the next step find their dependencies finished
        const int pidx = loc / I.n_vc, vc = loc - pidx * I.n_vc;
        const int xt = (pidx & 1) ? I.n_xt - 1 - (pidx >> 1) : (pidx >> 1);
        if (wait_ns > 0 && s > 1) {
            // poison (failure-detection check): the items of step 2 wait for a
            // step that never completes, so the bounded wait runs out
            const unsigned target = (poison && s == 2) ? 0xffffffffu : (unsigned)(s - 1);
            if (tid < 32) {
                bool ok = wait_tiles(I, xt, target, status, tid, (unsigned long long)wait_ns);
                if (tid == 0) s_ok = ok ? 1 : 0;
            }
            __syncthreads();
            if (!s_ok) break;
        }
        fine_item<T, H, V>(I, st[lo], s, nsteps, xt, vc, smem, status, ticket, &s_t);
    }
}

// Lift (Eq. 17): one CTA per (instance, x tile); tables of M[U_in] into
// tab[cur] with weight 1, moments of M into Ucur, a0 = 0.
template <typename T>
__global__ void __launch_bounds__(THREADS)
k_lift(const Inst* __restrict__ insts, InstState* st, const Active* __restrict__ active, int max_tiles,
       int* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int b = active->begin + blockIdx.y;
    if (b >= active->end) return;
    const Inst& I = insts[b];
    const int xt = blockIdx.x;
    if (xt >= I.n_xt) return;
    const int c0 = xt * I.tx, ncols = min(I.nx, c0 + I.tx) - c0;
    double* mom = reinterpret_cast<double*>(smem);
    double* par = mom + MAX_TX * 5;
    TabPar* tp = reinterpret_cast<TabPar*>(par);
    T* tb = reinterpret_cast<T*>(par + MAX_TX * 8);
    for (int i = threadIdx.x; i < ncols; i += THREADS) {
        double sm[5];
        sums_from_state(I.Uin, I.nx, c0 + i, I.dv, I.dv3, sm);
        if (sizeof(T) == 4) tp[i] = tabpar_from_sums(sm, 1.0, status);
        else prim_from_sums(sm, I.dv, I.dv3, 1.0, par + i * 8, status);
    }
    __syncthreads();
    InstState S = st[b];
    T* tout = reinterpret_cast<T*>(I.tab[S.cur]);
    write_tables<T, THREADS>(I, c0, ncols, par, tp, tout, tb);
    __syncthreads();
    project_columns<T, THREADS>(I, c0, ncols, mom, 0.0, tb, nullptr);
    if (xt == 0 && threadIdx.x == 0) st[b].a0 = 0.0;
}

__global__ void k_advance(const Inst* __restrict__ insts, InstState* st, const Active* __restrict__ active,
                          int nsteps)
{
    const int b = active->begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= active->end || nsteps <= 0) return;
    st[b].cur = (st[b].cur + nsteps) & 1;
    st[b].a0 = insts[b].a;
}

template <typename T>
__global__ void __launch_bounds__(THREADS)
k_materialize(const Inst* __restrict__ insts, const InstState* __restrict__ st, int b, double* out)
{
    const Inst& I = insts[b];
    const InstState S = st[b];
    const int c = blockIdx.x;
    const int v = blockIdx.y * CHUNK + threadIdx.x * VPT;
    if (v >= I.nv3) return;
    const int nv = I.nv, tw = 3 * nv;
    const int jz = v % nv, jy = (v / nv) % nv, jx = v / (nv * nv);
    const T* g = reinterpret_cast<const T*>(I.g[S.cur]) + (size_t)c * I.ldv + v;
    const T* tb = reinterpret_cast<const T*>(I.tab[S.cur]) + (size_t)c * tw;
    const T wg = (T)S.a0;
    T txy = tb[jx] * tb[nv + jy];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        T m = txy * tb[2 * nv + jz + q];
        T f = S.a0 != 0.0 ? wg * g[q] + m : m;
        out[(size_t)c * I.nv3 + v + q] = (double)f;
    }
}

template <typename T>
__global__ void __launch_bounds__(THREADS)
k_load_f(const Inst* __restrict__ insts, const InstState* __restrict__ st, int b, const double* f)
{
    const Inst& I = insts[b];
    const int c = blockIdx.x;
    const int v = blockIdx.y * CHUNK + threadIdx.x * VPT;
    if (v >= I.nv3) return;
    T* g = reinterpret_cast<T*>(I.g[st[b].cur]) + (size_t)c * I.ldv + v;
#pragma unroll
    for (int q = 0; q < 4; ++q) g[q] = (T)f[(size_t)c * I.nv3 + v + q];
}

// Moments of a loaded distribution (float64 accumulation, one CTA per x cell).
template <typename T>
__global__ void __launch_bounds__(THREADS)
k_state_moments(const Inst* __restrict__ insts, InstState* st, int b)
{
    const Inst& I = insts[b];
    const int c = blockIdx.x, nv = I.nv;
    const T* g = reinterpret_cast<const T*>(I.g[st[b].cur]) + (size_t)c * I.ldv;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int v = threadIdx.x; v < I.nv3; v += THREADS) {
        const int jz = v % nv, jy = (v / nv) % nv, jx = v / (nv * nv);
        double vx = -I.L + (jx + 0.5) * I.dv, vy = -I.L + (jy + 0.5) * I.dv, vz = -I.L + (jz + 0.5) * I.dv;
        double f = (double)g[v];
        acc[0] += f;
        acc[1] += vx * f;
        acc[2] += vy * f;
        acc[3] += vz * f;
        acc[4] += (vx * vx + vy * vy + vz * vz) * f;
    }
    __shared__ double sred[WARPS][5];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
        for (int o = 16; o; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 5; ++q) sred[warp][q] = acc[q];
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0.0;
        for (int k = 0; k < WARPS; ++k) t += sred[k][threadIdx.x];
        t *= I.dv3;
        if (threadIdx.x == 4) t *= 0.5;
        I.Ucur[(size_t)threadIdx.x * I.nx + c] = t;
    }
    if (c == 0 && threadIdx.x == 0) st[b].a0 = 1.0;
}

// ---- cluster-resident fine run ----
// For instances small enough to live in the shared memory of one thread-block
// cluster: CTA r of the cluster owns x cells [r w, r w + w) with all nv^3
// velocities, as the storage form above (g and the factor tables, two
// buffers each).  A step reconstructs f of its cells and of 2H halo cells --
// the neighbouring CTAs' cells (or the boundary ghosts) read from their
// shared memory through the cluster's distributed shared memory -- marches
// along x as the tiled kernel does, sums the moments of its own cells over
// all velocities in the CTA, and builds the tables of the next state; one
// cluster barrier per step publishes both buffers.  Lift, n steps and the
// projection run in one launch with no global-memory traffic in between, so
// a step costs a few microseconds instead of the dependency chain of global
// flags, partial sums and tile finalisers of the tiled kernel (which a
// batch too small to fill the GPU exposes).  float32 f, 8 v_z nodes per
// thread, nv^3 / 8 threads per CTA.
constexpr int CLV = 8;

__host__ __device__ inline size_t cl_floats_offset(int w, int nv, int nt)
{
    const size_t nv3 = (size_t)nv * nv * nv, tw = 3 * (size_t)nv;
    return align16((2 * (size_t)w * nv3 + 2 * (size_t)w * tw + (size_t)w * (nt / 32) * 5) * sizeof(float));
}

__host__ __device__ inline size_t cl_smem_bytes(int w, int nv, int nt)
{
    return align16(cl_floats_offset(w, nv, nt) + (size_t)w * 5 * sizeof(double) + (size_t)w * sizeof(TabPar));
}

// Factor tables of ncols cells from their parameter pairs tp[i], into
// shared memory only.
__device__ void cl_tables(const Inst& I, int ncols, const TabPar* tp, float* tb)
{
    const int tid = threadIdx.x, nt = blockDim.x, nv = I.nv, tw = 3 * nv;
    for (int idx = tid; idx < ncols * tw; idx += nt) {
        int i = idx / tw, rem = idx - i * tw, d = rem / nv, j = rem - d * nv;
        tb[idx] = tab_entry(tp[i], d, node_k(j, nv));
    }
}

__device__ __forceinline__ void ld8(const float* p, float (&o)[CLV])
{
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    o[0] = a.x, o[1] = a.y, o[2] = a.z, o[3] = a.w, o[4] = b.x, o[5] = b.y, o[6] = b.z, o[7] = b.w;
}

template <int SCHEME, int NT>
__global__ void __launch_bounds__(NT, 1)
k_fine_cluster(const Inst* __restrict__ insts, const Active* __restrict__ active, int nsteps, int w, int* status)
{
    constexpr int H = SCHEME == 1 ? 2 : 1, V = CLV, NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int b = active->begin + (int)blockIdx.x / C;  // one cluster per instance
    if (b >= active->end) return;                       // the same for every CTA of the cluster
    const Inst& I = insts[b];
    const int nx = I.nx, nv = I.nv, nv3 = I.nv3, tw = 3 * nv, bc = I.bc;
    const int c0 = rank * w, ncols = min(nx, c0 + w) - c0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    float* g = reinterpret_cast<float*>(smem);  // [2][w][nv3]
    float* tab = g + 2 * (size_t)w * nv3;        // [2][w][tw]
    float* red = tab + 2 * (size_t)w * tw;       // [w][NW][5] warp totals
    double* mom = reinterpret_cast<double*>(smem + cl_floats_offset(w, nv, NT));  // [w][5]
    TabPar* tp = reinterpret_cast<TabPar*>(mom + 5 * w);                            // [w]

    // lift (Eq. 17) of the own cells into tables buffer 0: the conserved
    // moments as grid-unit sums, the Maxwellian parameters in float64
    for (int i = tid; i < ncols; i += NT) {
        double sm[5];
        sums_from_state(I.Uin, nx, c0 + i, I.dv, I.dv3, sm);
        tp[i] = tabpar_from_sums(sm, 1.0, status);
    }
    __syncthreads();
    cl_tables(I, ncols, tp, tab);
    if (nsteps <= 0) {  // the projection of the lifted state
        __syncthreads();
        project_columns<float, NT>(I, c0, ncols, mom, 0.0, tab, I.Uout);
        cl.sync();
        return;
    }
    cl.sync();  // every rank's lifted tables visible

    const int v0 = tid * V;  // NT * V == nv3
    const int jz = v0 % nv, jy = (v0 / nv) % nv, jx = v0 / (nv * nv);
    const int jxf = nv - 1 - jx, v0f = (jxf * nv + jy) * nv + jz;
    const double vxd = -I.L + (jx + 0.5) * I.dv;
    const bool pos = vxd > 0.0;
    const float cour = (float)(I.nu * vxd);
    // moment weights in grid units, as in the tiled kernel
    const float kx = 0.5f * (float)(2 * jx + 1 - nv), ky = 0.5f * (float)(2 * jy + 1 - nv);
    const float kz0 = 0.5f * (float)(2 * jz + 1 - nv), kz1 = (float)(2 * jz + 1 - nv);
    const float kk0 = kx * kx + ky * ky + kz0 * kz0;
    const int qsel = lane < 4 ? 0 : lane < 8 ? 1 : lane < 16 ? 2 : lane < 24 ? 3 : 4;
    const bool writer = lane == 0 || lane == 4 || lane == 8 || lane == 16 || lane == 24;

    for (int s = 1; s <= nsteps; ++s) {
        const int p = (s - 1) & 1;
        const float wg = s == 1 ? 0.f : (float)I.a;  // the lifted state has no g part
        // f of extended cell e (x cell c0 - H + e) at this thread's velocities
        auto recon = [&](int e, float (&o)[V]) {
            bool fl;
            const int cc = map_col(c0 - H + e, nx, bc, fl);
            const int owner = cc / w, lc = cc - owner * w;
            const float* gp = g + ((size_t)p * w + lc) * nv3;
            const float* tp = tab + ((size_t)p * w + lc) * tw;
            if (owner != rank) {
                gp = cl.map_shared_rank(const_cast<float*>(gp), owner);
                tp = cl.map_shared_rank(const_cast<float*>(tp), owner);
            }
            const float txy = tp[fl ? jxf : jx] * tp[nv + jy];
            float tz[V];
            ld8(tp + 2 * nv + jz, tz);
            if (wg != 0.f) {
                float gv[V];
                ld8(gp + (fl ? v0f : v0), gv);
#pragma unroll
                for (int q = 0; q < V; ++q) o[q] = wg * gv[q] + txy * tz[q];
            } else {
#pragma unroll
                for (int q = 0; q < V; ++q) o[q] = txy * tz[q];
            }
        };
        float fc[V], fn[V], dm[V], dp[V], sp[V];
        if (H == 2) {
            float f0[V], f1[V];
            recon(0, f0);
            recon(1, f1);
            recon(2, fc);
            recon(3, fn);
#pragma unroll
            for (int q = 0; q < V; ++q) {
                float d0 = f1[q] - f0[q];
                dm[q] = fc[q] - f1[q];
                dp[q] = fn[q] - fc[q];
                sp[q] = pos ? f1[q] + 0.5f * minmod2(d0, dm[q]) : fc[q] - 0.5f * minmod2(dm[q], dp[q]);
            }
        } else {
            float f0[V];
            recon(0, f0);
            recon(1, fc);
#pragma unroll
            for (int q = 0; q < V; ++q) sp[q] = pos ? f0[q] : fc[q];
        }
        float* outp = g + (size_t)(p ^ 1) * w * nv3 + v0;
        for (int i = 0; i < ncols; ++i, outp += nv3) {
            float fs[V];
            if (H == 2) {
                float fnn[V];
                recon(i + 4, fnn);
#pragma unroll
                for (int q = 0; q < V; ++q) {
                    float dpp = fnn[q] - fn[q];
                    float face = pos ? fc[q] + 0.5f * minmod2(dm[q], dp[q]) : fn[q] - 0.5f * minmod2(dp[q], dpp);
                    fs[q] = fc[q] - cour * (face - sp[q]);
                    sp[q] = face;
                    fc[q] = fn[q];
                    fn[q] = fnn[q];
                    dm[q] = dp[q];
                    dp[q] = dpp;
                }
            } else {
                recon(i + 2, fn);
#pragma unroll
                for (int q = 0; q < V; ++q) {
                    float face = pos ? fc[q] : fn[q];
                    fs[q] = fc[q] - cour * (face - sp[q]);
                    sp[q] = face;
                    fc[q] = fn[q];
                }
            }
            reinterpret_cast<float4*>(outp)[0] = make_float4(fs[0], fs[1], fs[2], fs[3]);
            reinterpret_cast<float4*>(outp)[1] = make_float4(fs[4], fs[5], fs[6], fs[7]);
            float s0 = fs[0], t1 = 0.f, t2 = 0.f;
#pragma unroll
            for (int q = 1; q < V; ++q) {
                s0 += fs[q];
                t1 += float(q) * fs[q];
                t2 += float(q * q) * fs[q];
            }
            float r[5];
            r[0] = s0;
            r[1] = kx * s0;
            r[2] = ky * s0;
            r[3] = kz0 * s0 + t1;
            r[4] = kk0 * s0 + kz1 * t1 + t2;
            float tot = warp_sum5(r, lane);
            if (writer) red[(i * NW + warp) * 5 + qsel] = tot;
        }
        __syncthreads();
        // moment sums of the own cells: half a warp per (cell, moment), lane
        // k adding warp k's total, in float64 (NW <= 16)
        for (int vb = 2 * warp; vb < ncols * 5; vb += 2 * NW) {
            const int vi = vb + (lane >> 4), k = lane & 15;
            const bool on = vi < ncols * 5;
            double x = on && k < NW ? (double)red[((vi / 5) * NW + k) * 5 + vi % 5] : 0.0;
#pragma unroll
            for (int o = 8; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (on && k == 0) mom[vi] = x;
        }
        __syncthreads();
        for (int i = tid; i < ncols; i += NT) tp[i] = tabpar_from_sums(mom + i * 5, I.b, status);
        __syncthreads();
        float* tnext = tab + (size_t)(p ^ 1) * w * tw;
        cl_tables(I, ncols, tp, tnext);
        if (s == nsteps) {  // projection (Eq. 18) of f = a g + M
            __syncthreads();
            project_columns<float, NT>(I, c0, ncols, mom, I.a, tnext, I.Uout);
        }
        cl.sync();  // the next state of every rank visible; no rank still reads this one
    }
}

template <int SCHEME, int NT>
void* fine_cluster_ptr()
{
    return reinterpret_cast<void*>(&k_fine_cluster<SCHEME, NT>);
}

void* fine_cluster_kernel(int scheme, int nv)
{
    if (nv == 8) return scheme == 1 ? fine_cluster_ptr<1, 64>() : fine_cluster_ptr<0, 64>();
    if (nv == 16) return scheme == 1 ? fine_cluster_ptr<1, 512>() : fine_cluster_ptr<0, 512>();
    return nullptr;
}

template <typename T, int SCHEME, int V>
void* fine_kernel_ptr()
{
    return reinterpret_cast<void*>(&k_fine_run<T, SCHEME, V>);
}

void* fine_kernel(int precision, int scheme, int vpt)
{
    if (precision == 0 && vpt == 8) return scheme == 1 ? fine_kernel_ptr<double, 1, 8>() : fine_kernel_ptr<double, 0, 8>();
    if (precision == 0) return scheme == 1 ? fine_kernel_ptr<double, 1, 4>() : fine_kernel_ptr<double, 0, 4>();
    if (vpt == 8) return scheme == 1 ? fine_kernel_ptr<float, 1, 8>() : fine_kernel_ptr<float, 0, 8>();
    return scheme == 1 ? fine_kernel_ptr<float, 1, 4>() : fine_kernel_ptr<float, 0, 4>();
}

}  // namespace

size_t fine_run_smem(int precision, int vpt, int tx, int nv, int H)
{
    size_t es = precision == 0 ? sizeof(double) : sizeof(float);
    int nw = CHUNK / vpt / 32;
    size_t ring = (size_t)(precision == 0 ? Ring<double>::SLOTS : Ring<float>::SLOTS) * CHUNK * es;
    size_t item = ring + align16((size_t)(tx + 2 * H) * 3 * nv * es) + (size_t)tx * nw * 5 * es;
    size_t fin = (size_t)MAX_TX * 13 * sizeof(double) + (size_t)tx * 3 * nv * es;
    return item > fin ? item : fin;
}

size_t lift_smem(int precision, int tx, int nv)
{
    size_t es = precision == 0 ? sizeof(double) : sizeof(float);
    return (size_t)MAX_TX * 13 * sizeof(double) + (size_t)tx * 3 * nv * es;
}

// Dynamic shared memory may use what the static allocation leaves of the opt-in limit.
static void raise_smem(const void* fn, int max_smem)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - (int)fa.sharedSizeBytes);
    cudaGetLastError();
}

void prepare_fine_kernels(int max_smem)
{
    const int vp[4][2] = {{0, 4}, {0, 8}, {1, 4}, {1, 8}};
    for (auto& c : vp)
        for (int sch = 0; sch < 2; ++sch) raise_smem(fine_kernel(c[0], sch, c[1]), max_smem);
    raise_smem(reinterpret_cast<const void*>(&k_lift<double>), max_smem);
    raise_smem(reinterpret_cast<const void*>(&k_lift<float>), max_smem);
    for (int nv : {8, 16})
        for (int sch = 0; sch < 2; ++sch) {
            const void* fn = fine_cluster_kernel(sch, nv);
            raise_smem(fn, max_smem);
            cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaGetLastError();
        }
}

int fine_run_occupancy(int precision, int scheme, int vpt, size_t smem, int* blocks_per_sm)
{
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fine_kernel(precision, scheme, vpt),
                                                                  CHUNK / vpt, smem);
    return (int)e;
}

cudaError_t launch_fine_run(int precision, int scheme, int vpt, const Inst* insts, InstState* st,
                            const long long* prefix, const Active* active, int nsteps,
                            unsigned long long* ticket, int* status, long long wait_ns, int grid, size_t smem,
                            cudaStream_t s, int poison)
{
    void* args[] = {(void*)&insts, (void*)&st, (void*)&prefix, (void*)&active, (void*)&nsteps,
                    (void*)&ticket, (void*)&status, (void*)&wait_ns, (void*)&poison};
    return cudaLaunchKernel(fine_kernel(precision, scheme, vpt), dim3(grid), dim3(CHUNK / vpt), args, smem, s);
}

cudaError_t launch_lift(int precision, const Inst* insts, InstState* st, const Active* active, int max_tiles,
                        int n_inst_max, size_t smem, int* status, cudaStream_t s)
{
    dim3 grid(max_tiles, n_inst_max);
    if (precision == 0) k_lift<double><<<grid, THREADS, smem, s>>>(insts, st, active, max_tiles, status);
    else k_lift<float><<<grid, THREADS, smem, s>>>(insts, st, active, max_tiles, status);
    return cudaGetLastError();
}

cudaError_t launch_advance(const Inst* insts, InstState* st, const Active* active, int nsteps, int n_inst_max,
                           cudaStream_t s)
{
    int blocks = (n_inst_max + 127) / 128;
    k_advance<<<blocks, 128, 0, s>>>(insts, st, active, nsteps);
    return cudaGetLastError();
}

cudaError_t launch_materialize(int precision, const Inst* insts, const InstState* st, int b, const Inst& h,
                               double* out, cudaStream_t s)
{
    dim3 grid(h.nx, h.n_vc);
    if (precision == 0) k_materialize<double><<<grid, THREADS, 0, s>>>(insts, st, b, out);
    else k_materialize<float><<<grid, THREADS, 0, s>>>(insts, st, b, out);
    return cudaGetLastError();
}

cudaError_t launch_set_f(int precision, const Inst* insts, InstState* st, int b, const Inst& h, const double* f,
                         cudaStream_t s)
{
    dim3 grid(h.nx, h.n_vc);
    size_t es = precision == 0 ? sizeof(double) : sizeof(float);
    // tables of the loaded state are zero: f = 1 * g + 0
    cudaError_t e = cudaMemsetAsync(h.tab[0], 0, (size_t)h.nx * 3 * h.nv * es, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h.tab[1], 0, (size_t)h.nx * 3 * h.nv * es, s);
    if (e != cudaSuccess) return e;
    if (precision == 0) {
        k_load_f<double><<<grid, THREADS, 0, s>>>(insts, st, b, f);
        k_state_moments<double><<<h.nx, THREADS, 0, s>>>(insts, st, b);
    } else {
        k_load_f<float><<<grid, THREADS, 0, s>>>(insts, st, b, f);
        k_state_moments<float><<<h.nx, THREADS, 0, s>>>(insts, st, b);
    }
    return cudaGetLastError();
}

// Cluster-resident fine run: the cells per CTA w (the fewest that keep the
// cluster at <= 16 CTAs) and the shared memory of a CTA; false when nv has no
// instantiation (8 or 16) or the cells do not fit.
bool fine_cluster_plan(int nx, int nv, int max_smem, int* C, int* w, size_t* smem)
{
    const void* fn = fine_cluster_kernel(0, nv);
    if (!fn || nx < 1) return false;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int ww = (nx + 15) / 16;
    const size_t sm = cl_smem_bytes(ww, nv, nv * nv * nv / CLV);
    if (sm + fa.sharedSizeBytes > (size_t)max_smem) return false;
    *w = ww;
    *C = (nx + ww - 1) / ww;
    *smem = sm;
    return true;
}

static cudaLaunchConfig_t cluster_config(int nv, int n_inst, int C, size_t smem, cudaStream_t s,
                                         cudaLaunchAttribute* at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_inst * C, 1, 1);
    cfg.blockDim = dim3(nv * nv * nv / CLV, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

int fine_cluster_resident(int scheme, int nv, int C, size_t smem)
{
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_config(nv, 1, C, smem, 0, at);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fine_cluster_kernel(scheme, nv), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_fine_cluster(int scheme, int nv, const Inst* insts, const Active* active, int n_inst_max,
                                int nsteps, int C, int w, size_t smem, int* status, cudaStream_t s)
{
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_config(nv, n_inst_max, C, smem, s, at);
    void* args[] = {(void*)&insts, (void*)&active, (void*)&nsteps, (void*)&w, (void*)&status};
    return cudaLaunchKernelExC(&cfg, fine_cluster_kernel(scheme, nv), args);
}

}  // namespace prk
