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
// One CTA runs the whole sweep (the loop over n is sequential by nature);
// the state lives in shared memory when it fits.  This file is compiled
// without floating-point contraction so that the arithmetic is the plain
// IEEE sequence of the formulas above.
#include <math.h>

#include "pr_kernels.h"

namespace prk {

namespace {

constexpr int CT = 1024;  // threads of the coarse CTA

struct Prim {
    double ux, uy, uz, p, th;
};

__device__ __forceinline__ Prim prim(const double* v)
{
    Prim q;
    double rho = v[0];
    q.ux = v[1] / rho;
    q.uy = v[2] / rho;
    q.uz = v[3] / rho;
    q.th = (2.0 * v[4] / rho - (q.ux * q.ux + q.uy * q.uy + q.uz * q.uz)) / 3.0;
    q.p = rho * q.th;
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

__device__ __forceinline__ void fetch(const double* A, const double* Cc, int nx, int bc, int c, CellF& o)
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
#pragma unroll
    for (int q = 0; q < 5; ++q) o.v[q] = A[q * nx + cc];
    o.ux = Cc[cc];
    o.uy = Cc[nx + cc];
    o.uz = Cc[2 * nx + cc];
    o.th = Cc[3 * nx + cc];
    o.p = Cc[4 * nx + cc];
#pragma unroll
    for (int q = 0; q < 5; ++q) o.h[q] = Cc[(5 + q) * nx + cc];
    o.s = Cc[10 * nx + cc];
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
// with mu = rho theta, kappa = 5 rho theta / 2, gradients (b - a)/dx and
// coefficients and u averaged over the face.
__device__ __forceinline__ void face_flux(const CellF& a, const CellF& b, double visc, double dx, double* H)
{
    const double S = a.s > b.s ? a.s : b.s;
#pragma unroll
    for (int q = 0; q < 5; ++q) H[q] = 0.5 * (a.h[q] + b.h[q]) - 0.5 * S * (b.v[q] - a.v[q]);
    if (visc > 0.0) {
        const double eps = visc;
        double mu = 0.5 * (a.p + b.p);
        double kappa = 2.5 * mu;
        double dux = (b.ux - a.ux) / dx, duy = (b.uy - a.uy) / dx, duz = (b.uz - a.uz) / dx, dth = (b.th - a.th) / dx;
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

// G over dT applied to A (work B, cache Cc of NCACHE nx doubles); the result
// ends in A.  Needs the whole CTA.  Per local step: one pass caching each
// cell's primitives, flux and speed (and the two maxima of the CFL limits),
// one pass forming each cell's two face fluxes and its update, three CTA
// barriers; the two state buffers swap roles.
__device__ void coarse_G(const CoarseParams& p, double* A, double* B, double* Cc, double dT, int* status, double* sh)
{
    const int nx = p.nx;
    double* cur = A;
    double* nxt = B;
    double t = 0.0;
    while (t < dT) {
        double smax = 0.0, thmax = 0.0;
        bool bad = false;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            double v[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) v[q] = cur[q * nx + i];
            Prim pr = prim(v);
            if (!(v[0] > 0.0) || !(pr.th > 0.0)) bad = true;
            double c = p.sound == 1 ? sqrt(pr.th) : sqrt(5.0 * pr.th / 3.0);
            double s = fabs(pr.ux) + c;
            if (s > smax) smax = s;
            if (pr.th > thmax) thmax = pr.th;
            Cc[i] = pr.ux;
            Cc[nx + i] = pr.uy;
            Cc[2 * nx + i] = pr.uz;
            Cc[3 * nx + i] = pr.th;
            Cc[4 * nx + i] = pr.p;
            Cc[5 * nx + i] = v[1];
            Cc[6 * nx + i] = v[1] * pr.ux + pr.p;
            Cc[7 * nx + i] = v[1] * pr.uy;
            Cc[8 * nx + i] = v[1] * pr.uz;
            Cc[9 * nx + i] = pr.ux * (v[4] + pr.p);
            Cc[10 * nx + i] = s;
        }
        if (bad) atomicCAS(status, 0, ST_NONPHYS);
        block_max2(smax, thmax, sh);  // its barriers also publish the cache
        if (!(smax > 0.0) || isnan(smax)) break;
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
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            CellF L, M, R;
            fetch(cur, Cc, nx, p.bc, i - 1, L);
            fetch(cur, Cc, nx, p.bc, i, M);
            fetch(cur, Cc, nx, p.bc, i + 1, R);
            double Hl[5], Hr[5];
            face_flux(L, M, p.visc, p.dx, Hl);
            face_flux(M, R, p.visc, p.dx, Hr);
#pragma unroll
            for (int q = 0; q < 5; ++q) nxt[q * nx + i] = cur[q * nx + i] - dt / p.dx * (Hr[q] - Hl[q]);
            if (p.E) {  // exterior force: forward-Euler source on the old state
                nxt[1 * nx + i] += dt * cur[0 * nx + i] * p.E[i];
                nxt[4 * nx + i] += dt * cur[1 * nx + i] * p.E[i];
            }
        }
        __syncthreads();
        double* tmp = cur;
        cur = nxt;
        nxt = tmp;
        if (last) break;
        t += dt;
    }
    if (cur != A) {
        for (int i = threadIdx.x; i < 5 * nx; i += blockDim.x) A[i] = cur[i];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(CT)
k_coarse(CoarseParams p, const double* Vin, double* Vout, double dT, double* work, int use_smem, int* status)
{
    extern __shared__ __align__(16) double dsm[];
    __shared__ double sh[2 * (CT / 32)];
    double* A = use_smem ? dsm : work;
    double* B = A + 5 * p.nx;
    double* Cc = B + 5 * p.nx;
    for (int i = threadIdx.x; i < 5 * p.nx; i += blockDim.x) A[i] = Vin[i];
    __syncthreads();
    coarse_G(p, A, B, Cc, dT, status, sh);
    __syncthreads();
    for (int i = threadIdx.x; i < 5 * p.nx; i += blockDim.x) Vout[i] = A[i];
}

__global__ void __launch_bounds__(CT)
k_sweep(CoarseParams p, int N, double dT, const int* dk, double* U, const double* PFL, double* Gs, double* err,
        double* work, int use_smem, int* status, int bump, int* dk_mut)
{
    extern __shared__ __align__(16) double dsm[];
    __shared__ double sh[2 * (CT / 32)];
    const int nx = p.nx, sz = 5 * nx;
    const int k = *dk;
    double* A = use_smem ? dsm : work;
    double* B = A + sz;
    double* Cc = B + sz;
    double emax = 0.0;
    for (int n = (k > 1 ? k : 1); n <= N; ++n) {
        for (int i = threadIdx.x; i < sz; i += blockDim.x) A[i] = U[(size_t)(n - 1) * sz + i];
        __syncthreads();
        coarse_G(p, A, B, Cc, dT, status, sh);
        for (int i = threadIdx.x; i < sz; i += blockDim.x) {
            const size_t o = (size_t)n * sz + i;
            double gv = A[i];
            double nv = k > 0 ? gv + (PFL[o] - Gs[o]) : gv;
            double d = fabs(nv - U[o]);
            if (d > emax) emax = d;
            U[o] = nv;
            Gs[o] = gv;
        }
        __syncthreads();
    }
    emax = block_max(emax, sh);
    if (threadIdx.x == 0) {
        err[k] = emax;
        if (bump) *dk_mut = k + 1;
    }
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

// Doubles of workspace of one coarse step: state, next state, cell cache.
size_t work_doubles(int nx) { return (size_t)(10 + NCACHE) * nx; }

bool fits_smem(int nx) { return work_doubles(nx) * sizeof(double) <= 200 * 1024; }

}  // namespace

void prepare_coarse_kernels(int max_smem)
{
    const void* fns[2] = {reinterpret_cast<const void*>(&k_coarse), reinterpret_cast<const void*>(&k_sweep)};
    for (const void* fn : fns) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - (int)fa.sharedSizeBytes);
        cudaGetLastError();
    }
}

cudaError_t launch_coarse(const CoarseParams& p, const double* Vin, double* Vout, double dT, double* work,
                          int* status, cudaStream_t s)
{
    int use = fits_smem(p.nx);
    size_t smem = use ? work_doubles(p.nx) * sizeof(double) : 0;
    int threads = p.nx < CT ? ((p.nx + 31) / 32) * 32 : CT;
    k_coarse<<<1, threads, smem, s>>>(p, Vin, Vout, dT, work, use, status);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const CoarseParams& p, int N, double dT, const int* dk, double* U, const double* PFL,
                         double* Gs, double* err, double* work, int* status, int bump, int* dk_mut,
                         cudaStream_t s)
{
    int use = fits_smem(p.nx);
    size_t smem = use ? work_doubles(p.nx) * sizeof(double) : 0;
    int threads = p.nx < CT ? ((p.nx + 31) / 32) * 32 : CT;
    k_sweep<<<1, threads, smem, s>>>(p, N, dT, dk, U, PFL, Gs, err, work, use, status, bump, dk_mut);
    return cudaGetLastError();
}

size_t coarse_work_doubles(int nx) { return work_doubles(nx); }

cudaError_t launch_set_active(const int* dk, Active* active, int first_slice, int n_inst, int N, cudaStream_t s)
{
    k_set_active<<<1, 1, 0, s>>>(dk, active, first_slice, n_inst, N);
    return cudaGetLastError();
}

}  // namespace prk
