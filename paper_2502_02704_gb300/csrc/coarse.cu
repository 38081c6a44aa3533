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

__device__ __forceinline__ double speed(const double* v, int sound)
{
    Prim q = prim(v);
    double c = sound == 1 ? sqrt(q.th) : sqrt(5.0 * q.th / 3.0);
    return fabs(q.ux) + c;
}

// state of cell c (ghosts allowed) of V[5][nx]
__device__ __forceinline__ void cell(const double* V, int nx, int bc, int c, double* out)
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
    for (int q = 0; q < 5; ++q) out[q] = V[q * nx + cc];
    if (flip) out[1] = -out[1];
}

__device__ __forceinline__ void flux(const double* v, double* h)
{
    Prim q = prim(v);
    h[0] = v[1];
    h[1] = v[1] * q.ux + q.p;
    h[2] = v[1] * q.uy;
    h[3] = v[1] * q.uz;
    h[4] = q.ux * (v[4] + q.p);
}

__device__ void rusanov(const double* V, int nx, int bc, int sound, int c, double* H)
{
    double a[5], b[5], ha[5], hb[5];
    cell(V, nx, bc, c, a);
    cell(V, nx, bc, c + 1, b);
    flux(a, ha);
    flux(b, hb);
    double sa = speed(a, sound), sb = speed(b, sound);
    double S = sa > sb ? sa : sb;
#pragma unroll
    for (int q = 0; q < 5; ++q) H[q] = 0.5 * (ha[q] + hb[q]) - 0.5 * S * (b[q] - a[q]);
}

// Viscous flux D_{c+1/2} of the compressible Navier-Stokes model (Eq. 8):
// mu = rho theta, kappa = 5 rho theta / 2 (BGK, tau = 1), gradients
// (V_{c+1} - V_c)/dx, coefficients and u averaged over the face.
__device__ void viscous(const double* V, int nx, int bc, double dx, double eps, int c, double* D)
{
    double a[5], b[5];
    cell(V, nx, bc, c, a);
    cell(V, nx, bc, c + 1, b);
    Prim pa = prim(a), pb = prim(b);
    double mu = 0.5 * (pa.p + pb.p);
    double kappa = 2.5 * mu;
    double dux = (pb.ux - pa.ux) / dx, duy = (pb.uy - pa.uy) / dx, duz = (pb.uz - pa.uz) / dx, dth = (pb.th - pa.th) / dx;
    double ux = 0.5 * (pa.ux + pb.ux), uy = 0.5 * (pa.uy + pb.uy), uz = 0.5 * (pa.uz + pb.uz);
    double sxx = -eps * mu * (4.0 / 3.0) * dux, sxy = -eps * mu * duy, sxz = -eps * mu * duz;
    double q = -eps * kappa * dth;
    D[0] = 0.0;
    D[1] = sxx;
    D[2] = sxy;
    D[3] = sxz;
    D[4] = sxx * ux + sxy * uy + sxz * uz + q;
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

// G over dT applied in place to A (work B); result ends in A.  Needs the whole CTA.
__device__ void coarse_G(const CoarseParams& p, double* A, double* B, double dT, int* status, double* sh)
{
    const int nx = p.nx;
    double t = 0.0;
    while (t < dT) {
        double smax = 0.0, thmax = 0.0;
        bool bad = false;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            double v[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) v[q] = A[q * nx + i];
            Prim pr = prim(v);
            if (!(v[0] > 0.0) || !(pr.th > 0.0)) bad = true;
            double s = speed(v, p.sound);
            if (s > smax) smax = s;
            if (pr.th > thmax) thmax = pr.th;
        }
        if (bad) atomicCAS(status, 0, ST_NONPHYS);
        smax = block_max(smax, sh);
        if (!(smax > 0.0) || isnan(smax)) return;
        double rem = dT - t;
        double dt = p.cfl * p.dx / smax;
        if (p.visc > 0.0) {
            thmax = block_max(thmax, sh);
            double dtv = p.cfl * p.dx * p.dx / (2.0 * p.visc * (5.0 / 3.0) * thmax);
            if (dtv < dt) dt = dtv;
        }
        bool last = false;
        if (dt >= rem) {
            dt = rem;
            last = true;
        }
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            double Hr[5], Hl[5];
            rusanov(A, nx, p.bc, p.sound, i, Hr);
            rusanov(A, nx, p.bc, p.sound, i - 1, Hl);
            if (p.visc > 0.0) {  // compressible Navier-Stokes (Eq. 8)
                double Dr[5], Dl[5];
                viscous(A, nx, p.bc, p.dx, p.visc, i, Dr);
                viscous(A, nx, p.bc, p.dx, p.visc, i - 1, Dl);
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    Hr[q] += Dr[q];
                    Hl[q] += Dl[q];
                }
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) B[q * nx + i] = A[q * nx + i] - dt / p.dx * (Hr[q] - Hl[q]);
            if (p.E) {  // exterior force: forward-Euler source on the old state
                B[1 * nx + i] += dt * A[0 * nx + i] * p.E[i];
                B[4 * nx + i] += dt * A[1 * nx + i] * p.E[i];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 5 * nx; i += blockDim.x) A[i] = B[i];
        __syncthreads();
        if (last) break;
        t += dt;
    }
}

__global__ void __launch_bounds__(CT)
k_coarse(CoarseParams p, const double* Vin, double* Vout, double dT, double* work, int use_smem, int* status)
{
    extern __shared__ __align__(16) double dsm[];
    __shared__ double sh[CT / 32];
    double* A = use_smem ? dsm : work;
    double* B = A + 5 * p.nx;
    for (int i = threadIdx.x; i < 5 * p.nx; i += blockDim.x) A[i] = Vin[i];
    __syncthreads();
    coarse_G(p, A, B, dT, status, sh);
    __syncthreads();
    for (int i = threadIdx.x; i < 5 * p.nx; i += blockDim.x) Vout[i] = A[i];
}

__global__ void __launch_bounds__(CT)
k_sweep(CoarseParams p, int N, double dT, const int* dk, double* U, const double* PFL, double* Gs, double* err,
        double* work, int use_smem, int* status, int bump, int* dk_mut)
{
    extern __shared__ __align__(16) double dsm[];
    __shared__ double sh[CT / 32];
    const int nx = p.nx, sz = 5 * nx;
    const int k = *dk;
    double* A = use_smem ? dsm : work;
    double* B = A + sz;
    double emax = 0.0;
    for (int n = (k > 1 ? k : 1); n <= N; ++n) {
        for (int i = threadIdx.x; i < sz; i += blockDim.x) A[i] = U[(size_t)(n - 1) * sz + i];
        __syncthreads();
        coarse_G(p, A, B, dT, status, sh);
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

bool fits_smem(int nx) { return (size_t)10 * nx * sizeof(double) <= 200 * 1024; }

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
    size_t smem = use ? (size_t)10 * p.nx * sizeof(double) : 0;
    int threads = p.nx < CT ? ((p.nx + 31) / 32) * 32 : CT;
    k_coarse<<<1, threads, smem, s>>>(p, Vin, Vout, dT, work, use, status);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const CoarseParams& p, int N, double dT, const int* dk, double* U, const double* PFL,
                         double* Gs, double* err, double* work, int* status, int bump, int* dk_mut,
                         cudaStream_t s)
{
    int use = fits_smem(p.nx);
    size_t smem = use ? (size_t)10 * p.nx * sizeof(double) : 0;
    int threads = p.nx < CT ? ((p.nx + 31) / 32) * 32 : CT;
    k_sweep<<<1, threads, smem, s>>>(p, N, dT, dk, U, PFL, Gs, err, work, use, status, bump, dk_mut);
    return cudaGetLastError();
}

cudaError_t launch_set_active(const int* dk, Active* active, int first_slice, int n_inst, int N, cudaStream_t s)
{
    k_set_active<<<1, 1, 0, s>>>(dk, active, first_slice, n_inst, N);
    return cudaGetLastError();
}

}  // namespace prk
