// pr_fine_step_noalloc: one fused float64 fine step of one instance that
// allocates no memory.  For callers that cannot call cudaMalloc (for example a
// host application whose memory is owned by another allocator, or code running
// where allocation is forbidden once set up): the caller passes the input and
// output distributions, and every other buffer the fine kernel needs -- the
// instance descriptor, the Maxwellian factor tables, the velocity-chunk moment
// partials, the arrival/completion counters and the status word -- lives in
// one file-scope device array of fixed size (NOALLOC_BYTES, held by every GPU
// that loads the library until the process exits).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "pr.h"
#include "pr_kernels.h"

void pr_internal_set_global_error(const char* msg);

namespace {

constexpr size_t NOALLOC_BYTES = size_t(4) << 20;  // 4 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_pr_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_mu;
unsigned char* g_ptr[MAX_DEVICES] = {};

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array for the current device (set up once per
// device; cudaGetSymbolAddress must run with that device current).
int scratch_address(unsigned char** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return PR_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_pr_noalloc_scratch);
        if (e != cudaSuccess || !p) return PR_ECUDA;
        int smax = 0;
        cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        prk::prepare_fine_kernels(smax);
        g_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_ptr[dev];
    return PR_OK;
}

}  // namespace

extern "C" int pr_fine_step_noalloc(const pr_instance* d, const double* f_in, double* f_out, void* stream)
{
    auto reject = [](const char* why) {
        pr_internal_set_global_error(why);
        return PR_EINVAL;
    };
    auto cuda_fail = [](cudaError_t e) {
        char msg[160];
        snprintf(msg, sizeof msg, "pr_fine_step_noalloc: %s", cudaGetErrorString(e));
        pr_internal_set_global_error(msg);
        return PR_ECUDA;
    };
    if (!d || !f_in || !f_out || f_in == f_out) return reject("pr_fine_step_noalloc: null or aliased arguments");
    if (d->nx < 1 || d->nv < 4 || d->nv % 4 || !(d->x1 > d->x0) || !std::isfinite(d->x0) || !std::isfinite(d->x1) ||
        !(d->L > 0) || !std::isfinite(d->L) || !(d->eps > 0) || !(d->dt > 0) || !std::isfinite(d->dt) || d->bc < 0 ||
        d->bc > 2 || d->scheme < 0 || d->scheme > 1 || (d->scheme == PR_MUSCL && d->bc == PR_BC_REFLECT && d->nx < 2))
        return reject("pr_fine_step_noalloc: invalid instance parameters (sizes, domain, L, eps > 0, finite dt > 0, "
                      "bc, scheme)");
    if ((reinterpret_cast<uintptr_t>(f_in) | reinterpret_cast<uintptr_t>(f_out)) & 15)
        return reject("pr_fine_step_noalloc: f_in and f_out must be 16-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    prk::Inst I;
    memset(&I, 0, sizeof I);
    I.nx = d->nx;
    I.nv = d->nv;
    I.nv3 = d->nv * d->nv * d->nv;
    I.ldv = I.nv3;
    I.bc = d->bc;
    I.scheme = d->scheme;
    I.tx = d->nx < 32 ? d->nx : 32;
    I.n_xt = (I.nx + I.tx - 1) / I.tx;
    I.n_vc = (I.nv3 + prk::CHUNK - 1) / prk::CHUNK;
    I.L = d->L;
    I.dv = 2.0 * d->L / d->nv;
    I.dv3 = I.dv * I.dv * I.dv;
    I.dx = (d->x1 - d->x0) / d->nx;
    I.dt = d->dt;
    I.eps = d->eps;
    if (std::isinf(d->eps)) {
        I.a = 1.0;
        I.b = 0.0;
    } else {
        I.a = d->eps / (d->eps + d->dt);
        I.b = d->dt / (d->eps + d->dt);
    }
    I.nu = d->dt / I.dx;

    // scratch layout (each piece 256-byte aligned)
    const size_t tab = (size_t)I.nx * 3 * I.nv * sizeof(double);
    size_t off = 0;
    const size_t o_inst = off; off = up256(off + sizeof(prk::Inst));
    const size_t o_state = off; off = up256(off + sizeof(prk::InstState));
    const size_t o_prefix = off; off = up256(off + 2 * sizeof(long long));
    const size_t o_active = off; off = up256(off + sizeof(prk::Active));
    const size_t o_status = off; off = up256(off + sizeof(int));
    const size_t o_sync = off; off = up256(off + 8 + 2 * sizeof(unsigned) * I.n_xt);
    const size_t o_deps = off; off = up256(off + sizeof(int) * prk::MAXDEP * I.n_xt);
    const size_t o_tab0 = off; off = up256(off + tab);
    const size_t o_tab1 = off; off = up256(off + tab);
    const size_t o_part = off; off = up256(off + (size_t)I.nx * I.n_vc * 5 * sizeof(double));
    const size_t o_U = off; off = up256(off + (size_t)5 * I.nx * sizeof(double));
    if (off > NOALLOC_BYTES) {
        char msg[160];
        snprintf(msg, sizeof msg, "pr_fine_step_noalloc: instance needs %zu bytes of scratch, the static array holds %zu",
                 off, NOALLOC_BYTES);
        return reject(msg);
    }

    // the fine kernel's shared memory for this instance against the device's limit
    const int H = d->scheme == PR_MUSCL ? 2 : 1;
    const size_t smem = prk::fine_run_smem(0, 4, I.tx, I.nv, H);
    int dev = 0, smax = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        pr_internal_set_global_error("pr_fine_step_noalloc: no usable CUDA device");
        return PR_ECUDA;
    }
    if (smem > (size_t)smax) {
        char msg[160];
        snprintf(msg, sizeof msg, "pr_fine_step_noalloc: instance needs %zu bytes of shared memory per CTA, the "
                 "device allows %d", smem, smax);
        return reject(msg);
    }

    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) {
        pr_internal_set_global_error("pr_fine_step_noalloc: looking up the static scratch array failed");
        return rc;
    }
    unsigned* sync = reinterpret_cast<unsigned*>(base + o_sync + 8);
    I.g[0] = const_cast<double*>(f_in);
    I.g[1] = f_out;
    I.tab[0] = base + o_tab0;
    I.tab[1] = base + o_tab1;
    I.part = reinterpret_cast<double*>(base + o_part);
    I.Ucur = reinterpret_cast<double*>(base + o_U);
    I.done = sync;
    I.arrive = sync + I.n_xt;
    I.deps = reinterpret_cast<const int*>(base + o_deps);  // unused: one step needs no waits
    prk::InstState st{0, 0, 1.0};                            // f = 1 * f_in + 0 (zero tables)
    long long prefix[2] = {0, (long long)I.n_xt * I.n_vc};
    prk::Active act{0, 1};

    // every call starts from cleared counters, tables and status
    cudaError_t e = cudaMemcpyAsync(base + o_inst, &I, sizeof I, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_state, &st, sizeof st, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_prefix, prefix, sizeof prefix, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_active, &act, sizeof act, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_sync, 0, 8 + 2 * sizeof(unsigned) * I.n_xt, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_tab0, 0, tab, s);
    if (e != cudaSuccess) return cuda_fail(e);

    const prk::Inst* dI = reinterpret_cast<const prk::Inst*>(base + o_inst);
    prk::InstState* dS = reinterpret_cast<prk::InstState*>(base + o_state);
    const prk::Active* dA = reinterpret_cast<const prk::Active*>(base + o_active);
    int* dstatus = reinterpret_cast<int*>(base + o_status);
    int per_sm = 0;
    if (prk::fine_run_occupancy(0, d->scheme, 4, smem, &per_sm) != 0 || per_sm < 1) {
        cudaGetLastError();
        return reject("pr_fine_step_noalloc: the fine kernel cannot be resident with this instance's shared memory");
    }
    long long items = prefix[1];
    int grid = (int)(items < (long long)per_sm * sms ? items : (long long)per_sm * sms);
    e = prk::launch_fine_run(0, d->scheme, 4, dI, dS, reinterpret_cast<const long long*>(base + o_prefix), dA, 1,
                             reinterpret_cast<unsigned long long*>(base + o_sync), dstatus, 0LL, grid, smem, s);
    // f_out now holds f*; apply the implicit relaxation in place: f = a f* + b M
    if (e == cudaSuccess) e = prk::launch_advance(dI, dS, dA, 1, 1, s);
    if (e == cudaSuccess) e = prk::launch_materialize(0, dI, dS, 0, I, f_out, s);
    if (e != cudaSuccess) return cuda_fail(e);
    int status = 0;
    e = cudaMemcpyAsync(&status, dstatus, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (status == PR_ENONPHYS) pr_internal_set_global_error("pr_fine_step_noalloc: a density or temperature became <= 0");
    return status;
}
