// Host runtime of libpr: the C ABI of include/pr.h.  Owns device memory, the
// per-instance descriptors of the fine kernels, the dependency tables of the
// persistent launch, the parareal iterate buffers and the captured CUDA graph
// of one Algorithm 2 iteration (Laidin & Rey, arXiv 2502.02704, Sec. 2.2).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "force_rt.h"
#include "pr.h"
#include "pr_kernels.h"

using prk::Inst;
using prk::InstState;

namespace {

std::atomic<long long> g_launches{0};
std::mutex g_init_mu;
std::string g_init_error;


size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool kernels_prepared = false;
std::mutex g_prep_mu;

int max_optin_smem()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

int sm_count()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v;
}

// Halo tiles of tile xt: tiles holding the cells [c0-H, c1+H) after the
// boundary mapping (periodic wrap, outflow clamp, reflecting mirror).
std::set<int> halo_tiles(int nx, int tx, int bc, int H, int xt)
{
    std::set<int> s;
    int c0 = xt * tx, c1 = std::min(nx, c0 + tx);
    for (int c = c0 - H; c < c1 + H; ++c) {
        int cc = c;
        if (c < 0 || c >= nx) {
            if (bc == PR_BC_PERIODIC) cc = ((c % nx) + nx) % nx;
            else if (bc == PR_BC_OUTFLOW) cc = c < 0 ? 0 : nx - 1;
            else cc = c < 0 ? -1 - c : 2 * nx - 1 - c;
        }
        s.insert(cc / tx);
    }
    return s;
}

}  // namespace

// Dependency lists: halo tiles made symmetric (if A reads B's cells then B
// reads A's), so that waiting on them also orders the ping-pong overwrite.
static bool build_deps(int nx, int tx, int bc, int H, std::vector<int>& deps)
{
    int n_xt = (nx + tx - 1) / tx;
    std::vector<std::set<int>> d(n_xt);
    for (int a = 0; a < n_xt; ++a)
        for (int b : halo_tiles(nx, tx, bc, H, a)) {
            d[a].insert(b);
            d[b].insert(a);
        }
    deps.assign((size_t)n_xt * prk::MAXDEP, -1);
    for (int a = 0; a < n_xt; ++a) {
        if ((int)d[a].size() > prk::MAXDEP) return false;
        int k = 0;
        for (int b : d[a]) deps[(size_t)a * prk::MAXDEP + k++] = b;
    }
    return true;
}

// Raise the dynamic shared-memory limit of every kernel to the device maximum
// once, before any launch or graph capture.
static void prepare_kernels_once()
{
    std::lock_guard<std::mutex> lk(g_prep_mu);
    if (kernels_prepared) return;
    int smax = max_optin_smem();
    prk::prepare_fine_kernels(smax);
    prk::prepare_coarse_kernels(smax);
    kernels_prepared = true;
}

// ------------------------------------------------------------------ batch

struct pr_batch {
    int n = 0, precision = PR_MIXED, scheme = PR_UPWIND, H = 1;
    int vpt = 4;  // velocities per thread of the fine kernel
    int vpt_req = 0;  // 0: 8 when every nv allows it, else 4; 4: always 4 (autotuner's choice)
    size_t es = 4;
    std::vector<pr_instance> desc;
    std::vector<Inst> h;
    std::vector<int> tuned;
    std::vector<InstState> hstate;
    Inst* d_inst = nullptr;
    InstState* d_state = nullptr;
    long long* d_prefix = nullptr;
    prk::Active* d_active = nullptr;
    int* d_deps = nullptr;
    unsigned char* d_sync = nullptr;
    size_t sync_bytes = 0;
    int* d_status = nullptr;
    unsigned char* pool = nullptr;
    double* d_stage = nullptr;
    size_t stage_elems = 0;
    double* h_pinned = nullptr;
    cudaStream_t stream = nullptr;
    int grid = 0;
    long long slots = 0;  // resident CTAs of the fine kernel (SMs x CTAs per SM)
    size_t smem = 0, lift_smem = 0;
    int max_tiles = 1;
    int nx_max = 1;
    int lift_order = 0;  // 0: Maxwellian lift fused into the first step; 1: first-order lift (lift_ce.cu)
    std::string err;
    // kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    double time_ms = 0.0;
    int time_launches = 0;
};

static int bfail(pr_batch* b, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return code;
}

#define BCUDA(b, call)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return bfail((b), PR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static int validate_instance(const pr_instance& d, std::string& why)
{
    char buf[256];
    if (d.nx < 1) why = "nx must be >= 1";
    else if (d.nv < 4 || d.nv % 4) why = "nv must be a positive multiple of 4";
    else if (!(d.x1 > d.x0)) why = "x1 must exceed x0";
    else if (!(d.L > 0)) why = "L must be > 0";
    else if (!(d.eps > 0)) why = "eps must be > 0 (or +inf)";
    else if (!(d.dt > 0) || !std::isfinite(d.dt)) why = "dt must be finite and > 0";
    else if (d.bc < 0 || d.bc > 2) why = "unknown boundary condition";
    else if (d.scheme < 0 || d.scheme > 1) why = "unknown scheme";
    else if (d.scheme == PR_MUSCL && d.bc == PR_BC_REFLECT && d.nx < 2) why = "MUSCL with reflecting walls needs nx >= 2";
    else return PR_OK;
    snprintf(buf, sizeof buf, "%s", why.c_str());
    why = buf;
    return PR_EINVAL;
}


// Fill descriptors for the given tile widths; pool pointers already set.
static int layout_tiles(pr_batch* b, const std::vector<int>& txs, std::vector<long long>& prefix,
                        std::vector<int>& deps_all, std::vector<size_t>& deps_off)
{
    prefix.assign(b->n + 1, 0);
    deps_all.clear();
    deps_off.assign(b->n, 0);
    b->max_tiles = 1;
    for (int i = 0; i < b->n; ++i) {
        Inst& I = b->h[i];
        I.tx = txs[i];
        I.n_xt = (I.nx + I.tx - 1) / I.tx;
        b->max_tiles = std::max(b->max_tiles, I.n_xt);
        b->nx_max = std::max(b->nx_max, I.nx);
        std::vector<int> deps;
        if (!build_deps(I.nx, I.tx, I.bc, b->H, deps))
            return bfail(b, PR_EINVAL, "instance %d: tile dependencies exceed %d", i, prk::MAXDEP);
        deps_off[i] = deps_all.size();
        deps_all.insert(deps_all.end(), deps.begin(), deps.end());
        I.item0 = prefix[i];
        prefix[i + 1] = prefix[i] + (long long)I.n_xt * I.n_vc;
    }
    return PR_OK;
}

static int upload_layout(pr_batch* b, const std::vector<int>& txs)
{
    std::vector<long long> prefix;
    std::vector<int> deps_all;
    std::vector<size_t> deps_off;
    int rc = layout_tiles(b, txs, prefix, deps_all, deps_off);
    if (rc) return rc;
    BCUDA(b, prk::copy_now(b->d_deps, deps_all.data(), deps_all.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    for (int i = 0; i < b->n; ++i) b->h[i].deps = b->d_deps + deps_off[i];
    BCUDA(b, prk::copy_now(b->d_prefix, prefix.data(), prefix.size() * sizeof(long long), cudaMemcpyHostToDevice,
                           b->stream));
    BCUDA(b, prk::copy_now(b->d_inst, b->h.data(), b->h.size() * sizeof(Inst), cudaMemcpyHostToDevice, b->stream));
    // launch geometry
    int maxtx = 1, maxnv = 4;
    for (auto& I : b->h) {
        maxtx = std::max(maxtx, I.tx);
        maxnv = std::max(maxnv, I.nv);
    }
    // eight v_z nodes per thread when every row allows it (float64: the
    // per-column warp sums, FP64 additions, then cover twice the cells; 15 %
    // faster on the 3 x 512 x 32^3 workload)
    bool all8 = true;
    for (auto& I : b->h) all8 = all8 && I.nv % 8 == 0;
    b->vpt = (all8 && b->vpt_req != 4) ? 8 : 4;
    b->smem = prk::fine_run_smem(b->precision == PR_FP64 ? 0 : 1, b->vpt, maxtx, maxnv, b->H);
    b->lift_smem = prk::lift_smem(b->precision == PR_FP64 ? 0 : 1, maxtx, maxnv);
    if ((int)b->smem > max_optin_smem() || (int)b->lift_smem > max_optin_smem())
        return bfail(b, PR_EINVAL, "shared memory per CTA (%zu B) exceeds the device limit", b->smem);
    int per_sm = 0;
    int e = prk::fine_run_occupancy(b->precision == PR_FP64 ? 0 : 1, b->scheme, b->vpt, b->smem, &per_sm);
    if (e != 0 || per_sm < 1) return bfail(b, PR_ECUDA, "fine kernel cannot be resident (occupancy %d)", per_sm);
    long long items = prefix[b->n];
    b->slots = (long long)per_sm * sm_count();
    b->grid = (int)std::min<long long>(b->slots, std::max<long long>(items, 1));
    return PR_OK;
}

// Default tile widths: 32 columns (the fastest width on batches that fill the
// GPU), narrowed to 16 and then 8 while the batch has fewer work items than
// resident CTAs.  A small batch (a few slices of 64-128 cells) is latency
// bound, and more, shorter items per step shorten each step: 8 columns run
// 8 slices of 64 cells 1.6x faster than 32.
static int default_layout(pr_batch* b)
{
    std::vector<int> prev;
    for (int cap : {32, 16, 8}) {
        std::vector<int> txs(b->n);
        for (int i = 0; i < b->n; ++i) txs[i] = std::min(b->h[i].nx, cap);
        int rc = upload_layout(b, txs);
        if (rc) return prev.empty() ? rc : upload_layout(b, prev);
        if (b->grid >= b->slots) break;
        prev = txs;
    }
    return PR_OK;
}

static void free_batch(pr_batch* b)
{
    if (!b) return;
    for (auto e : b->ev_pool) cudaEventDestroy(e);
    for (auto& p : b->ev_pending) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    cudaFree(b->d_inst);
    cudaFree(b->d_state);
    cudaFree(b->d_prefix);
    cudaFree(b->d_active);
    cudaFree(b->d_deps);
    cudaFree(b->d_sync);
    cudaFree(b->d_status);
    cudaFree(b->pool);
    cudaFree(b->d_stage);
    if (b->h_pinned) cudaFreeHost(b->h_pinned);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

static int create_batch(pr_batch** out, const pr_instance* inst, int n, int precision, std::string& err)
{
    *out = nullptr;
    if (!inst || n < 1) {
        err = "need at least one instance";
        return PR_EINVAL;
    }
    if (precision != PR_FP64 && precision != PR_MIXED) {
        err = "precision must be PR_FP64 or PR_MIXED";
        return PR_EINVAL;
    }
    for (int i = 0; i < n; ++i) {
        std::string why;
        if (validate_instance(inst[i], why)) {
            err = "instance " + std::to_string(i) + ": " + why;
            return PR_EINVAL;
        }
        if (inst[i].scheme != inst[0].scheme) {
            err = "all instances of a batch must use the same scheme";
            return PR_EINVAL;
        }
    }
    prepare_kernels_once();
    pr_batch* b = new pr_batch();
    b->n = n;
    b->precision = precision;
    b->es = precision == PR_FP64 ? sizeof(double) : sizeof(float);
    b->scheme = inst[0].scheme;
    b->H = b->scheme == PR_MUSCL ? 2 : 1;
    b->desc.assign(inst, inst + n);
    b->h.resize(n);
    b->tuned.assign(n, 0);
    b->hstate.assign(n, InstState{0, 0, 0.0});
    auto fail = [&](int code, const std::string& m) {
        err = m;
        free_batch(b);
        return code;
    };
    // pool layout
    size_t off = 0, sync_words = 2;  // ticket (u64)
    std::vector<size_t> o_g0(n), o_g1(n), o_t0(n), o_t1(n), o_part(n), o_U(n), o_Uin(n);
    std::vector<size_t> o_done(n), o_arr(n);
    size_t deps_total = 0;
    for (int i = 0; i < n; ++i) {
        const pr_instance& d = inst[i];
        Inst& I = b->h[i];
        memset(&I, 0, sizeof I);
        I.nx = d.nx;
        I.nv = d.nv;
        I.nv3 = d.nv * d.nv * d.nv;
        I.ldv = (int)round_up((size_t)I.nv3, 32);
        I.bc = d.bc;
        I.scheme = d.scheme;
        I.n_vc = (I.nv3 + prk::CHUNK - 1) / prk::CHUNK;
        I.L = d.L;
        I.dv = 2.0 * d.L / d.nv;
        I.dv3 = I.dv * I.dv * I.dv;
        I.dx = (d.x1 - d.x0) / d.nx;
        I.dt = d.dt;
        I.eps = d.eps;
        if (std::isinf(d.eps)) {
            I.a = 1.0;
            I.b = 0.0;
        } else if (precision == PR_MIXED) {
            // the float32 steps scale g by float(a) (Eq. 7: f = a f* + b M):
            // with a = float(eps/(eps+dt)) and b = 1 - a the weights the
            // kernels use sum to 1, so the relaxation keeps the moments (the
            // relaxation rate moves by less than 1e-6 relative)
            I.a = (double)(float)(d.eps / (d.eps + d.dt));
            I.b = 1.0 - I.a;
        } else {
            I.a = d.eps / (d.eps + d.dt);
            I.b = d.dt / (d.eps + d.dt);
        }
        I.nu = d.dt / I.dx;
        size_t gsz = (size_t)I.nx * I.ldv * b->es, tsz = (size_t)I.nx * 3 * I.nv * b->es;
        o_g0[i] = off; off = round_up(off + gsz, 256);
        o_g1[i] = off; off = round_up(off + gsz, 256);
        o_t0[i] = off; off = round_up(off + tsz, 256);
        o_t1[i] = off; off = round_up(off + tsz, 256);
        o_part[i] = off; off = round_up(off + (size_t)I.nx * I.n_vc * 5 * sizeof(double), 256);
        o_U[i] = off; off = round_up(off + (size_t)5 * I.nx * sizeof(double), 256);
        o_Uin[i] = off; off = round_up(off + (size_t)5 * I.nx * sizeof(double), 256);
        int max_xt = (I.nx + 7) / 8;  // room for the smallest tile width (8, or nx below 8)
        o_done[i] = sync_words; sync_words += max_xt;
        o_arr[i] = sync_words; sync_words += max_xt;
        deps_total += (size_t)max_xt * prk::MAXDEP;
        b->stage_elems = std::max(b->stage_elems, (size_t)I.nx * I.nv3);
    }
    cudaError_t e = cudaMalloc(&b->pool, std::max<size_t>(off, 256));
    if (e != cudaSuccess) return fail(PR_ENOMEM, std::string("device pool of ") + std::to_string(off) + " bytes: " + cudaGetErrorString(e));
    b->sync_bytes = sync_words * 4;
    if (cudaMalloc(&b->d_sync, b->sync_bytes) != cudaSuccess || cudaMalloc(&b->d_status, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_inst, sizeof(Inst) * n) != cudaSuccess ||
        cudaMalloc(&b->d_state, sizeof(InstState) * n) != cudaSuccess ||
        cudaMalloc(&b->d_prefix, sizeof(long long) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&b->d_active, sizeof(prk::Active)) != cudaSuccess ||
        cudaMalloc(&b->d_deps, sizeof(int) * std::max<size_t>(deps_total, 1)) != cudaSuccess ||
        cudaMallocHost(&b->h_pinned, sizeof(double) * 64) != cudaSuccess)
        return fail(PR_ENOMEM, "small device buffers");
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(PR_ECUDA, "stream");
    cudaMemset(b->pool, 0, off);
    cudaMemset(b->d_sync, 0, b->sync_bytes);
    cudaMemset(b->d_status, 0, sizeof(int));
    unsigned* words = reinterpret_cast<unsigned*>(b->d_sync);
    for (int i = 0; i < n; ++i) {
        Inst& I = b->h[i];
        I.g[0] = b->pool + o_g0[i];
        I.g[1] = b->pool + o_g1[i];
        I.tab[0] = b->pool + o_t0[i];
        I.tab[1] = b->pool + o_t1[i];
        I.part = reinterpret_cast<double*>(b->pool + o_part[i]);
        I.Ucur = reinterpret_cast<double*>(b->pool + o_U[i]);
        I.Uin = reinterpret_cast<const double*>(b->pool + o_Uin[i]);
        I.Uout = nullptr;
        I.done = words + o_done[i];
        I.arrive = words + o_arr[i];
    }
    int rc = default_layout(b);
    if (rc) return fail(rc, b->err);
    prk::Active all{0, n};
    if (prk::copy_now(b->d_active, &all, sizeof all, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        prk::copy_now(b->d_state, b->hstate.data(), sizeof(InstState) * n, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
        return fail(PR_ECUDA, "initial uploads");
    *out = b;
    return PR_OK;
}

static cudaStream_t pick(pr_batch* b, void* s) { return s ? reinterpret_cast<cudaStream_t>(s) : b->stream; }

// Read and clear the device status word (after a synchronisation).
static int take_status(pr_batch* b, cudaStream_t s)
{
    BCUDA(b, cudaStreamSynchronize(s));
    int st = 0;
    BCUDA(b, cudaMemcpy(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        prk::zero_now(b->d_status, sizeof(int), s);
        prk::zero_now(b->d_sync, b->sync_bytes, s);
        if (st == PR_ETIMEOUT) return bfail(b, PR_ETIMEOUT, "a device-side wait timed out; the launch was aborted");
        if (st == PR_ENONPHYS) return bfail(b, PR_ENONPHYS, "non-positive density or temperature (or NaN) encountered");
        return bfail(b, st, "device status %d", st);
    }
    return PR_OK;
}

static cudaEvent_t get_event(pr_batch* b)
{
    if (!b->ev_pool.empty()) {
        cudaEvent_t e = b->ev_pool.back();
        b->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static void fold_events(pr_batch* b)
{
    for (auto& p : b->ev_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.second) == cudaSuccess && cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) {
            b->time_ms += ms;
            b->time_launches += 1;
        }
        b->ev_pool.push_back(p.first);
        b->ev_pool.push_back(p.second);
    }
    b->ev_pending.clear();
}

// Enqueue one persistent run over the active range already set on the device.
static int enqueue_run(pr_batch* b, int nsteps, int project_out, cudaStream_t s, bool count_timing,
                       long long wait_ns = prk::WAIT_LIMIT_NS, int poison = 0)
{
    (void)project_out;
    BCUDA(b, cudaMemsetAsync(b->d_sync, 0, b->sync_bytes, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (b->timing && count_timing) {
        if (b->ev_pending.size() > 2048) fold_events(b);
        e0 = get_event(b);
        e1 = get_event(b);
        cudaEventRecord(e0, s);
    }
    BCUDA(b, prk::launch_fine_run(b->precision == PR_FP64 ? 0 : 1, b->scheme, b->vpt, b->d_inst, b->d_state, b->d_prefix,
                                  b->d_active, nsteps, reinterpret_cast<unsigned long long*>(b->d_sync),
                                  b->d_status, nsteps > 1 ? wait_ns : 0, b->grid, b->smem, s, poison));
    if (e1) {
        cudaEventRecord(e1, s);
        b->ev_pending.push_back({e0, e1});
    }
    BCUDA(b, prk::launch_advance(b->d_inst, b->d_state, b->d_active, nsteps, b->n, s));
    g_launches += 2;
    return PR_OK;
}

static void prim_to_cons_host(int nx, const double* U, double* V)
{
    for (int i = 0; i < nx; ++i) {
        double rho = U[i], ux = U[nx + i], uy = U[2 * nx + i], uz = U[3 * nx + i], th = U[4 * nx + i];
        V[i] = rho;
        V[nx + i] = rho * ux;
        V[2 * nx + i] = rho * uy;
        V[3 * nx + i] = rho * uz;
        V[4 * nx + i] = 0.5 * rho * (ux * ux + uy * uy + uz * uz) + 1.5 * rho * th;
    }
}

static void cons_to_prim_host(int nx, const double* V, double* U)
{
    for (int i = 0; i < nx; ++i) {
        double rho = V[i];
        double ux = V[nx + i] / rho, uy = V[2 * nx + i] / rho, uz = V[3 * nx + i] / rho;
        double th = (2.0 * V[4 * nx + i] / rho - (ux * ux + uy * uy + uz * uz)) / 3.0;
        U[i] = rho;
        U[nx + i] = ux;
        U[2 * nx + i] = uy;
        U[3 * nx + i] = uz;
        U[4 * nx + i] = th;
    }
}

static int check_prim(const double* U, int nx)
{
    for (int i = 0; i < nx; ++i) {
        if (!(U[i] > 0.0) || !(U[4 * nx + i] > 0.0)) return PR_ENONPHYS;
        for (int q = 0; q < 5; ++q)
            if (!std::isfinite(U[q * nx + i])) return PR_ENONPHYS;
    }
    return PR_OK;
}

// Conserved state: every component finite, rho > 0 and a positive temperature.
static int check_cons(const double* V, int nx)
{
    for (int i = 0; i < nx; ++i) {
        for (int q = 0; q < 5; ++q)
            if (!std::isfinite(V[q * nx + i])) return PR_ENONPHYS;
        const double rho = V[i];
        if (!(rho > 0.0)) return PR_ENONPHYS;
        const double m2 = V[nx + i] * V[nx + i] + V[2 * nx + i] * V[2 * nx + i] + V[3 * nx + i] * V[3 * nx + i];
        if (!(2.0 * V[4 * nx + i] - m2 / rho > 0.0)) return PR_ENONPHYS;
    }
    return PR_OK;
}

static int lift_instances(pr_batch* b, int begin, int end, cudaStream_t s)
{
    prk::Active a{begin, end};
    BCUDA(b, cudaMemcpyAsync(b->d_active, &a, sizeof a, cudaMemcpyHostToDevice, s));
    if (b->lift_order == 1) {
        BCUDA(b, prk::launch_lift_ce(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->d_state, b->d_active, b->nx_max,
                                     end - begin, 1, b->d_status, s));
        g_launches += 2;
    } else {
        BCUDA(b, prk::launch_lift(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->d_state, b->d_active, b->max_tiles,
                                  end - begin, b->lift_smem, b->d_status, s));
        g_launches += 1;
    }
    prk::Active all{0, b->n};
    BCUDA(b, cudaMemcpyAsync(b->d_active, &all, sizeof all, cudaMemcpyHostToDevice, s));
    return PR_OK;
}

int pr_fine_dt_stab(const pr_instance* d, double cfl, double* dt)
{
    if (!d || !dt) return PR_EINVAL;
    if (d->nx < 1 || d->nv < 1 || !(d->x1 > d->x0) || !std::isfinite(d->x1 - d->x0) || !(d->L > 0) ||
        !std::isfinite(d->L) || !(cfl > 0) || !std::isfinite(cfl))
        return PR_EINVAL;
    const double dx = (d->x1 - d->x0) / d->nx, dv = 2.0 * d->L / d->nv;
    *dt = cfl * dx / (d->L - 0.5 * dv);
    return PR_OK;
}

// Message for pr_batch_last_error(NULL) from entry points that own no object.
void pr_internal_count_launches(long long n) { g_launches += n; }

void pr_internal_set_global_error(const char* msg)
{
    std::lock_guard<std::mutex> lk(g_init_mu);
    g_init_error = msg ? msg : "";
}

extern "C" {

int pr_batch_create(pr_batch** out, const pr_instance* inst, int n, int precision)
{
    if (!out) return PR_EINVAL;
    std::string err;
    int rc = create_batch(out, inst, n, precision, err);
    if (rc) {
        std::lock_guard<std::mutex> lk(g_init_mu);
        g_init_error = err;
    }
    return rc;
}

int pr_batch_destroy(pr_batch* b)
{
    if (b) {
        cudaStreamSynchronize(b->stream);
        free_batch(b);
    }
    return PR_OK;
}

const char* pr_batch_last_error(const pr_batch* b)
{
    if (!b) return g_init_error.c_str();
    return b->err.c_str();
}

int pr_batch_set_initial_device(pr_batch* b, int i, const double* U_dev, int kind, void* stream)
{
    if (!b) return PR_EINVAL;
    if (i < 0 || i >= b->n || !U_dev) return bfail(b, PR_EINVAL, "bad instance index or null state");
    if (kind != PR_CONSERVED)
        return bfail(b, PR_EINVAL, "device lifting takes conserved states (PR_CONSERVED)");
    cudaStream_t s = pick(b, stream);
    const Inst& I = b->h[i];
    BCUDA(b, cudaMemcpyAsync(const_cast<double*>(I.Uin), U_dev, sizeof(double) * 5 * I.nx, cudaMemcpyDeviceToDevice, s));
    return lift_instances(b, i, i + 1, s);
}

int pr_batch_set_initial(pr_batch* b, int i, const double* U, int kind)
{
    if (!b) return PR_EINVAL;
    if (i < 0 || i >= b->n || !U) return bfail(b, PR_EINVAL, "bad instance index or null state");
    if (kind != PR_PRIMITIVE && kind != PR_CONSERVED) return bfail(b, PR_EINVAL, "kind must be primitive or conserved");
    const Inst& I = b->h[i];
    std::vector<double> V(5 * I.nx), P(5 * I.nx);
    if (kind == PR_PRIMITIVE) {
        memcpy(P.data(), U, sizeof(double) * 5 * I.nx);
        prim_to_cons_host(I.nx, U, V.data());
    } else {
        memcpy(V.data(), U, sizeof(double) * 5 * I.nx);
        cons_to_prim_host(I.nx, U, P.data());
    }
    if (check_prim(P.data(), I.nx)) return bfail(b, PR_ENONPHYS, "initial state has rho <= 0 or theta <= 0");
    BCUDA(b, cudaMemcpyAsync(const_cast<double*>(I.Uin), V.data(), sizeof(double) * 5 * I.nx, cudaMemcpyHostToDevice,
                             b->stream));
    return lift_instances(b, i, i + 1, b->stream);
}

int pr_batch_set_f(pr_batch* b, int i, const double* f)
{
    if (!b) return PR_EINVAL;
    if (i < 0 || i >= b->n || !f) return bfail(b, PR_EINVAL, "bad instance index or null f");
    const Inst& I = b->h[i];
    size_t cnt = (size_t)I.nx * I.nv3;
    if (!b->d_stage) BCUDA(b, cudaMalloc(&b->d_stage, sizeof(double) * b->stage_elems));
    BCUDA(b, cudaMemcpyAsync(b->d_stage, f, sizeof(double) * cnt, cudaMemcpyHostToDevice, b->stream));
    BCUDA(b, prk::launch_set_f(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->d_state, i, I, b->d_stage, b->stream));
    g_launches += 2;
    return take_status(b, b->stream);
}

int pr_batch_run(pr_batch* b, int nsteps, void* stream)
{
    if (!b) return PR_EINVAL;
    if (nsteps < 0) return bfail(b, PR_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0) return PR_OK;
    return enqueue_run(b, nsteps, 0, pick(b, stream), true);
}

int pr_batch_propagate(pr_batch* b, const double* U_dev, int nsteps, void* stream)
{
    if (!b) return PR_EINVAL;
    if (nsteps < 1) return bfail(b, PR_EINVAL, "nsteps must be >= 1");
    cudaStream_t s = pick(b, stream);
    if (U_dev) {  // the lift sources: the instances' conserved states one after another
        size_t off = 0;
        for (const Inst& I : b->h) {
            BCUDA(b, cudaMemcpyAsync(const_cast<double*>(I.Uin), U_dev + off, sizeof(double) * 5 * I.nx,
                                     cudaMemcpyDeviceToDevice, s));
            off += 5 * (size_t)I.nx;
        }
    }
    // cluster-resident when every instance has one shape that fits a
    // cluster (the rule of the parareal fine phase)
    const Inst& I0 = b->h[0];
    bool same = true;
    for (const Inst& I : b->h) same = same && I.nx == I0.nx && I.nv == I0.nv;
    int C = 0, w = 0;
    size_t sm = 0;
    const bool fits = same && b->precision == PR_MIXED && b->lift_order == 0 &&
                      prk::fine_cluster_plan(I0.nx, I0.nv, max_optin_smem(), &C, &w, &sm);
    const int resident = fits ? prk::fine_cluster_resident(b->scheme, I0.nv, C, sm) : 0;
    if (fits && resident > 0 && b->n <= 2 * resident) {
        const prk::Active all{0, b->n};
        BCUDA(b, cudaMemcpyAsync(b->d_active, &all, sizeof all, cudaMemcpyHostToDevice, s));
        BCUDA(b, prk::launch_fine_cluster(b->scheme, I0.nv, b->d_inst, b->d_active, b->n, nsteps, C, w, sm,
                                          b->d_status, s));
        g_launches += 1;
        return PR_OK;
    }
    const int rc = lift_instances(b, 0, b->n, s);
    if (rc) return rc;
    return enqueue_run(b, nsteps, 0, s, true);
}

int pr_batch_run_range(pr_batch* b, int first, int count, int nsteps, void* stream)
{
    if (!b) return PR_EINVAL;
    if (first < 0 || count < 1 || first > b->n - count || nsteps < 0)
        return bfail(b, PR_EINVAL, "instances [first, first + count) must lie in the batch and nsteps >= 0");
    if (nsteps == 0) return PR_OK;
    cudaStream_t s = pick(b, stream);
    if (count == b->n) return enqueue_run(b, nsteps, 0, s, true);
    prk::Active a{first, first + count};
    BCUDA(b, cudaMemcpyAsync(b->d_active, &a, sizeof a, cudaMemcpyHostToDevice, s));
    const int rc = enqueue_run(b, nsteps, 0, s, true);
    prk::Active all{0, b->n};
    BCUDA(b, cudaMemcpyAsync(b->d_active, &all, sizeof all, cudaMemcpyHostToDevice, s));
    return rc;
}

int pr_batch_inject_wait_timeout(pr_batch* b, int nsteps, int wait_ms)
{
    if (!b) return PR_EINVAL;
    if (nsteps < 2 || wait_ms < 1) return bfail(b, PR_EINVAL, "needs nsteps >= 2 and wait_ms >= 1");
    BCUDA(b, cudaStreamSynchronize(b->stream));
    int rc = enqueue_run(b, nsteps, 0, b->stream, false, (long long)wait_ms * 1000000LL, 1);
    if (rc) return rc;
    return take_status(b, b->stream);
}

int pr_batch_set_lift_order(pr_batch* b, int order)
{
    if (!b) return PR_EINVAL;
    if (order != 0 && order != 1) return bfail(b, PR_EINVAL, "lift order must be 0 or 1");
    if (order == 1)
        for (const pr_instance& d : b->desc)
            if (!std::isfinite(d.eps)) return bfail(b, PR_EINVAL, "the first-order lift needs a finite eps");
    b->lift_order = order;
    return PR_OK;
}

int pr_batch_sync(pr_batch* b)
{
    if (!b) return PR_EINVAL;
    return take_status(b, b->stream);
}

int pr_batch_moments_device(pr_batch* b, int i, double* out_dev, void* stream)
{
    if (!b) return PR_EINVAL;
    if (i < 0 || i >= b->n || !out_dev) return bfail(b, PR_EINVAL, "bad instance index or null output");
    const Inst& I = b->h[i];
    BCUDA(b, cudaMemcpyAsync(out_dev, I.Ucur, sizeof(double) * 5 * I.nx, cudaMemcpyDeviceToDevice, pick(b, stream)));
    return PR_OK;
}

int pr_batch_moments(pr_batch* b, int i, int kind, double* out)
{
    if (!b) return PR_EINVAL;
    if (i < 0 || i >= b->n || !out) return bfail(b, PR_EINVAL, "bad instance index or null output");
    if (kind != PR_PRIMITIVE && kind != PR_CONSERVED) return bfail(b, PR_EINVAL, "kind must be primitive or conserved");
    const Inst& I = b->h[i];
    std::vector<double> V(5 * I.nx);
    BCUDA(b, cudaMemcpyAsync(V.data(), I.Ucur, sizeof(double) * 5 * I.nx, cudaMemcpyDeviceToHost, b->stream));
    int rc = take_status(b, b->stream);
    if (kind == PR_CONSERVED) memcpy(out, V.data(), sizeof(double) * 5 * I.nx);
    else cons_to_prim_host(I.nx, V.data(), out);
    return rc;
}

int pr_batch_get_f(pr_batch* b, int i, double* out)
{
    if (!b) return PR_EINVAL;
    if (i < 0 || i >= b->n || !out) return bfail(b, PR_EINVAL, "bad instance index or null output");
    const Inst& I = b->h[i];
    size_t cnt = (size_t)I.nx * I.nv3;
    if (!b->d_stage) BCUDA(b, cudaMalloc(&b->d_stage, sizeof(double) * b->stage_elems));
    BCUDA(b, prk::launch_materialize(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->d_state, i, I, b->d_stage, b->stream));
    g_launches += 1;
    BCUDA(b, cudaMemcpyAsync(out, b->d_stage, sizeof(double) * cnt, cudaMemcpyDeviceToHost, b->stream));
    return take_status(b, b->stream);
}

int pr_batch_tile(const pr_batch* b, int i, int* tx, int* tuned)
{
    if (!b || i < 0 || i >= b->n) return PR_EINVAL;
    if (tx) *tx = b->h[i].tx;
    if (tuned) *tuned = b->tuned[i];
    return PR_OK;
}

int pr_batch_vpt(const pr_batch* b, int* vpt)
{
    if (!b || !vpt) return PR_EINVAL;
    *vpt = b->vpt;
    return PR_OK;
}

int pr_batch_set_tile(pr_batch* b, int tx)
{
    if (!b) return PR_EINVAL;
    if (tx < 1 || tx > prk::MAX_TX) return bfail(b, PR_EINVAL, "tile width must be in 1..%d", prk::MAX_TX);
    BCUDA(b, cudaStreamSynchronize(b->stream));
    std::vector<int> txs(b->n);
    for (int i = 0; i < b->n; ++i) {
        // the dependency tables were sized for tiles of at least 8 cells (or the default width)
        int t = std::min(tx, b->h[i].nx);
        txs[i] = std::max(t, std::min(8, b->h[i].nx));
        b->tuned[i] = 0;
    }
    return upload_layout(b, txs);
}

int pr_batch_kernel_time(pr_batch* b, double* avg_ms, int* launches, int reset)
{
    if (!b) return PR_EINVAL;
    b->timing = true;
    fold_events(b);
    if (avg_ms) *avg_ms = b->time_launches ? b->time_ms / b->time_launches : 0.0;
    if (launches) *launches = b->time_launches;
    if (reset) {
        b->time_ms = 0.0;
        b->time_launches = 0;
    }
    return PR_OK;
}

long long pr_kernel_launches(int reset)
{
    long long v = g_launches.load();
    if (reset) g_launches = 0;
    return v;
}

}  // extern "C"

// ------------------------------------------------------------------ adjoint

// Checkpointed reverse sweep of the float64 upwind fine run (see adjoint.cu).
extern "C" int pr_batch_adjoint(pr_batch* b, int i, int nsteps, int ckpt, const double* lamV, double* dU0,
                                double* dlogeps)
{
    if (!b) return PR_EINVAL;
    if (i < 0 || i >= b->n || !lamV || !dU0 || nsteps < 0 || ckpt < 1)
        return bfail(b, PR_EINVAL, "bad instance, buffers, step count or checkpoint interval");
    if (b->precision != PR_FP64 || b->scheme != PR_UPWIND)
        return bfail(b, PR_EINVAL, "the adjoint covers the float64 upwind scheme");
    const Inst I = b->h[i];
    if (I.bc == PR_BC_REFLECT) return bfail(b, PR_EINVAL, "the adjoint covers periodic and outflow boundaries");
    cudaStream_t s = b->stream;
    const size_t st = (size_t)I.nx * I.ldv, sv = (size_t)I.nx * I.nv3, m5 = (size_t)5 * I.nx;
    const int nck = nsteps > 0 ? (nsteps + ckpt - 1) / ckpt : 0;
    const int seg = std::min(ckpt, std::max(nsteps, 1));
    // work: checkpoints, segment states and their moment sums, two adjoint
    // buffers, small vectors
    size_t need =
        ((size_t)nck * sv + (size_t)seg * st + (size_t)seg * m5 + 2 * sv + 5 * I.nx + I.nx + 2 * m5) * sizeof(double);
    double* w = nullptr;
    if (cudaMalloc(&w, need) != cudaSuccess) return bfail(b, PR_ENOMEM, "adjoint work buffers (%zu bytes)", need);
    double* ck = w;
    double* sg = ck + (size_t)nck * sv;
    double* smm = sg + (size_t)seg * st;
    double* la = smm + (size_t)seg * m5;
    double* lb = la + sv;
    double* coef = lb + sv;
    double* eps = coef + 5 * I.nx;
    double* dv = eps + I.nx;   // lamV on the device
    double* du = dv + m5;      // dU0 on the device
    int rc = PR_OK;
    // one fine step of instance i alone (a batch of one needs no change of
    // the active range)
    const bool solo = b->n == 1;
    auto runk = [&](int k) -> int {
        if (solo) return enqueue_run(b, k, 0, s, false);
        prk::Active a{i, i + 1};
        BCUDA(b, cudaMemcpyAsync(b->d_active, &a, sizeof a, cudaMemcpyHostToDevice, s));
        int r = enqueue_run(b, k, 0, s, false);
        prk::Active all{0, b->n};
        BCUDA(b, cudaMemcpyAsync(b->d_active, &all, sizeof all, cudaMemcpyHostToDevice, s));
        return r;
    };
    do {
        // forward from the lifted state, storing f every ckpt steps: one
        // persistent launch per segment (the same bits as single steps)
        if ((rc = lift_instances(b, i, i + 1, s))) break;
        for (int t = 0; t < nsteps && !rc; t += ckpt) {
            if (prk::launch_materialize(0, b->d_inst, b->d_state, i, I, ck + (size_t)(t / ckpt) * sv, s) != cudaSuccess) {
                rc = bfail(b, PR_ECUDA, "checkpoint");
                break;
            }
            g_launches += 1;
            rc = runk(std::min(ckpt, nsteps - t));
        }
        if (rc) break;
        if (cudaMemcpyAsync(dv, lamV, sizeof(double) * m5, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(eps, 0, sizeof(double) * I.nx, s) != cudaSuccess ||
            prk::adj_seed(I, dv, la, s) != cudaSuccess) {
            rc = bfail(b, PR_ECUDA, "adjoint seed");
            break;
        }
        g_launches += 1;
        for (int k = nck - 1; k >= 0 && !rc; --k) {
            const int s0 = k * ckpt, s1 = std::min(s0 + ckpt, nsteps);
            if (k == 0) rc = lift_instances(b, i, i + 1, s);
            else if (prk::launch_set_f(0, b->d_inst, b->d_state, i, I, ck + (size_t)k * sv, s) != cudaSuccess)
                rc = bfail(b, PR_ECUDA, "reload checkpoint");
            else g_launches += 2;
            if (rc) break;
            // the segment recomputed in one persistent launch that records each
            // step's f* and its moment sums (the same bits as single steps)
            Inst tr = b->h[i];
            tr.trace = sg;
            tr.trace_m = smm;
            BCUDA(b, cudaMemcpyAsync(b->d_inst + i, &tr, sizeof(Inst), cudaMemcpyHostToDevice, s));
            rc = runk(s1 - s0);
            BCUDA(b, cudaMemcpyAsync(b->d_inst + i, &b->h[i], sizeof(Inst), cudaMemcpyHostToDevice, s));
            for (int t = s1 - 1; t >= s0 && !rc; --t) {
                if (prk::adj_step(I, la, sg + (size_t)(t - s0) * st, smm + (size_t)(t - s0) * m5, coef, eps, lb, s) !=
                    cudaSuccess)
                    rc = bfail(b, PR_ECUDA, "adjoint step");
                g_launches += 2;
                std::swap(la, lb);
            }
        }
        if (rc) break;
        if (prk::adj_lift(I, la, I.Uin, du, s) != cudaSuccess) {
            rc = bfail(b, PR_ECUDA, "lift adjoint");
            break;
        }
        g_launches += 1;
        std::vector<double> e(I.nx);
        if (cudaMemcpyAsync(dU0, du, sizeof(double) * m5, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(e.data(), eps, sizeof(double) * I.nx, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            rc = bfail(b, PR_ECUDA, "adjoint readback");
            break;
        }
        rc = take_status(b, s);
        double tot = 0.0;
        for (double x : e) tot += x;
        if (dlogeps) *dlogeps = tot;
    } while (false);
    cudaStreamSynchronize(s);
    cudaFree(w);
    return rc;
}

// ------------------------------------------------------------------ autotuner

// Candidate tile widths are timed with CUDA events on a copy of the current
// state (saved and restored), one persistent launch of 16 steps each after one
// untimed launch; the fastest width is kept for all instances.
extern "C" int pr_batch_autotune(pr_batch* b)
{
    if (!b) return PR_EINVAL;
    BCUDA(b, cudaStreamSynchronize(b->stream));
    // save state of every instance (g of the current buffer, tables, Ucur, InstState)
    std::vector<InstState> st(b->n);
    BCUDA(b, cudaMemcpy(st.data(), b->d_state, sizeof(InstState) * b->n, cudaMemcpyDeviceToHost));
    size_t total = 0;
    for (auto& I : b->h) total += (size_t)I.nx * I.ldv * b->es * 2 + (size_t)I.nx * 3 * I.nv * b->es * 2;
    void* save = nullptr;
    if (cudaMalloc(&save, total) != cudaSuccess) return bfail(b, PR_ENOMEM, "autotune needs %zu bytes of scratch", total);
    auto copy_all = [&](bool to_save) {
        size_t off = 0;
        for (auto& I : b->h) {
            size_t gs = (size_t)I.nx * I.ldv * b->es, ts = (size_t)I.nx * 3 * I.nv * b->es;
            void* ptrs[4] = {I.g[0], I.g[1], I.tab[0], I.tab[1]};
            size_t sz[4] = {gs, gs, ts, ts};
            for (int k = 0; k < 4; ++k) {
                char* sv = static_cast<char*>(save) + off;
                if (to_save) prk::copy_now(sv, ptrs[k], sz[k], cudaMemcpyDeviceToDevice, b->stream);
                else prk::copy_now(ptrs[k], sv, sz[k], cudaMemcpyDeviceToDevice, b->stream);
                off += sz[k];
            }
        }
    };
    copy_all(true);
    // candidates: tile widths x velocities per thread (8 and 4 where every
    // nv allows 8, else 4 only)
    const int cands[4] = {8, 16, 32, 64};
    bool all8 = true;
    for (auto& I : b->h) all8 = all8 && I.nv % 8 == 0;
    const int nvpt = all8 ? 2 : 1, vpts[2] = {0, 4};
    double best_ms = 1e300;
    int best_c = -1, best_v = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int steps = 16;  // long enough for the steady state of the persistent launch
    int rc = PR_OK;
    for (int cv = 0; cv < 4 * nvpt && rc == PR_OK; ++cv) {
        const int ci = cv % 4;
        b->vpt_req = vpts[cv / 4];
        std::vector<int> txs(b->n);
        for (int i = 0; i < b->n; ++i) txs[i] = std::min(cands[ci], b->h[i].nx);
        rc = upload_layout(b, txs);
        if (rc) break;
        double ms_sum = 0;
        for (int rep = 0; rep < 2; ++rep) {
            copy_all(false);
            prk::copy_now(b->d_state, st.data(), sizeof(InstState) * b->n, cudaMemcpyHostToDevice, b->stream);
            cudaEventRecord(e0, b->stream);
            rc = enqueue_run(b, steps, 0, b->stream, false);
            cudaEventRecord(e1, b->stream);
            if (rc) break;
            rc = take_status(b, b->stream);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 1) ms_sum += ms;
        }
        if (rc == PR_OK && ms_sum < best_ms) {
            best_ms = ms_sum;
            best_c = ci;
            best_v = b->vpt_req;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc2;
    b->vpt_req = best_c >= 0 ? best_v : 0;
    if (best_c >= 0) {
        std::vector<int> txs(b->n);
        for (int i = 0; i < b->n; ++i) txs[i] = std::min(cands[best_c], b->h[i].nx);
        rc2 = upload_layout(b, txs);
    } else {
        rc2 = default_layout(b);
    }
    copy_all(false);
    prk::copy_now(b->d_state, st.data(), sizeof(InstState) * b->n, cudaMemcpyHostToDevice, b->stream);
    cudaFree(save);
    if (rc == PR_OK && rc2 == PR_OK && best_c >= 0)
        for (int i = 0; i < b->n; ++i) b->tuned[i] = 1;
    BCUDA(b, cudaDeviceSynchronize());
    return rc ? rc : rc2;
}

// ------------------------------------------------------------------ parareal

struct pr_ctx {
    pr_grid g;
    pr_velocity v;
    double eps = 0;
    pr_time t;
    int nx = 0, N = 0, nf = 0, n_res = 0;
    double dtf = 0, dT = 0;
    pr_batch* fine = nullptr;   // E = 0 fine propagator (pr_init)
    pr_force* ff = nullptr;     // force-path fine propagator (pr_init_force)
    double *dU = nullptr, *dPFL = nullptr, *dGs = nullptr, *derr = nullptr, *dwork = nullptr, *dtmp = nullptr;
    int* dk = nullptr;
    int* dstatus = nullptr;
    double* h_pinned = nullptr;
    prk::CoarseParams cp;
    int k = 0;
    bool initialized = false;
    std::vector<int> live;  // slice whose live f each resident instance holds (0 = none)
    int fpath_req = PR_FINE_AUTO;
    bool use_cluster = false;  // fine phase on the cluster-resident kernel
    int cl_C = 0, cl_w = 0;    // its CTAs per cluster and x cells per CTA
    size_t cl_smem = 0;
    int cl_resident = 0;       // clusters of that shape the device runs at once
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool descs_dirty = false;
    std::string err;
};

static int cfail(pr_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CCUDA(c, call)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return cfail((c), PR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static void free_ctx(pr_ctx* c)
{
    if (!c) return;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->fine) free_batch(c->fine);
    if (c->ff) prf::destroy(c->ff);
    cudaFree(c->dU);
    cudaFree(c->dPFL);
    cudaFree(c->dGs);
    cudaFree(c->derr);
    cudaFree(c->dwork);
    cudaFree(c->dtmp);
    cudaFree(c->dk);
    cudaFree(c->dstatus);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    delete c;
}

static cudaStream_t ctx_stream(const pr_ctx* c) { return c->ff ? c->ff->stream : c->fine->stream; }

// Pinned host memory of a problem: the iteration errors [N + 2], a staging
// copy of the conserved initial state [5][nx], then two status words.
static size_t pinned_doubles(const pr_ctx* c) { return (size_t)(c->N + 2) + 5 * (size_t)c->nx + 1; }
static double* pinned_state(pr_ctx* c) { return c->h_pinned + (c->N + 2); }
static int* pinned_status(pr_ctx* c) { return reinterpret_cast<int*>(c->h_pinned + (c->N + 2) + 5 * (size_t)c->nx); }

// Point resident instance b at slice n (lift source U^{n-1}, projection PFL^n).
static void bind_slice(pr_ctx* c, int b, int n)
{
    const double* uin = c->dU + (size_t)(n - 1) * 5 * c->nx;
    double* uout = c->dPFL + (size_t)n * 5 * c->nx;
    if (c->ff) {
        prf::bind(c->ff, b, uin, uout);
        return;
    }
    Inst& I = c->fine->h[b];
    I.Uin = uin;
    I.Uout = uout;
}

// The fine phase of an iteration runs on the cluster-resident kernel when
// the slices are mixed precision with the Maxwellian lifting, their shape has
// an instantiation and fits one cluster's shared memory, and the resident
// slices' clusters run in at most two waves (clusters that finish free their
// SMs for the next); else on the tiled persistent kernel, which a batch that
// fills the GPU runs near the HBM roofline.
static int choose_fine_path(pr_ctx* c)
{
    c->use_cluster = false;
    if (c->ff) return PR_OK;
    pr_batch* b = c->fine;
    int C = 0, w = 0;
    size_t sm = 0;
    const bool fits = b->precision == PR_MIXED && b->lift_order == 0 &&
                      prk::fine_cluster_plan(c->nx, c->v.nv, max_optin_smem(), &C, &w, &sm);
    const int resident = fits ? prk::fine_cluster_resident(b->scheme, c->v.nv, C, sm) : 0;
    if (c->fpath_req == PR_FINE_CLUSTER) {
        if (!fits || resident < 1)
            return cfail(c, PR_EINVAL, "the cluster-resident fine run needs mixed precision, the Maxwellian lifting, "
                                       "nv = 8 or 16 and a slice that fits a cluster's shared memory");
        c->use_cluster = true;
    } else if (c->fpath_req == PR_FINE_AUTO) {
        c->use_cluster = fits && resident > 0 && c->n_res <= 2 * resident;
    }
    c->cl_C = fits ? C : 0;
    c->cl_w = fits ? w : 0;
    c->cl_smem = sm;
    c->cl_resident = resident;
    return PR_OK;
}

static int take_ctx_status(pr_ctx* c)
{
    if (!c->ff) {  // both status words in one round trip; the slow path below on an error
        int* hs = pinned_status(c);
        cudaStream_t s = ctx_stream(c);
        CCUDA(c, cudaMemcpyAsync(hs, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
        CCUDA(c, cudaMemcpyAsync(hs + 1, c->fine->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        CCUDA(c, cudaStreamSynchronize(s));
        if (hs[0] == 0 && hs[1] == 0) return PR_OK;
    }
    CCUDA(c, cudaStreamSynchronize(ctx_stream(c)));
    int st = 0;
    CCUDA(c, cudaMemcpy(&st, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost));
    int rc = c->ff ? prf::take_status(c->ff) : take_status(c->fine, c->fine->stream);
    if (st != 0) {
        prk::zero_now(c->dstatus, sizeof(int), ctx_stream(c));
        return cfail(c, st, st == PR_ENONPHYS ? "coarse propagator met a non-physical state" : "coarse status %d", st);
    }
    if (rc) return cfail(c, rc, "%s", c->ff ? c->ff->err.c_str() : c->fine->err.c_str());
    return PR_OK;
}

extern "C" {

// Shared by pr_init (E = 0, force = false) and pr_init_force.
static int ctx_create(pr_ctx** out, const pr_grid* g, const pr_velocity* v, double eps, const pr_time* t,
                      bool force, int nvx, const double* E)
{
    auto init_fail = [](int code, const std::string& m) {
        std::lock_guard<std::mutex> lk(g_init_mu);
        g_init_error = m;
        return code;
    };
    if (!out) return PR_EINVAL;
    *out = nullptr;
    if (!g || !v || !t) return init_fail(PR_EINVAL, "null parameter block");
    if (t->n_slices < 1) return init_fail(PR_EINVAL, "n_slices must be >= 1");
    if (!(t->T > 0) || !(t->cfl_f > 0) || !(t->cfl_g > 0) || !std::isfinite(t->T) || !std::isfinite(t->cfl_f) ||
        !std::isfinite(t->cfl_g))
        return init_fail(PR_EINVAL, "T, cfl_f and cfl_g must be finite and > 0");
    if (t->precision != PR_FP64 && t->precision != PR_MIXED) return init_fail(PR_EINVAL, "bad precision");
    if (t->sound_speed != PR_SOUND_GAMMA53 && t->sound_speed != PR_SOUND_SQRT_THETA)
        return init_fail(PR_EINVAL, "bad sound speed");
    if (t->nf < 0 || t->max_batch < 0) return init_fail(PR_EINVAL, "nf and max_batch must be >= 0");
    if (t->coarse_model != PR_COARSE_EULER && t->coarse_model != PR_COARSE_CNS)
        return init_fail(PR_EINVAL, "bad coarse model");
    if (t->lift_order != 0 && t->lift_order != 1) return init_fail(PR_EINVAL, "lift order must be 0 or 1");
    if ((t->coarse_model == PR_COARSE_CNS || t->lift_order == 1) && !(std::isfinite(eps) && eps > 0))
        return init_fail(PR_EINVAL, "the Navier-Stokes model and the first-order lift need a finite eps > 0");
    pr_ctx* c = new pr_ctx();
    c->g = *g;
    c->v = *v;
    c->eps = eps;
    c->t = *t;
    c->nx = g->nx;
    c->N = t->n_slices;
    c->dT = t->T / t->n_slices;
    // fine steps per slice: n_f = ceil(dT / dt_stab), dt_stab = cfl dx / max|v_x| (Sec. 2.2),
    // with the force cfl / (max|v_x|/dx + E_max/dv_x)
    double dx = (g->x1 - g->x0) / g->nx;
    pr_force_instance fd{g->nx, g->x0, g->x1, g->bc, nvx, v->nv, v->L, eps, 1.0, E};
    double dts = 0.0;
    if (force) {
        if (nvx < 2 || pr_force_dt_stab(&fd, t->cfl_f, &dts) != PR_OK) {
            free_ctx(c);
            return init_fail(PR_EINVAL, "bad force-path velocity grid");
        }
    } else {
        pr_instance gi{g->nx, g->x0, g->x1, g->bc, v->nv, v->L, eps, 1.0, t->scheme};
        if (pr_fine_dt_stab(&gi, t->cfl_f, &dts) != PR_OK) {
            free_ctx(c);
            return init_fail(PR_EINVAL, "bad grid or velocity box");
        }
    }
    if (t->nf > 0) c->nf = t->nf;
    else {
        double r = c->dT / dts;
        c->nf = std::max(1, (int)std::ceil(r * (1.0 - 1e-9)));
    }
    c->dtf = c->dT / c->nf;
    c->n_res = t->max_batch > 0 ? std::min(t->max_batch, c->N) : c->N;
    std::string err;
    int rc;
    if (force) {
        fd.dt = c->dtf;
        std::vector<pr_force_instance> descs(c->n_res, fd);
        rc = prf::create(&c->ff, descs.data(), c->n_res, t->scheme, t->precision, err);
    } else {
        pr_instance d{g->nx, g->x0, g->x1, g->bc, v->nv, v->L, eps, c->dtf, t->scheme};
        std::vector<pr_instance> descs(c->n_res, d);
        rc = create_batch(&c->fine, descs.data(), c->n_res, t->precision, err);
    }
    if (rc) {
        free_ctx(c);
        return init_fail(rc, err);
    }
    size_t lvl = (size_t)(c->N + 1) * 5 * c->nx * sizeof(double);
    if (cudaMalloc(&c->dU, lvl) != cudaSuccess || cudaMalloc(&c->dPFL, lvl) != cudaSuccess ||
        cudaMalloc(&c->dGs, lvl) != cudaSuccess || cudaMalloc(&c->derr, sizeof(double) * (c->N + 2)) != cudaSuccess ||
        cudaMalloc(&c->dwork, sizeof(double) * prk::coarse_work_doubles(c->nx)) != cudaSuccess ||
        cudaMalloc(&c->dtmp, sizeof(double) * 10 * c->nx) != cudaSuccess || cudaMalloc(&c->dk, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->dstatus, sizeof(int)) != cudaSuccess || cudaMallocHost(&c->h_pinned, sizeof(double) * pinned_doubles(c)) != cudaSuccess) {
        free_ctx(c);
        return init_fail(PR_ENOMEM, "parareal iterate buffers");
    }
    cudaMemset(c->dU, 0, lvl);
    cudaMemset(c->dPFL, 0, lvl);
    cudaMemset(c->dGs, 0, lvl);
    cudaMemset(c->derr, 0, sizeof(double) * (c->N + 2));
    cudaMemset(c->dk, 0, sizeof(int));
    cudaMemset(c->dstatus, 0, sizeof(int));
    c->cp.nx = g->nx;
    c->cp.bc = g->bc;
    c->cp.sound = t->sound_speed;
    c->cp.x0 = g->x0;
    c->cp.x1 = g->x1;
    c->cp.dx = dx;
    c->cp.cfl = t->cfl_g;
    c->cp.E = force ? c->ff->d_E : nullptr;
    c->cp.visc = t->coarse_model == PR_COARSE_CNS ? eps : 0.0;
    if (force) c->ff->lift_order = t->lift_order;
    else c->fine->lift_order = t->lift_order;
    c->live.assign(c->n_res, 0);
    for (int b = 0; b < c->n_res; ++b) bind_slice(c, b, b + 1);
    cudaError_t ue = force ? prf::upload(c->ff, 0, c->n_res, c->ff->stream)
                           : prk::copy_now(c->fine->d_inst, c->fine->h.data(), sizeof(Inst) * c->n_res,
                                           cudaMemcpyHostToDevice, c->fine->stream);
    if (ue != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        free_ctx(c);
        return init_fail(PR_ECUDA, "descriptor upload");
    }
    choose_fine_path(c);
    *out = c;
    return PR_OK;
}

int pr_init(pr_ctx** out, const pr_grid* g, const pr_velocity* v, double eps, const pr_time* t)
{
    return ctx_create(out, g, v, eps, t, false, 0, nullptr);
}

int pr_init_force(pr_ctx** out, const pr_grid* g, const pr_velocity* v, double eps, const pr_time* t, int nvx,
                  const double* E)
{
    return ctx_create(out, g, v, eps, t, true, nvx, E);
}

int pr_destroy(pr_ctx* c)
{
    if (c) {
        if (c->fine || c->ff) cudaStreamSynchronize(ctx_stream(c));
        free_ctx(c);
    }
    return PR_OK;
}

const char* pr_last_error(const pr_ctx* c)
{
    if (!c) return g_init_error.c_str();
    return c->err.c_str();
}

int pr_fine_steps_per_slice(const pr_ctx* c, int* nf, double* dt)
{
    if (!c) return PR_EINVAL;
    if (nf) *nf = c->nf;
    if (dt) *dt = c->dtf;
    return PR_OK;
}

int pr_iterations(const pr_ctx* c, int* k)
{
    if (!c || !k) return PR_EINVAL;
    *k = c->k;
    return PR_OK;
}

// ---- parareal resume: the iteration state in a file ----
//
// Layout (host byte order): "PRPARA01"; 16 int32 (nx, bc, nv, N, nf, scheme,
// precision, sound speed, coarse model, lift order, force, nvx, k, 0, 0, 0);
// 12 doubles (x0, x1, L, eps, T, cfl_f, cfl_g, dt_f, dT, 0, 0, 0); with the
// force, E [nx]; the errors [N+2]; U^{n,k} and the coarse values
// G(U^{n-1,k}) the next correction reuses, each [N+1][5][nx] conserved.
static const char kStateMagic[8] = {'P', 'R', 'P', 'A', 'R', 'A', '0', '1'};

static void state_header(const pr_ctx* c, int32_t* hi, double* hd)
{
    std::memset(hi, 0, 16 * sizeof(int32_t));
    std::memset(hd, 0, 12 * sizeof(double));
    const int32_t v[13] = {c->nx, c->g.bc, c->v.nv, c->N, c->nf, c->t.scheme, c->t.precision, c->t.sound_speed,
                           c->t.coarse_model, c->t.lift_order, c->ff ? 1 : 0, c->ff ? c->ff->nvx : 0, c->k};
    std::memcpy(hi, v, sizeof v);
    const double d[9] = {c->g.x0, c->g.x1, c->v.L, c->eps, c->t.T, c->t.cfl_f, c->t.cfl_g, c->dtf, c->dT};
    std::memcpy(hd, d, sizeof d);
}

// The problem's force field from the device (empty without one).
static int state_force(pr_ctx* c, std::vector<double>& E)
{
    E.clear();
    if (!c->ff) return PR_OK;
    E.resize(c->nx);
    CCUDA(c, cudaMemcpy(E.data(), c->ff->d_E, sizeof(double) * c->nx, cudaMemcpyDeviceToHost));
    return PR_OK;
}

int pr_save(pr_ctx* c, const char* path)
{
    if (!c) return PR_EINVAL;
    if (!path) return cfail(c, PR_EINVAL, "null path");
    if (!c->initialized) return cfail(c, PR_EINVAL, "call pr_set_initial first");
    CCUDA(c, cudaStreamSynchronize(ctx_stream(c)));
    int rc = take_ctx_status(c);
    if (rc) return rc;
    const size_t lvl = (size_t)(c->N + 1) * 5 * c->nx;
    std::vector<double> U(lvl), G(lvl), err(c->N + 2), E;
    CCUDA(c, cudaMemcpy(U.data(), c->dU, sizeof(double) * lvl, cudaMemcpyDeviceToHost));
    CCUDA(c, cudaMemcpy(G.data(), c->dGs, sizeof(double) * lvl, cudaMemcpyDeviceToHost));
    CCUDA(c, cudaMemcpy(err.data(), c->derr, sizeof(double) * (c->N + 2), cudaMemcpyDeviceToHost));
    if ((rc = state_force(c, E))) return rc;
    int32_t hi[16];
    double hd[12];
    state_header(c, hi, hd);
    FILE* f = std::fopen(path, "wb");
    if (!f) return cfail(c, PR_EINVAL, "cannot open %s for writing", path);
    bool ok = std::fwrite(kStateMagic, 1, 8, f) == 8 && std::fwrite(hi, sizeof hi, 1, f) == 1 &&
              std::fwrite(hd, sizeof hd, 1, f) == 1 && (E.empty() || std::fwrite(E.data(), sizeof(double), E.size(), f) == E.size()) &&
              std::fwrite(err.data(), sizeof(double), err.size(), f) == err.size() &&
              std::fwrite(U.data(), sizeof(double), lvl, f) == lvl && std::fwrite(G.data(), sizeof(double), lvl, f) == lvl;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return cfail(c, PR_EINVAL, "writing %s failed", path);
    return PR_OK;
}

int pr_load(pr_ctx* c, const char* path)
{
    if (!c) return PR_EINVAL;
    if (!path) return cfail(c, PR_EINVAL, "null path");
    FILE* f = std::fopen(path, "rb");
    if (!f) return cfail(c, PR_EINVAL, "cannot open %s", path);
    char magic[8];
    int32_t hi[16], want_i[16];
    double hd[12], want_d[12];
    std::vector<double> E, Ew;
    int rc = state_force(c, Ew);
    if (rc) {
        std::fclose(f);
        return rc;
    }
    state_header(c, want_i, want_d);
    const size_t lvl = (size_t)(c->N + 1) * 5 * c->nx;
    std::vector<double> U(lvl), G(lvl), err(c->N + 2);
    E.resize(Ew.size());
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kStateMagic, 8) == 0 &&
              std::fread(hi, sizeof hi, 1, f) == 1 && std::fread(hd, sizeof hd, 1, f) == 1;
    // every size and setting but k must be this problem's, bit for bit
    bool same = ok && std::memcmp(hi, want_i, 12 * sizeof(int32_t)) == 0 && std::memcmp(hd, want_d, sizeof hd) == 0;
    ok = same && (E.empty() || std::fread(E.data(), sizeof(double), E.size(), f) == E.size()) &&
         std::fread(err.data(), sizeof(double), err.size(), f) == err.size() &&
         std::fread(U.data(), sizeof(double), lvl, f) == lvl && std::fread(G.data(), sizeof(double), lvl, f) == lvl;
    char extra;
    const bool at_end = ok && std::fread(&extra, 1, 1, f) == 0;
    std::fclose(f);
    if (!same) return cfail(c, PR_EINVAL, "%s is not a state of this problem (sizes, settings or format differ)", path);
    if (!ok || !at_end) return cfail(c, PR_EINVAL, "%s is truncated or has trailing bytes", path);
    if (!E.empty() && std::memcmp(E.data(), Ew.data(), sizeof(double) * E.size()) != 0)
        return cfail(c, PR_EINVAL, "%s was saved with another force field", path);
    const int k = hi[12];
    if (k < 0 || k > c->N + 1) return cfail(c, PR_EINVAL, "%s holds an iteration count outside 0..N+1", path);
    for (int n = 0; n <= c->N; ++n)
        if (check_cons(U.data() + (size_t)n * 5 * c->nx, c->nx))
            return cfail(c, PR_ENONPHYS, "%s holds a non-physical iterate (slice %d)", path, n);
    for (double e : err)
        if (!std::isfinite(e)) return cfail(c, PR_EINVAL, "%s holds a non-finite error", path);
    cudaStream_t s = ctx_stream(c);
    CCUDA(c, cudaStreamSynchronize(s));
    CCUDA(c, prk::copy_now(c->dU, U.data(), sizeof(double) * lvl, cudaMemcpyHostToDevice, s));
    CCUDA(c, prk::copy_now(c->dGs, G.data(), sizeof(double) * lvl, cudaMemcpyHostToDevice, s));
    CCUDA(c, prk::copy_now(c->derr, err.data(), sizeof(double) * err.size(), cudaMemcpyHostToDevice, s));
    const int next = k + 1;  // the device counter holds the iteration the next sweep runs
    CCUDA(c, prk::copy_now(c->dk, &next, sizeof(int), cudaMemcpyHostToDevice, s));
    c->k = k;
    c->initialized = true;
    std::fill(c->live.begin(), c->live.end(), 0);
    return PR_OK;
}

int pr_set_initial(pr_ctx* c, const double* U0)
{
    if (!c) return PR_EINVAL;
    if (!U0) return cfail(c, PR_EINVAL, "null initial state");
    if (check_prim(U0, c->nx)) return cfail(c, PR_ENONPHYS, "initial state has rho <= 0 or theta <= 0");
    // stream-ordered after any enqueued iteration; the staging copy is free
    // (every call that fills it ends synchronised)
    double* hV = pinned_state(c);
    prim_to_cons_host(c->nx, U0, hV);
    cudaStream_t s = ctx_stream(c);
    CCUDA(c, cudaMemcpyAsync(c->dU, hV, sizeof(double) * 5 * c->nx, cudaMemcpyHostToDevice, s));
    CCUDA(c, cudaMemsetAsync(c->dk, 0, sizeof(int), s));
    CCUDA(c, prk::launch_sweep(c->cp, c->N, c->dT, c->dk, c->dU, c->dPFL, c->dGs, c->derr, c->dwork, c->dstatus, 1,
                               c->dk, s));
    g_launches += 1;
    c->k = 0;
    c->initialized = true;
    std::fill(c->live.begin(), c->live.end(), 0);
    return take_ctx_status(c);
}

int pr_coarse_step(pr_ctx* c, const double* Vin, double* Vout, double dT)
{
    if (!c) return PR_EINVAL;
    if (!Vin || !Vout || !(dT >= 0) || !std::isfinite(dT))
        return cfail(c, PR_EINVAL, "null state, or dT negative or not finite");
    if (check_cons(Vin, c->nx))
        return cfail(c, PR_ENONPHYS, "state has a non-finite component, rho <= 0 or theta <= 0");
    cudaStream_t s = ctx_stream(c);
    CCUDA(c, cudaMemcpyAsync(c->dtmp, Vin, sizeof(double) * 5 * c->nx, cudaMemcpyHostToDevice, s));
    CCUDA(c, prk::launch_coarse(c->cp, c->dtmp, c->dtmp + 5 * c->nx, dT, c->dwork, c->dstatus, s));
    g_launches += 1;
    CCUDA(c, cudaMemcpyAsync(Vout, c->dtmp + 5 * c->nx, sizeof(double) * 5 * c->nx, cudaMemcpyDeviceToHost, s));
    return take_ctx_status(c);
}

int pr_fine_step(pr_ctx* c, int slice, int nsteps, void* stream)
{
    if (!c) return PR_EINVAL;
    if (!c->initialized) return cfail(c, PR_EINVAL, "call pr_set_initial first");
    if (slice < 1 || slice > c->N || nsteps < 0) return cfail(c, PR_EINVAL, "slice must be in 1..N and nsteps >= 0");
    if (c->ff) {
        pr_force* b = c->ff;
        cudaStream_t s = stream ? reinterpret_cast<cudaStream_t>(stream) : b->stream;
        int bi = (slice - 1) % c->n_res;
        if (c->live[bi] != slice) {
            bind_slice(c, bi, slice);
            prf::bind(b, bi, b->h[bi].Uin, nullptr);  // a free-running slice does not overwrite the fine results
            CCUDA(c, prf::upload(b, bi, bi + 1, s));
            c->descs_dirty = true;
            int rc = prf::enqueue_lift_run(b, bi, bi + 1, 0, s, false);
            if (rc) return cfail(c, rc, "%s", b->err.c_str());
            c->live[bi] = slice;
        }
        int rc = prf::enqueue_run(b, bi, bi + 1, nsteps, s, true);
        if (rc) return cfail(c, rc, "%s", b->err.c_str());
        return PR_OK;
    }
    pr_batch* b = c->fine;
    cudaStream_t s = stream ? reinterpret_cast<cudaStream_t>(stream) : b->stream;
    int bi = (slice - 1) % c->n_res;
    if (c->live[bi] != slice) {
        bind_slice(c, bi, slice);
        Inst tmp = b->h[bi];
        tmp.Uout = nullptr;  // a free-running slice does not overwrite the parareal fine results
        CCUDA(c, cudaMemcpyAsync(b->d_inst + bi, &tmp, sizeof(Inst), cudaMemcpyHostToDevice, s));
        c->descs_dirty = true;
        int rc = lift_instances(b, bi, bi + 1, s);
        if (rc) return cfail(c, rc, "%s", b->err.c_str());
        c->live[bi] = slice;
    }
    if (nsteps == 0) return PR_OK;
    prk::Active a{bi, bi + 1};
    CCUDA(c, cudaMemcpyAsync(b->d_active, &a, sizeof a, cudaMemcpyHostToDevice, s));
    int rc = enqueue_run(b, nsteps, 0, s, true);
    prk::Active all{0, b->n};
    CCUDA(c, cudaMemcpyAsync(b->d_active, &all, sizeof all, cudaMemcpyHostToDevice, s));
    if (rc) return cfail(c, rc, "%s", b->err.c_str());
    return PR_OK;
}

int pr_fine_moments(pr_ctx* c, int slice, int kind, double* out)
{
    if (!c) return PR_EINVAL;
    if (slice < 1 || slice > c->N) return cfail(c, PR_EINVAL, "slice must be in 1..N");
    int bi = (slice - 1) % c->n_res;
    if (c->live[bi] != slice) return cfail(c, PR_EINVAL, "slice %d has no live distribution", slice);
    if (c->ff) {
        int rc = pr_force_moments(c->ff, bi, kind, out);
        if (rc) return cfail(c, rc, "%s", c->ff->err.c_str());
        return PR_OK;
    }
    int rc = pr_batch_moments(c->fine, bi, kind, out);
    if (rc) return cfail(c, rc, "%s", c->fine->err.c_str());
    return PR_OK;
}

int pr_fine_get_f(pr_ctx* c, int slice, double* out)
{
    if (!c) return PR_EINVAL;
    if (slice < 1 || slice > c->N) return cfail(c, PR_EINVAL, "slice must be in 1..N");
    int bi = (slice - 1) % c->n_res;
    if (c->live[bi] != slice) return cfail(c, PR_EINVAL, "slice %d has no live distribution", slice);
    if (c->ff) {
        int rc = pr_force_get_f(c->ff, bi, out);
        if (rc) return cfail(c, rc, "%s", c->ff->err.c_str());
        return PR_OK;
    }
    int rc = pr_batch_get_f(c->fine, bi, out);
    if (rc) return cfail(c, rc, "%s", c->fine->err.c_str());
    return PR_OK;
}

}  // extern "C"

// Enqueue one iteration (k = c->k + 1 on the device counter) without graphs.
static int enqueue_iteration_plain(pr_ctx* c, int k)
{
    int first = std::max(k, 1);
    if (c->ff) {
        pr_force* b = c->ff;
        cudaStream_t s = b->stream;
        for (int w0 = first; w0 <= c->N; w0 += c->n_res) {
            int cnt = std::min(c->n_res, c->N - w0 + 1);
            for (int bi = 0; bi < cnt; ++bi) bind_slice(c, bi, w0 + bi);
            CCUDA(c, prf::upload(b, 0, c->n_res, s));
            int rc = prf::enqueue_lift_run(b, 0, cnt, c->nf, s, true);
            if (rc) return cfail(c, rc, "%s", b->err.c_str());
        }
        CCUDA(c, prk::launch_sweep(c->cp, c->N, c->dT, c->dk, c->dU, c->dPFL, c->dGs, c->derr, c->dwork, c->dstatus,
                                   1, c->dk, s));
        g_launches += 1;
        return PR_OK;
    }
    pr_batch* b = c->fine;
    cudaStream_t s = b->stream;
    for (int w0 = first; w0 <= c->N; w0 += c->n_res) {
        int cnt = std::min(c->n_res, c->N - w0 + 1);
        for (int bi = 0; bi < cnt; ++bi) bind_slice(c, bi, w0 + bi);
        CCUDA(c, cudaMemcpyAsync(b->d_inst, b->h.data(), sizeof(Inst) * c->n_res, cudaMemcpyHostToDevice, s));
        if (c->use_cluster) {  // lift, n_f steps and projection of the wave's slices in one launch
            prk::Active a{0, cnt};
            CCUDA(c, cudaMemcpyAsync(b->d_active, &a, sizeof a, cudaMemcpyHostToDevice, s));
            CCUDA(c, prk::launch_fine_cluster(b->scheme, c->v.nv, b->d_inst, b->d_active, cnt, c->nf, c->cl_C,
                                              c->cl_w, c->cl_smem, b->d_status, s));
            g_launches += 1;
            prk::Active all{0, b->n};
            CCUDA(c, cudaMemcpyAsync(b->d_active, &all, sizeof all, cudaMemcpyHostToDevice, s));
            continue;
        }
        int rc = lift_instances(b, 0, cnt, s);
        if (rc) return cfail(c, rc, "%s", b->err.c_str());
        prk::Active a{0, cnt};
        CCUDA(c, cudaMemcpyAsync(b->d_active, &a, sizeof a, cudaMemcpyHostToDevice, s));
        rc = enqueue_run(b, c->nf, 1, s, true);
        if (rc) return cfail(c, rc, "%s", b->err.c_str());
        prk::Active all{0, b->n};
        CCUDA(c, cudaMemcpyAsync(b->d_active, &all, sizeof all, cudaMemcpyHostToDevice, s));
    }
    CCUDA(c, prk::launch_sweep(c->cp, c->N, c->dT, c->dk, c->dU, c->dPFL, c->dGs, c->derr, c->dwork, c->dstatus, 1,
                               c->dk, s));
    g_launches += 1;
    return PR_OK;
}

// The graph of one iteration when all slices are resident: set the active
// slices from the device counter k, lift them, run n_f fused fine steps in
// one persistent launch, then the sequential correction sweep (which bumps k).
static int build_graph_force(pr_ctx* c)
{
    pr_force* b = c->ff;
    cudaStream_t s = b->stream;
    for (int bi = 0; bi < c->n_res; ++bi) bind_slice(c, bi, bi + 1);
    CCUDA(c, prf::upload(b, 0, c->n_res, s));
    CCUDA(c, cudaStreamSynchronize(s));
    c->descs_dirty = false;
    CCUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = prf::enqueue_graph_body(b, c->dk, c->N, c->nf, s);
    if (e == cudaSuccess)
        e = prk::launch_sweep(c->cp, c->N, c->dT, c->dk, c->dU, c->dPFL, c->dGs, c->derr, c->dwork, c->dstatus, 1,
                              c->dk, s);
    cudaGraph_t gr = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return cfail(c, PR_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, gr, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(gr);
        return cfail(c, PR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    c->graph = gr;
    c->gexec = ex;
    return PR_OK;
}

static int build_graph(pr_ctx* c)
{
    if (c->ff) return build_graph_force(c);
    pr_batch* b = c->fine;
    cudaStream_t s = b->stream;
    for (int bi = 0; bi < c->n_res; ++bi) bind_slice(c, bi, bi + 1);
    CCUDA(c, prk::copy_now(b->d_inst, b->h.data(), sizeof(Inst) * c->n_res, cudaMemcpyHostToDevice, s));
    CCUDA(c, cudaStreamSynchronize(s));
    c->descs_dirty = false;
    CCUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = prk::launch_set_active(c->dk, b->d_active, 1, c->n_res, c->N, s);
    if (c->use_cluster) {
        if (e == cudaSuccess)
            e = prk::launch_fine_cluster(b->scheme, c->v.nv, b->d_inst, b->d_active, c->n_res, c->nf, c->cl_C,
                                         c->cl_w, c->cl_smem, b->d_status, s);
    } else {
    if (e == cudaSuccess)
        e = b->lift_order == 1
                ? prk::launch_lift_ce(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->d_state, b->d_active, b->nx_max,
                                      b->n, 0, b->d_status, s)
                : prk::launch_lift(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->d_state, b->d_active, b->max_tiles,
                                   b->n, b->lift_smem, b->d_status, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_sync, 0, b->sync_bytes, s);
    if (e == cudaSuccess)
        e = prk::launch_fine_run(b->precision == PR_FP64 ? 0 : 1, b->scheme, b->vpt, b->d_inst, b->d_state, b->d_prefix,
                                 b->d_active, c->nf, reinterpret_cast<unsigned long long*>(b->d_sync), b->d_status,
                                 c->nf > 1 ? prk::WAIT_LIMIT_NS : 0, b->grid, b->smem, s);
    }
    if (e == cudaSuccess)
        e = prk::launch_sweep(c->cp, c->N, c->dT, c->dk, c->dU, c->dPFL, c->dGs, c->derr, c->dwork, c->dstatus, 1,
                              c->dk, s);
    cudaGraph_t gr = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return cfail(c, PR_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, gr, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(gr);
        return cfail(c, PR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    c->graph = gr;
    c->gexec = ex;
    return PR_OK;
}

static int run_iterations(pr_ctx* c, int count, bool use_graph)
{
    cudaStream_t cs = ctx_stream(c);
    for (int it = 0; it < count; ++it) {
        int k = c->k + 1;
        if (k > c->N) {
            // every slice is already exact; the iteration changes nothing (error 0)
            CCUDA(c, cudaMemsetAsync(c->derr + std::min(k, c->N + 1), 0, sizeof(double), cs));
            c->k = k;
            continue;
        }
        if (use_graph && c->n_res == c->N) {
            if (!c->gexec || c->descs_dirty) {
                if (c->gexec) {
                    cudaGraphExecDestroy(c->gexec);
                    cudaGraphDestroy(c->graph);
                    c->gexec = nullptr;
                    c->graph = nullptr;
                }
                int rc = build_graph(c);
                if (rc) return rc;
            }
            CCUDA(c, cudaGraphLaunch(c->gexec, cs));
            g_launches += c->ff ? 1 + prf::graph_body_launches(c->ff, c->nf) : c->use_cluster ? 3 : 5;
        } else {
            int rc = enqueue_iteration_plain(c, k);
            if (rc) return rc;
        }
        c->k = k;
    }
    std::fill(c->live.begin(), c->live.end(), 0);
    return PR_OK;
}

extern "C" {

int pr_parareal_iter(pr_ctx* c, double* err_out)
{
    if (!c) return PR_EINVAL;
    if (!c->initialized) return cfail(c, PR_EINVAL, "call pr_set_initial first");
    int rc = run_iterations(c, 1, true);
    if (rc) return rc;
    if (err_out) {
        int k = std::min(c->k, c->N + 1);
        CCUDA(c, cudaMemcpyAsync(c->h_pinned, c->derr + k, sizeof(double), cudaMemcpyDeviceToHost, ctx_stream(c)));
        rc = take_ctx_status(c);
        *err_out = c->h_pinned[0];
        return rc;
    }
    return PR_OK;
}

int pr_set_fine_path(pr_ctx* c, int mode)
{
    if (!c) return PR_EINVAL;
    if (mode < PR_FINE_AUTO || mode > PR_FINE_CLUSTER) return cfail(c, PR_EINVAL, "unknown fine path %d", mode);
    if (c->ff && mode == PR_FINE_CLUSTER)
        return cfail(c, PR_EINVAL, "the cluster-resident fine run has no exterior force");
    CCUDA(c, cudaStreamSynchronize(ctx_stream(c)));
    const int old = c->fpath_req;
    c->fpath_req = mode;
    int rc = choose_fine_path(c);
    if (rc) {
        c->fpath_req = old;
        choose_fine_path(c);
        return rc;
    }
    c->descs_dirty = true;  // the captured iteration holds the old launches
    return PR_OK;
}

int pr_get_fine_path(const pr_ctx* c, int* path)
{
    if (!c || !path) return PR_EINVAL;
    *path = c->use_cluster ? PR_FINE_CLUSTER : PR_FINE_TILED;
    return PR_OK;
}

int pr_fine_cluster_shape(const pr_ctx* c, int* cluster, int* cells_per_cta, int* resident)
{
    if (!c) return PR_EINVAL;
    if (cluster) *cluster = c->cl_C;
    if (cells_per_cta) *cells_per_cta = c->cl_w;
    if (resident) *resident = c->cl_resident;
    return PR_OK;
}

int pr_set_force_step(pr_ctx* c, int cluster, int columns, int persistent)
{
    if (!c) return PR_EINVAL;
    if (!c->ff) return cfail(c, PR_EINVAL, "the problem has no exterior force (pr_init_force)");
    int rc = cluster > 0 ? pr_force_set_cluster(c->ff, cluster) : PR_OK;
    if (rc == PR_OK) rc = pr_force_set_march(c->ff, columns);
    if (rc == PR_OK) rc = pr_force_set_persistent(c->ff, persistent);
    if (rc) return cfail(c, rc, "%s", c->ff->err.c_str());
    c->descs_dirty = true;  // the captured iteration holds the old launches
    return PR_OK;
}

int pr_parareal_run(pr_ctx* c, int K, double tol, int* k_done, double* errs)
{
    if (!c) return PR_EINVAL;
    if (!c->initialized) return cfail(c, PR_EINVAL, "call pr_set_initial first");
    if (K < 0) return cfail(c, PR_EINVAL, "K must be >= 0");
    int done = 0, rc = PR_OK;
    double last = 0.0;
    if (tol > 0) {
        while (done < K) {
            double e = 0;
            rc = pr_parareal_iter(c, &e);
            if (rc) break;
            if (errs) errs[done] = e;
            ++done;
            last = e;
            if (e < tol) break;
        }
    } else {
        int k0 = c->k;
        rc = run_iterations(c, K, true);
        if (rc == PR_OK) {
            CCUDA(c, cudaMemcpyAsync(c->h_pinned, c->derr, sizeof(double) * (c->N + 2), cudaMemcpyDeviceToHost,
                                     ctx_stream(c)));
            rc = take_ctx_status(c);
            for (int i = 0; i < K; ++i) {
                int k = std::min(k0 + 1 + i, c->N + 1);
                double e = k0 + 1 + i > c->N ? 0.0 : c->h_pinned[k];
                if (errs) errs[i] = e;
                last = e;
            }
            done = K;
        }
    }
    if (k_done) *k_done = done;
    if (rc == PR_OK && tol > 0 && done == K && last >= tol) return cfail(c, PR_ENOTCONV, "error %g >= tol after %d iterations", last, K);
    return rc;
}

int pr_moments(pr_ctx* c, int n, int kind, double* out)
{
    if (!c) return PR_EINVAL;
    if (n < 0 || n > c->N || !out) return cfail(c, PR_EINVAL, "n must be in 0..N");
    if (kind != PR_PRIMITIVE && kind != PR_CONSERVED) return cfail(c, PR_EINVAL, "bad kind");
    std::vector<double> V(5 * c->nx);
    CCUDA(c, cudaMemcpyAsync(V.data(), c->dU + (size_t)n * 5 * c->nx, sizeof(double) * 5 * c->nx, cudaMemcpyDeviceToHost,
                             ctx_stream(c)));
    int rc = take_ctx_status(c);
    if (kind == PR_CONSERVED) memcpy(out, V.data(), sizeof(double) * 5 * c->nx);
    else cons_to_prim_host(c->nx, V.data(), out);
    return rc;
}

}  // extern "C"

// ======================= several problems in one launch =======================
//
// The batching of Algorithm 2 across problems: every slice of every problem
// and a set of independent instances are instances of one batch, so one
// persistent launch per iteration runs the fine propagations of all of them;
// each problem's correction sweep then runs on a stream of its own (the sweeps
// are sequential inside a problem, independent across problems).  The
// problems iterate in lockstep (one k); the slices are ordered by slice index,
// so the slices n >= k of every problem and the independent instances after
// them form one contiguous active range.
struct pr_multi {
    std::vector<pr_ctx*> ctx;
    pr_batch* b = nullptr;
    int n_sl = 0, n_extra = 0, nf = 0, Nmin = 0;
    int* d_n = nullptr;             // slice index of each slice instance
    prk::Active* d_act = nullptr;   // [0] lift range, [1] the independent instances
    std::vector<std::pair<int, int>> owner;  // (problem, slice) of each slice instance
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;    // fork, then one join per problem
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::string err;
};

static int mfail(pr_multi* m, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (m) m->err = buf;
    return code;
}

#define MCUDA(m, call)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return mfail((m), PR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Failure of pr_multi_create (no object yet): the message goes where
// pr_multi_last_error(NULL) reads it.
static int minit_fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> lk(g_init_mu);
    g_init_error = buf;
    return code;
}

static void free_multi(pr_multi* m)
{
    if (!m) return;
    if (m->gexec) cudaGraphExecDestroy(m->gexec);
    if (m->graph) cudaGraphDestroy(m->graph);
    for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
    for (cudaStream_t s : m->side) cudaStreamDestroy(s);
    if (m->b) free_batch(m->b);
    cudaFree(m->d_n);
    cudaFree(m->d_act);
    delete m;
}

// The graph of one lockstep iteration: active ranges from k, lift of the
// active slices, one persistent run of n_f steps over slices and independent
// instances, the independent instances' state advance, and every problem's
// correction sweep on its own stream (fork and join through events).
static int build_multi_graph(pr_multi* m)
{
    pr_batch* b = m->b;
    cudaStream_t s = b->stream;
    const int n = b->n, np = (int)m->ctx.size();
    MCUDA(m, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = prk::launch_set_active_multi(m->ctx[0]->dk, m->d_n, m->n_sl, n, b->d_active, m->d_act, s);
    if (e == cudaSuccess)
        e = b->lift_order == 1
                ? prk::launch_lift_ce(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->d_state, m->d_act, b->nx_max, n,
                                      0, b->d_status, s)
                : prk::launch_lift(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->d_state, m->d_act, b->max_tiles, n,
                                   b->lift_smem, b->d_status, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_sync, 0, b->sync_bytes, s);
    if (e == cudaSuccess)
        e = prk::launch_fine_run(b->precision == PR_FP64 ? 0 : 1, b->scheme, b->vpt, b->d_inst, b->d_state,
                                 b->d_prefix, b->d_active, m->nf, reinterpret_cast<unsigned long long*>(b->d_sync),
                                 b->d_status, m->nf > 1 ? prk::WAIT_LIMIT_NS : 0, b->grid, b->smem, s);
    if (e == cudaSuccess && m->n_extra > 0) e = prk::launch_advance(b->d_inst, b->d_state, m->d_act + 1, m->nf, n, s);
    if (e == cudaSuccess) e = cudaEventRecord(m->ev[0], s);
    for (int p = 0; p < np && e == cudaSuccess; ++p) {
        pr_ctx* c = m->ctx[p];
        e = cudaStreamWaitEvent(m->side[p], m->ev[0], 0);
        if (e == cudaSuccess)
            e = prk::launch_sweep(c->cp, c->N, c->dT, c->dk, c->dU, c->dPFL, c->dGs, c->derr, c->dwork, c->dstatus, 1,
                                  c->dk, m->side[p]);
        if (e == cudaSuccess) e = cudaEventRecord(m->ev[1 + p], m->side[p]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, m->ev[1 + p], 0);
    }
    cudaGraph_t gr = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return mfail(m, PR_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, gr, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(gr);
        return mfail(m, PR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    m->graph = gr;
    m->gexec = ex;
    return PR_OK;
}

extern "C" {

int pr_multi_create(pr_multi** out, pr_ctx* const* ctxs, int n_ctx, const pr_instance* extra, int n_extra)
{
    if (!out) return PR_EINVAL;
    *out = nullptr;
    if (!ctxs || n_ctx < 1 || n_extra < 0 || (n_extra > 0 && !extra))
        return minit_fail(PR_EINVAL, "need at least one problem, and the independent instances when n_extra > 0");
    const pr_ctx* c0 = ctxs[0];
    std::set<const pr_ctx*> seen;
    for (int p = 0; p < n_ctx; ++p) {
        const pr_ctx* c = ctxs[p];
        if (!c) return minit_fail(PR_EINVAL, "problem %d is null", p);
        if (!seen.insert(c).second) return minit_fail(PR_EINVAL, "problem %d is given twice", p);
        if (c->ff) return minit_fail(PR_EINVAL, "problem %d has an exterior force (pr_init_force): not supported here", p);
        if (c->t.precision != c0->t.precision || c->t.scheme != c0->t.scheme || c->nf != c0->nf ||
            c->fine->lift_order != c0->fine->lift_order)
            return minit_fail(PR_EINVAL, "problem %d differs from problem 0 in precision, scheme, fine steps per slice "
                                        "or lifting order", p);
    }
    for (int i = 0; i < n_extra; ++i)
        if (extra[i].scheme != c0->t.scheme)
            return minit_fail(PR_EINVAL, "independent instance %d has another scheme than the problems", i);
    pr_multi* m = new pr_multi();
    m->ctx.assign(ctxs, ctxs + n_ctx);
    m->nf = c0->nf;
    m->n_extra = n_extra;
    m->Nmin = c0->N;
    for (const pr_ctx* c : m->ctx) m->Nmin = std::min(m->Nmin, c->N);
    // slice instances by slice index (then problem), the independent ones after them
    for (int n = 1;; ++n) {
        bool any = false;
        for (int p = 0; p < n_ctx; ++p)
            if (n <= ctxs[p]->N) {
                m->owner.push_back({p, n});
                any = true;
            }
        if (!any) break;
    }
    m->n_sl = (int)m->owner.size();
    std::vector<pr_instance> descs;
    descs.reserve(m->n_sl + n_extra);
    std::vector<int> nidx;
    for (auto [p, n] : m->owner) {
        const pr_ctx* c = ctxs[p];
        descs.push_back(pr_instance{c->nx, c->g.x0, c->g.x1, c->g.bc, c->v.nv, c->v.L, c->eps, c->dtf, c->t.scheme});
        nidx.push_back(n);
    }
    descs.insert(descs.end(), extra, extra + n_extra);
    std::string err;
    int rc = create_batch(&m->b, descs.data(), (int)descs.size(), c0->t.precision, err);
    if (rc) {
        free_multi(m);
        return minit_fail(rc, "%s", err.c_str());
    }
    m->b->lift_order = c0->fine->lift_order;
    for (int i = 0; i < m->n_sl; ++i) {  // lift from U^{n-1}, project into P F L^n of the owning problem
        const pr_ctx* c = ctxs[m->owner[i].first];
        const int n = m->owner[i].second;
        m->b->h[i].Uin = c->dU + (size_t)(n - 1) * 5 * c->nx;
        m->b->h[i].Uout = c->dPFL + (size_t)n * 5 * c->nx;
    }
    const prk::Active act[2] = {{0, m->n_sl}, {m->n_sl, m->n_sl + n_extra}};
    bool ok = cudaMalloc(&m->d_n, sizeof(int) * std::max(1, m->n_sl)) == cudaSuccess &&
              cudaMalloc(&m->d_act, sizeof act) == cudaSuccess &&
              prk::copy_now(m->d_n, nidx.data(), sizeof(int) * m->n_sl, cudaMemcpyHostToDevice, m->b->stream) ==
                  cudaSuccess &&
              prk::copy_now(m->d_act, act, sizeof act, cudaMemcpyHostToDevice, m->b->stream) == cudaSuccess &&
              prk::copy_now(m->b->d_inst, m->b->h.data(), sizeof(Inst) * m->b->n, cudaMemcpyHostToDevice,
                            m->b->stream) == cudaSuccess;
    m->side.assign(n_ctx, nullptr);
    m->ev.assign(n_ctx + 1, nullptr);
    for (int p = 0; p < n_ctx && ok; ++p) ok = cudaStreamCreateWithFlags(&m->side[p], cudaStreamNonBlocking) == cudaSuccess;
    for (auto& e : m->ev)
        if (ok) ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok || cudaDeviceSynchronize() != cudaSuccess) {
        free_multi(m);
        return minit_fail(PR_ECUDA, "multi-problem set-up");
    }
    *out = m;
    return PR_OK;
}

int pr_multi_destroy(pr_multi* m)
{
    if (!m) return PR_EINVAL;
    cudaStreamSynchronize(m->b->stream);
    free_multi(m);
    return PR_OK;
}

const char* pr_multi_last_error(const pr_multi* m) { return m ? m->err.c_str() : g_init_error.c_str(); }

int pr_multi_batch(pr_multi* m, pr_batch** batch, int* first_independent)
{
    if (!m) return PR_EINVAL;
    if (batch) *batch = m->b;
    if (first_independent) *first_independent = m->n_sl;
    return PR_OK;
}

int pr_multi_iterate(pr_multi* m, int count, double* errs)
{
    if (!m) return PR_EINVAL;
    if (count < 0) return mfail(m, PR_EINVAL, "count must be >= 0");
    const int np = (int)m->ctx.size(), k = m->ctx[0]->k;
    for (int p = 0; p < np; ++p) {
        const pr_ctx* c = m->ctx[p];
        if (!c->initialized) return mfail(m, PR_EINVAL, "problem %d: call pr_set_initial first", p);
        if (c->k != k) return mfail(m, PR_EINVAL, "the problems must be at the same iteration (problem %d: k = %d, "
                                                  "problem 0: k = %d)", p, c->k, k);
    }
    if (k + count > m->Nmin)
        return mfail(m, PR_EINVAL, "k + count = %d exceeds the smallest N (%d): the slices of that problem are exact",
                     k + count, m->Nmin);
    cudaStream_t s = m->b->stream;
    for (int p = 0; p < np; ++p) MCUDA(m, cudaStreamSynchronize(ctx_stream(m->ctx[p])));  // their own work first
    if (!m->gexec) {
        int rc = build_multi_graph(m);
        if (rc) return rc;
    }
    for (int it = 0; it < count; ++it) {
        MCUDA(m, cudaGraphLaunch(m->gexec, s));
        g_launches += 4 + (m->n_extra > 0 ? 1 : 0) + np;
    }
    MCUDA(m, cudaStreamSynchronize(s));
    int rc = take_status(m->b, s);
    if (rc) return mfail(m, rc, "%s", m->b->err.c_str());
    for (int p = 0; p < np; ++p) {
        pr_ctx* c = m->ctx[p];
        c->k = k + count;
        std::fill(c->live.begin(), c->live.end(), 0);
        const int rc2 = take_ctx_status(c);
        if (rc2) return mfail(m, rc2, "problem %d: %s", p, c->err.c_str());
        if (errs && count > 0) {
            std::vector<double> e(count);
            MCUDA(m, cudaMemcpy(e.data(), c->derr + k + 1, sizeof(double) * count, cudaMemcpyDeviceToHost));
            for (int it = 0; it < count; ++it) errs[(size_t)it * np + p] = e[it];
        }
    }
    return PR_OK;
}

}  // extern "C"
