// Host runtime of the exterior-force path: the pr_force_* entry points of
// include/pr.h and the helpers the parareal context uses (force_rt.h).
// Owns the instances' state buffers, descriptors, velocity tables and the
// per-run CUDA-event timing.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "force_rt.h"

namespace {

std::mutex g_fprep_mu;
bool g_fprepared = false;
std::mutex g_ferr_mu;
std::string g_ferr;

int dev_attr(cudaDeviceAttr a)
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, a, dev);
    return v;
}

void prepare_once()
{
    std::lock_guard<std::mutex> lk(g_fprep_mu);
    if (g_fprepared) return;
    prk::prepare_force_kernels(dev_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin));
    cudaGetLastError();
    g_fprepared = true;
}

int ffail(pr_force* b, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return code;
}

#define FCUDA(b, call)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return ffail((b), PR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

size_t elem(int precision) { return precision == PR_FP64 ? sizeof(double) : sizeof(float); }

double dt_stab(const pr_force_instance& d, double cfl)
{
    double dx = (d.x1 - d.x0) / d.nx, dvx = 2.0 * d.L / d.nvx, vmax = d.L - 0.5 * dvx;
    double em = 0.0;
    if (d.E)
        for (int i = 0; i < d.nx; ++i) em = std::max(em, std::fabs(d.E[i]));
    if (em == 0.0) return cfl * dx / vmax;
    return cfl / (vmax / dx + em / dvx);
}

// Geometry for cluster size C (the v_x rows split over C CTAs); false if a
// CTA would be empty or its rows do not fit shared memory.
bool geometry(int precision, int scheme, int nvx, int nvp, int C, int max_threads, prk::FGeom* g, size_t* smem)
{
    long long ncol = (long long)nvx * nvp * nvp;
    if (C < 1 || C > prk::FORCE_MAX_CLUSTER) return false;
    int rows = (nvx + C - 1) / C;
    if ((C - 1) * rows >= nvx) return false;  // an empty CTA
    if ((size_t)rows * nvp * nvp * elem(precision) > (size_t)prk::FORCE_MAX_CHUNK_BYTES) return false;
    size_t sm = prk::force_step_smem(precision, scheme, nvx, nvp, rows);
    if (sm > (size_t)dev_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin) - 1024) return false;
    g->nvx = nvx;
    g->nvp = nvp;
    g->ncol = ncol;
    g->C = C;
    g->rows = rows;
    g->bulk = ((size_t)nvp * nvp * elem(precision)) % 16 == 0 ? 1 : 0;
    g->vec = g->bulk ? (int)(16 / elem(precision)) : 1;
    prk::force_step_layout(nvp, g->vec, rows, max_threads, &g->groups, &g->threads);
    if (g->threads > (g->vec == 1 ? 1024 : 512)) return false;
    g->buf_off = (int)prk::force_step_buf_off(precision, nvx, nvp);
    g->march = 0;
    g->scheme = scheme;
    *smem = sm;
    return true;
}

// Default cluster size: the smallest that fits, raised (up to 8) while a CTA
// holds more than 8192 cells.
int default_cluster(int precision, int scheme, int nvx, int nvp)
{
    prk::FGeom g;
    size_t sm;
    int C = 1;
    while (C <= prk::FORCE_MAX_CLUSTER && !geometry(precision, scheme, nvx, nvp, C, 256, &g, &sm)) ++C;
    if (C > prk::FORCE_MAX_CLUSTER) return 0;
    while (C < 8 && (long long)g.rows * nvp * nvp > 8192) {
        int D = C + 1;
        while (D <= 8 && !geometry(precision, scheme, nvx, nvp, D, 256, &g, &sm)) ++D;
        if (D > 8) break;
        C = D;
    }
    geometry(precision, scheme, nvx, nvp, C, 256, &g, &sm);
    return C;
}

// Fused-step geometry with C CTAs per column (sets g.march to the walk
// length, *smem): false when the fused step does not apply (precision,
// scheme, row size, a CTA straddling v_x = 0, shared memory).  walk_req >= 1:
// walks of about that length; -1 (automatic): the columns per resident CTA
// group (so a step's items fill the resident CTAs once), capped where the
// walk's tables would cost a resident CTA per SM and at 32, and false below 2
// (too few columns: the clustered step is as fast there).  The columns split
// into equal walks.
bool fused_geometry(const pr_force* b, int C, int max_threads, int walk_req, prk::FGeom* out, size_t* smem)
{
    prk::FGeom gg;
    prk::FGeom* g = &gg;
    size_t sm0;
    if (!geometry(b->precision, b->scheme, b->nvx, b->nvp, C, max_threads, g, &sm0)) return false;
    if (!prk::force_fused_fits(b->precision, b->scheme, *g)) return false;
    for (const prk::FInst& I : b->h) {
        if (I.hpos < b->nvx && I.hpos % g->rows != 0) return false;
        if (b->scheme != 0 && I.bc == 2) return false;  // MUSCL: periodic and outflow only
    }
    const size_t optin = (size_t)dev_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin) - 1024;
    auto resident = [&](int S) {
        const size_t sm = prk::force_fused_smem(b->precision, b->scheme, b->nvp, g->rows, S);
        int per_sm = 0;
        if (sm > optin || prk::force_fused_occupancy(b->precision, b->scheme, g->threads, sm, &per_sm) != 0) return 0;
        return per_sm;
    };
    const int per1 = resident(1);
    if (per1 < 1) return false;
    const int cap = std::min(32, b->nx);
    long long S = walk_req;
    if (S < 0) {
        int scap = 1;
        while (scap < cap && resident(scap + 1) == per1) ++scap;
        const long long groups = std::max<long long>(1, (long long)per1 * dev_attr(cudaDevAttrMultiProcessorCount) / C);
        S = std::min<long long>(scap, (long long)b->n * b->nx / groups);
        if (S < 2) return false;
        // one resident CTA per SM (FP64 Test 3): half the walk, two waves of
        // items per step balance better (one instance 234 instead of 250 us)
        if (per1 == 1) S = std::max<long long>(2, S / 2);
    }
    S = std::max<long long>(1, std::min<long long>(S, cap));
    long long walks = (b->nx + S - 1) / S;
    S = (b->nx + walks - 1) / walks;
    if (b->scheme != 0) {
        // a MUSCL walk reads three columns past each end: every walk needs
        // at least three so that those belong to its neighbour walks (the
        // next longer walk whose last walk is long enough)
        for (S = std::max<long long>(S, 3); S < b->nx; ++S) {
            walks = (b->nx + S - 1) / S;
            if (b->nx - (walks - 1) * S >= 3) break;
        }
        S = std::min<long long>(S, b->nx);
        walks = (b->nx + S - 1) / S;
    }
    const size_t sm = prk::force_fused_smem(b->precision, b->scheme, b->nvp, g->rows, (int)S);
    if (resident((int)S) < 1) return false;
    g->march = (int)S;
    *out = gg;
    *smem = sm;
    return true;
}

// Cluster size of the fused step by default: the fewest CTAs per column for
// which two CTAs of an 8-column walk share an SM, else the fewest that fit;
// 0 if the fused step does not apply.  (Rows per thread amortise the
// per-column reduction: on Test 3, 8 CTAs of 32 rows at two per SM beat 16 of
// 16 rows at three per SM by a fifth.)
int default_fused_cluster(const pr_force* b)
{
    const size_t half = (size_t)dev_attr(cudaDevAttrMaxSharedMemoryPerMultiprocessor) / 2 - 1024;
    int any = 0;
    for (int C = 1; C <= prk::FORCE_MAX_CLUSTER; ++C) {
        prk::FGeom g;
        size_t sm;
        if (!fused_geometry(b, C, b->max_threads, 1, &g, &sm)) continue;
        if (prk::force_fused_smem(b->precision, b->scheme, b->nvp, g.rows, std::min(8, b->nx)) <= half) return C;
        if (!any) any = C;
    }
    return any;
}

// CTAs of the persistent fused run that fit the device at once (0: none).
int fused_resident(const pr_force* b)
{
    int per_sm = 0;
    if (prk::force_fused_occupancy(b->precision, b->scheme, b->g.threads, b->smem, &per_sm) != 0) return 0;
    return per_sm * dev_attr(cudaDevAttrMultiProcessorCount);
}

// Whether a fused run of nsteps steps over n_inst instances takes one
// persistent launch: asked for, or (automatic) for every run of two steps or
// more (Test 3: 15.4 instead of 20.5 us per step for one instance, 85 instead
// of 83 % of the copy bandwidth for 64; steps overlap where a step's last
// items would leave CTAs idle).
bool fused_persistent(const pr_force* b, int n_inst, int nsteps)
{
    if (b->g.march <= 0 || b->persist_req == 0 || nsteps < 1) return false;
    const long long walks = (b->nx + b->g.march - 1) / b->g.march;
    const long long items = (long long)n_inst * walks * b->g.C;
    if (items * nsteps >= (1LL << 30) || fused_resident(b) < 1) return false;  // ticket range
    return b->persist_req == 1 || nsteps >= 2;
}

// Partials for the fused step's geometry (grown when needed; zeroed) and the
// descriptors' pointers into them (host copies; the caller uploads).
bool ensure_partials(pr_force* b)
{
    if (b->g.march <= 0) return true;
    const size_t per = (size_t)b->nx * prk::force_partials_per_column(b->g) * 8;  // one state's partials
    const size_t need = 2 * per * b->n;
    if (need > b->part_bytes) {
        cudaFree(b->d_part);
        b->d_part = nullptr;
        b->part_bytes = 0;
        if (cudaMalloc(&b->d_part, need) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        b->part_bytes = need;
    }
    if (prk::zero_now(b->d_part, need, b->stream) != cudaSuccess) return false;
    const int words = 1 + b->n * ((b->nx + b->g.march - 1) / b->g.march);
    if (words > b->fsync_words) {
        cudaFree(b->d_fsync);
        b->d_fsync = nullptr;
        b->fsync_words = 0;
        if (cudaMalloc(&b->d_fsync, sizeof(int) * words) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        b->fsync_words = words;
    }
    for (int k = 0; k < b->n; ++k)
        for (int j = 0; j < 2; ++j)
            b->h[k].part[j] = static_cast<unsigned char*>(b->d_part) + ((size_t)2 * k + j) * per;
    std::fill(b->sums_ok.begin(), b->sums_ok.end(), 0);
    return true;
}

// Byte size of an instance's node tables: v_x, v_y, v_z, v_y^2 + v_z^2 in the
// element type, then (float path) the nodes as float pairs hi + lo (v_x, then
// v_y = v_z), from which the float32 Maxwellian factors are evaluated.
static size_t vtab_bytes(int nvx, int nvp, size_t es)
{
    const size_t base = ((size_t)nvx + 3 * (size_t)nvp * nvp) * es;
    return es == sizeof(float) ? (base + 15) / 16 * 16 + 2 * ((size_t)nvx + nvp) * sizeof(float) : base;
}

static size_t vpair_offset(int nvx, int nvp, size_t es) { return (((size_t)nvx + 3 * (size_t)nvp * nvp) * es + 15) / 16 * 16; }

template <typename T>
void fill_vtab(std::vector<unsigned char>& out, int nvx, int nvp, double L)
{
    int nvp2 = nvp * nvp;
    std::vector<T> t((size_t)nvx + 3 * nvp2);
    double dvx = 2.0 * L / nvx, dvp = 2.0 * L / nvp;
    for (int j = 0; j < nvx; ++j) t[j] = (T)(-L + (j + 0.5) * dvx);
    for (int jp = 0; jp < nvp2; ++jp) {
        int jy = jp / nvp, jz = jp % nvp;
        double y = -L + (jy + 0.5) * dvp, z = -L + (jz + 0.5) * dvp;
        t[nvx + jp] = (T)y;
        t[nvx + nvp2 + jp] = (T)z;
        t[nvx + 2 * nvp2 + jp] = (T)(y * y + z * z);
    }
    out.assign(vtab_bytes(nvx, nvp, sizeof(T)), 0);
    memcpy(out.data(), t.data(), t.size() * sizeof(T));
    if (sizeof(T) == sizeof(float)) {
        float* pp = reinterpret_cast<float*>(out.data() + vpair_offset(nvx, nvp, sizeof(T)));
        auto put = [&](int k, double v) {
            const float h = (float)v;
            pp[2 * k] = h;
            pp[2 * k + 1] = (float)(v - (double)h);
        };
        for (int j = 0; j < nvx; ++j) put(j, -L + (j + 0.5) * dvx);
        for (int j = 0; j < nvp; ++j) put(nvx + j, -L + (j + 0.5) * dvp);
    }
}

void fold_events(pr_force* b)
{
    for (auto& p : b->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            b->step_ms_sum += ms;
            b->steps_timed += p.steps;
        }
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    b->pending.clear();
    cudaGetLastError();
}

void prim_to_cons(int nx, const double* U, double* V)
{
    for (int i = 0; i < nx; ++i) {
        double r = U[i], ux = U[nx + i], uy = U[2 * nx + i], uz = U[3 * nx + i], th = U[4 * nx + i];
        V[i] = r;
        V[nx + i] = r * ux;
        V[2 * nx + i] = r * uy;
        V[3 * nx + i] = r * uz;
        V[4 * nx + i] = 0.5 * r * (ux * ux + uy * uy + uz * uz) + 1.5 * r * th;
    }
}

int cons_to_prim(int nx, const double* V, double* U)
{
    int bad = 0;
    for (int i = 0; i < nx; ++i) {
        double r = V[i], ux = V[nx + i] / r, uy = V[2 * nx + i] / r, uz = V[3 * nx + i] / r;
        double th = (2.0 * V[4 * nx + i] / r - (ux * ux + uy * uy + uz * uz)) / 3.0;
        if (!(r > 0) || !(th > 0)) bad = 1;
        U[i] = r;
        U[nx + i] = ux;
        U[2 * nx + i] = uy;
        U[3 * nx + i] = uz;
        U[4 * nx + i] = th;
    }
    return bad;
}

// Active instance range for the next launches (a copy from pageable memory:
// the value is staged before the call returns).
cudaError_t set_active(pr_force* b, int b0, int b1, cudaStream_t s)
{
    prk::Active a{b0, b1};
    return cudaMemcpyAsync(b->d_active, &a, sizeof a, cudaMemcpyHostToDevice, s);
}

}  // namespace

namespace prf {

void destroy(pr_force* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    fold_events(b);
    for (void* p : b->bufs) cudaFree(p);
    cudaFree(b->d_inst);
    cudaFree(b->d_active);
    cudaFree(b->d_cur);
    cudaFree(b->d_status);
    cudaFree(b->d_E);
    cudaFree(b->d_Ef);
    cudaFree(b->d_U);
    cudaFree(b->d_Ulift);
    cudaFree(b->d_vtab);
    cudaFree(b->d_tmp);
    cudaFree(b->d_part);
    cudaFree(b->d_fsync);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int create(pr_force** out, const pr_force_instance* inst, int n, int scheme, int precision, std::string& err)
{
    *out = nullptr;
    auto fail = [&](int code, const std::string& m) {
        err = m;
        return code;
    };
    if (!inst || n < 1 || n > 65535) return fail(PR_EINVAL, "need 1..65535 instances");
    if (scheme != PR_UPWIND && scheme != PR_MUSCL) return fail(PR_EINVAL, "bad scheme");
    if (precision != PR_FP64 && precision != PR_MIXED) return fail(PR_EINVAL, "bad precision");
    const pr_force_instance& d0 = inst[0];
    for (int k = 0; k < n; ++k) {
        const pr_force_instance& d = inst[k];
        if (d.nx != d0.nx || d.nvx != d0.nvx || d.nvp != d0.nvp)
            return fail(PR_EINVAL, "instances of one force batch share nx, nvx and nvp");
        if (d.nx < 1 || d.nx > 65535 || d.nvx < 2 || d.nvp < 1 || d.nvp > 32 || d.nvx > 4096)
            return fail(PR_EINVAL, "need 1 <= nx <= 65535, 2 <= nvx <= 4096, 1 <= nvp <= 32");
        if (!(d.L > 0) || !(d.x1 > d.x0) || !(d.dt > 0) || !(d.eps > 0))
            return fail(PR_EINVAL, "need L > 0, x1 > x0, dt > 0, eps > 0");
        if (d.bc < PR_BC_PERIODIC || d.bc > PR_BC_REFLECT) return fail(PR_EINVAL, "bad boundary condition");
        if (scheme == PR_MUSCL && d.bc == PR_BC_REFLECT && d.nx < 2)
            return fail(PR_EINVAL, "MUSCL with reflecting walls needs nx >= 2");
        if (d.E)
            for (int i = 0; i < d.nx; ++i)
                if (!std::isfinite(d.E[i])) return fail(PR_EINVAL, "E must be finite");
    }
    prepare_once();
    int C = default_cluster(precision, scheme, d0.nvx, d0.nvp);
    if (C == 0) return fail(PR_EINVAL, "velocity column too large for 16 CTAs of shared memory");
    pr_force* b = new pr_force();
    b->n = n;
    b->precision = precision;
    b->scheme = scheme;
    b->nx = d0.nx;
    b->nvx = d0.nvx;
    b->nvp = d0.nvp;
    geometry(precision, scheme, d0.nvx, d0.nvp, C, b->max_threads, &b->g, &b->smem);
    int clusters = 0;
    if (prk::force_step_occupancy(precision, scheme, b->g.vec, C, b->g.threads, b->smem, &clusters) != 0 ||
        clusters < 1) {
        destroy(b);
        return fail(PR_EINVAL, "no cluster of this shape fits the device");
    }
    const size_t es = elem(precision);
    const int nx = b->nx;
    const size_t state = (size_t)nx * b->g.ncol * es;
    const size_t vt = (vtab_bytes(b->nvx, b->nvp, es) + 255) / 256 * 256;
    auto cm = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cm((void**)&b->d_inst, sizeof(prk::FInst) * n) && cm((void**)&b->d_active, sizeof(prk::Active)) &&
              cm((void**)&b->d_cur, sizeof(int) * n) && cm((void**)&b->d_status, sizeof(int)) &&
              cm((void**)&b->d_E, sizeof(double) * n * nx) && cm((void**)&b->d_Ef, sizeof(float) * n * nx) &&
              cm((void**)&b->d_U, sizeof(double) * n * 5 * nx) &&
              cm((void**)&b->d_Ulift, sizeof(double) * n * 5 * nx) && cm(&b->d_vtab, vt * n);
    for (int k = 0; ok && k < 2 * n; ++k) {
        void* p = nullptr;
        ok = cm(&p, state);
        if (ok) b->bufs.push_back(p);
    }
    if (!ok) {
        destroy(b);
        cudaGetLastError();
        return fail(PR_ENOMEM, "device allocation of the force batch");
    }
    std::vector<double> E((size_t)n * nx, 0.0);
    std::vector<unsigned char> tabs(vt * n);
    b->h.resize(n);
    for (int k = 0; k < n; ++k) {
        const pr_force_instance& d = inst[k];
        prk::FInst& I = b->h[k];
        memset(&I, 0, sizeof I);
        if (d.E) memcpy(&E[(size_t)k * nx], d.E, sizeof(double) * nx);
        double em = 0.0;
        for (int i = 0; i < nx; ++i) em = std::max(em, std::fabs(E[(size_t)k * nx + i]));
        I.nx = nx;
        I.bc = d.bc;
        I.collide = std::isfinite(d.eps) ? 1 : 0;
        I.L = d.L;
        I.dx = (d.x1 - d.x0) / nx;
        I.dvx = 2.0 * d.L / b->nvx;
        I.dvp = 2.0 * d.L / b->nvp;
        I.dv3 = I.dvx * I.dvp * I.dvp;
        I.dt = d.dt;
        I.eps = d.eps;
        I.a = I.collide ? d.eps / (d.eps + d.dt) : 1.0;
        I.b = I.collide ? d.dt / (d.eps + d.dt) : 0.0;
        I.nu = d.dt / I.dx;
        I.nuv = d.dt / I.dvx;
        I.Emax = em;
        I.E = b->d_E + (size_t)k * nx;
        I.Ef = b->d_Ef + (size_t)k * nx;
        // the float32 step forms a f* + b M with float weights: the larger one
        // rounded to float32 and the smaller one 1 - larger (exact by
        // Sterbenz, the larger lying in [1/2, 1]), so that a + b = 1 holds for
        // the weights in use and the relaxation keeps the moments (Eq. 7)
        if (I.a >= I.b) {
            I.fa = (float)I.a;
            I.fb = 1.0f - I.fa;
        } else {
            I.fb = (float)I.b;
            I.fa = 1.0f - I.fb;
        }
        I.fnu = (float)I.nu;
        I.fnuv = (float)I.nuv;
        I.fEmax = (float)I.Emax;
        I.fdv3 = (float)I.dv3;
        I.f[0] = b->bufs[2 * k];
        I.f[1] = b->bufs[2 * k + 1];
        I.vtab = static_cast<unsigned char*>(b->d_vtab) + vt * k;
        I.vpair = es == sizeof(float)
                      ? reinterpret_cast<const float*>(static_cast<unsigned char*>(b->d_vtab) + vt * k +
                                                       vpair_offset(b->nvx, b->nvp, es))
                      : nullptr;
        I.Uin = b->d_Ulift + (size_t)k * 5 * nx;
        I.Uout = nullptr;
        I.Ucur = b->d_U + (size_t)k * 5 * nx;
        std::vector<unsigned char> t;
        if (precision == PR_FP64) fill_vtab<double>(t, b->nvx, b->nvp, d.L);
        else fill_vtab<float>(t, b->nvx, b->nvp, d.L);
        memcpy(&tabs[vt * k], t.data(), t.size());
        // first v_x row whose node, in the element type, is > 0 (the kernel
        // takes the upwind side from the same comparison)
        I.hpos = b->nvx;
        for (int j = 0; j < b->nvx; ++j) {
            bool pos = precision == PR_FP64 ? reinterpret_cast<const double*>(t.data())[j] > 0.0
                                            : reinterpret_cast<const float*>(t.data())[j] > 0.0f;
            if (pos) {
                I.hpos = j;
                break;
            }
        }
    }
    b->sums_ok.assign(n, 0);
    if (int Cf = default_fused_cluster(b)) {
        prk::FGeom g;
        size_t sm;
        if (fused_geometry(b, Cf, b->max_threads, b->march_req, &g, &sm)) {
            b->g = g;
            b->smem = sm;
        }
    }
    if (!ensure_partials(b)) {
        err = "fused-step partials: out of device memory";
        destroy(b);
        return PR_ENOMEM;
    }
    prk::Active all{0, n};
    std::vector<float> Ef(E.begin(), E.end());
    ok = cudaMemcpy(b->d_E, E.data(), sizeof(double) * E.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->d_Ef, Ef.data(), sizeof(float) * Ef.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->d_vtab, tabs.data(), tabs.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->d_inst, b->h.data(), sizeof(prk::FInst) * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->d_active, &all, sizeof all, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(b->d_cur, 0, sizeof(int) * n) == cudaSuccess &&
         cudaMemset(b->d_status, 0, sizeof(int)) == cudaSuccess &&
         cudaMemset(b->d_U, 0, sizeof(double) * n * 5 * nx) == cudaSuccess &&
         cudaMemset(b->d_Ulift, 0, sizeof(double) * n * 5 * nx) == cudaSuccess;
    for (void* p : b->bufs) ok = ok && cudaMemset(p, 0, state) == cudaSuccess;
    if (!ok || cudaDeviceSynchronize() != cudaSuccess) {
        err = std::string("force batch set-up: ") + cudaGetErrorString(cudaGetLastError());
        destroy(b);
        return PR_ECUDA;
    }
    *out = b;
    return PR_OK;
}

void bind(pr_force* b, int i, const double* Uin, double* Uout)
{
    b->h[i].Uin = Uin;
    b->h[i].Uout = Uout;
}

cudaError_t upload(pr_force* b, int b0, int b1, cudaStream_t s)
{
    if (b1 <= b0) return cudaSuccess;
    return cudaMemcpyAsync(b->d_inst + b0, b->h.data() + b0, sizeof(prk::FInst) * (b1 - b0), cudaMemcpyHostToDevice,
                           s);
}

// Steps of the active window [b0, b1): the fused step first makes the
// window's partials current (after a lift or a load) and ends with the
// moments of the final state from its partials.
static int enqueue_steps(pr_force* b, int b0, int b1, int nsteps, cudaStream_t s, bool timing)
{
    const int n_inst = b->n;
    const bool fused = b->g.march > 0;
    if (fused && nsteps > 0 && std::find(b->sums_ok.begin() + b0, b->sums_ok.begin() + b1, 0) != b->sums_ok.begin() + b1) {
        FCUDA(b, prk::launch_force_sums(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->g, b->nx, n_inst, b->d_active, b->d_cur, s));
        pr_internal_count_launches(1);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timing && nsteps > 0) {
        FCUDA(b, cudaEventCreate(&e0));
        FCUDA(b, cudaEventCreate(&e1));
        FCUDA(b, cudaEventRecord(e0, s));
    }
    if (fused_persistent(b, b1 - b0, nsteps)) {
        const long long walks = (b->nx + b->g.march - 1) / b->g.march;
        const long long items = (long long)(b1 - b0) * walks * b->g.C * nsteps;
        const int ctas = (int)std::min<long long>(fused_resident(b), items);
        FCUDA(b, prk::launch_force_fused_run(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->g, n_inst, b->d_active, b->d_cur, nsteps, b->d_fsync,
                                             b->fsync_words, b->d_status, b->smem, s, ctas));
        pr_internal_count_launches(1);
    } else {
        for (int k = 0; k < nsteps; ++k)
            FCUDA(b, prk::launch_force_step(b->precision == PR_FP64 ? 0 : 1, b->scheme, b->d_inst, b->g, b->nx,
                                            n_inst, b->d_active, b->d_cur, k, k == nsteps - 1, b->d_status, b->smem,
                                            s));
        pr_internal_count_launches(nsteps);
    }
    FCUDA(b, prk::launch_force_advance(b->d_active, b->d_cur, nsteps, n_inst, s));
    pr_internal_count_launches(nsteps & 1);
    if (e0) {
        FCUDA(b, cudaEventRecord(e1, s));
        b->pending.push_back({e0, e1, nsteps});
    }
    if (fused && nsteps > 0) {
        FCUDA(b, prk::launch_force_finalize(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->g, b->nx, n_inst, b->d_active, b->d_cur, s));
        pr_internal_count_launches(1);
    }
    std::fill(b->sums_ok.begin() + b0, b->sums_ok.begin() + b1, fused ? 1 : 0);
    return PR_OK;
}

int enqueue_run(pr_force* b, int b0, int b1, int nsteps, cudaStream_t s, bool timing)
{
    if (nsteps <= 0 || b1 <= b0) return PR_OK;
    FCUDA(b, set_active(b, b0, b1, s));
    int rc = enqueue_steps(b, b0, b1, nsteps, s, timing);
    FCUDA(b, set_active(b, 0, b->n, s));
    return rc;
}

int enqueue_lift_run(pr_force* b, int b0, int b1, int nsteps, cudaStream_t s, bool timing)
{
    if (b1 <= b0) return PR_OK;
    FCUDA(b, set_active(b, b0, b1, s));
    const int p = b->precision == PR_FP64 ? 0 : 1;
    FCUDA(b, b->lift_order == 1
                 ? prk::launch_force_lift_ce(p, b->d_inst, b->g, b->nx, b->n, b->d_active, b->d_cur, b->d_status, s)
                 : prk::launch_force_lift(p, b->d_inst, b->g, b->nx, b->n, b->d_active, b->d_cur, b->d_status, s));
    pr_internal_count_launches(1);
    std::fill(b->sums_ok.begin() + b0, b->sums_ok.begin() + b1, 0);
    int rc = PR_OK;
    if (nsteps > 0) {
        rc = enqueue_steps(b, b0, b1, nsteps, s, timing);
    } else {
        FCUDA(b, prk::launch_force_moments(p, b->d_inst, b->g, b->nx, b0, b1, b->d_cur, s));
        pr_internal_count_launches(1);
    }
    FCUDA(b, set_active(b, 0, b->n, s));
    return rc;
}

cudaError_t enqueue_graph_body(pr_force* b, const int* dk, int N, int nsteps, cudaStream_t s)
{
    const int p = b->precision == PR_FP64 ? 0 : 1;
    cudaError_t e = prk::launch_set_active(dk, b->d_active, 1, b->n, N, s);
    if (e == cudaSuccess)
        e = b->lift_order == 1
                ? prk::launch_force_lift_ce(p, b->d_inst, b->g, b->nx, b->n, b->d_active, b->d_cur, b->d_status, s)
                : prk::launch_force_lift(p, b->d_inst, b->g, b->nx, b->n, b->d_active, b->d_cur, b->d_status, s);
    const bool fused = b->g.march > 0 && nsteps > 0;
    if (e == cudaSuccess && fused) e = prk::launch_force_sums(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->g, b->nx, b->n, b->d_active, b->d_cur, s);
    if (fused && fused_persistent(b, b->n, nsteps)) {
        const long long walks = (b->nx + b->g.march - 1) / b->g.march;
        const long long items = (long long)b->n * walks * b->g.C * nsteps;
        const int ctas = (int)std::min<long long>(fused_resident(b), items);
        if (e == cudaSuccess)
            e = prk::launch_force_fused_run(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->g, b->n, b->d_active, b->d_cur, nsteps, b->d_fsync,
                                            b->fsync_words, b->d_status, b->smem, s, ctas);
    } else
        for (int k = 0; e == cudaSuccess && k < nsteps; ++k)
            e = prk::launch_force_step(p, b->scheme, b->d_inst, b->g, b->nx, b->n, b->d_active, b->d_cur, k,
                                       k == nsteps - 1, b->d_status, b->smem, s);
    if (e == cudaSuccess) e = prk::launch_force_advance(b->d_active, b->d_cur, nsteps, b->n, s);
    if (e == cudaSuccess && fused)
        e = prk::launch_force_finalize(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->g, b->nx, b->n, b->d_active, b->d_cur, s);
    std::fill(b->sums_ok.begin(), b->sums_ok.end(), 0);  // replays change the states behind the host's back
    return e;
}

int graph_body_launches(const pr_force* b, int nsteps)
{
    const bool fused = b->g.march > 0 && nsteps > 0;
    int n = 2 + (nsteps & 1);  // set-active, lift, advance
    if (fused) n += 2 + (fused_persistent(b, b->n, nsteps) ? 1 : nsteps);  // partials, steps, moments
    else n += nsteps;
    return n;
}

int take_status(pr_force* b)
{
    FCUDA(b, cudaStreamSynchronize(b->stream));
    fold_events(b);
    int st = 0;
    FCUDA(b, cudaMemcpy(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        prk::zero_now(b->d_status, sizeof(int), b->stream);
        return ffail(b, st,
                     st == PR_ENONPHYS   ? "a density or temperature became non-positive"
                     : st == PR_ETIMEOUT ? "a staging wait timed out"
                                         : "device status %d",
                     st);
    }
    return PR_OK;
}

double emax(const pr_force* b, int i) { return b->h[i].Emax; }

int launches_per_step() { return 1; }

}  // namespace prf

extern "C" {

int pr_force_create(pr_force** out, const pr_force_instance* inst, int n, int scheme, int precision)
{
    if (!out) return PR_EINVAL;
    std::string err;
    int rc = prf::create(out, inst, n, scheme, precision, err);
    if (rc) {
        std::lock_guard<std::mutex> lk(g_ferr_mu);
        g_ferr = err;
    }
    return rc;
}

int pr_force_destroy(pr_force* b)
{
    prf::destroy(b);
    return PR_OK;
}

const char* pr_force_last_error(const pr_force* b)
{
    if (!b) return g_ferr.c_str();
    return b->err.c_str();
}

int pr_force_set_initial(pr_force* b, int i, const double* U, int kind)
{
    if (!b) return PR_EINVAL;
    if (i < 0 || i >= b->n || !U) return ffail(b, PR_EINVAL, "bad instance index or null state");
    if (kind != PR_PRIMITIVE && kind != PR_CONSERVED) return ffail(b, PR_EINVAL, "bad kind");
    const int nx = b->nx;
    std::vector<double> V(5 * nx), P(5 * nx);
    if (kind == PR_PRIMITIVE) {
        memcpy(P.data(), U, sizeof(double) * 5 * nx);
        prim_to_cons(nx, U, V.data());
    } else {
        memcpy(V.data(), U, sizeof(double) * 5 * nx);
    }
    if (cons_to_prim(nx, V.data(), P.data())) return ffail(b, PR_ENONPHYS, "initial state has rho <= 0 or theta <= 0");
    cudaStream_t s = b->stream;
    FCUDA(b, cudaStreamSynchronize(s));
    double* dst = b->d_Ulift + (size_t)i * 5 * nx;
    FCUDA(b, prk::copy_now(dst, V.data(), sizeof(double) * 5 * nx, cudaMemcpyHostToDevice, s));
    prf::bind(b, i, dst, nullptr);
    FCUDA(b, prf::upload(b, i, i + 1, s));
    int rc = prf::enqueue_lift_run(b, i, i + 1, 0, s, false);
    if (rc) return rc;
    return prf::take_status(b);
}

int pr_force_set_f(pr_force* b, int i, const double* f)
{
    if (!b) return PR_EINVAL;
    if (i < 0 || i >= b->n || !f) return ffail(b, PR_EINVAL, "bad instance index or null f");
    const long long n = (long long)b->nx * b->g.ncol;
    cudaStream_t s = b->stream;
    FCUDA(b, cudaStreamSynchronize(s));
    if (!b->d_tmp && cudaMalloc(&b->d_tmp, sizeof(double) * n) != cudaSuccess) {
        cudaGetLastError();
        b->d_tmp = nullptr;
        return ffail(b, PR_ENOMEM, "staging buffer");
    }
    FCUDA(b, prk::copy_now(b->d_tmp, f, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    const int p = b->precision == PR_FP64 ? 0 : 1;
    FCUDA(b, prk::launch_force_load(p, b->d_inst, i, b->d_cur, b->d_tmp, n, s));
    b->sums_ok[i] = 0;
    FCUDA(b, prk::launch_force_moments(p, b->d_inst, b->g, b->nx, i, i + 1, b->d_cur, s));
    pr_internal_count_launches(2);
    return prf::take_status(b);
}

int pr_force_run(pr_force* b, int nsteps, void* stream)
{
    if (!b) return PR_EINVAL;
    if (nsteps < 0) return ffail(b, PR_EINVAL, "nsteps must be >= 0");
    cudaStream_t s = stream ? reinterpret_cast<cudaStream_t>(stream) : b->stream;
    return prf::enqueue_run(b, 0, b->n, nsteps, s, true);
}

int pr_force_moments(pr_force* b, int i, int kind, double* out)
{
    if (!b) return PR_EINVAL;
    if (i < 0 || i >= b->n || !out) return ffail(b, PR_EINVAL, "bad instance index or null output");
    if (kind != PR_PRIMITIVE && kind != PR_CONSERVED) return ffail(b, PR_EINVAL, "bad kind");
    FCUDA(b, cudaDeviceSynchronize());
    std::vector<double> V(5 * b->nx);
    FCUDA(b, cudaMemcpy(V.data(), b->d_U + (size_t)i * 5 * b->nx, sizeof(double) * V.size(), cudaMemcpyDeviceToHost));
    int rc = prf::take_status(b);
    if (kind == PR_CONSERVED) memcpy(out, V.data(), sizeof(double) * V.size());
    else cons_to_prim(b->nx, V.data(), out);
    return rc;
}

int pr_force_get_f(pr_force* b, int i, double* out)
{
    if (!b) return PR_EINVAL;
    if (i < 0 || i >= b->n || !out) return ffail(b, PR_EINVAL, "bad instance index or null output");
    const long long n = (long long)b->nx * b->g.ncol;
    FCUDA(b, cudaDeviceSynchronize());
    if (!b->d_tmp && cudaMalloc(&b->d_tmp, sizeof(double) * n) != cudaSuccess) {
        cudaGetLastError();
        b->d_tmp = nullptr;
        return ffail(b, PR_ENOMEM, "staging buffer");
    }
    FCUDA(b, prk::launch_force_store(b->precision == PR_FP64 ? 0 : 1, b->d_inst, i, b->d_cur, b->d_tmp, n,
                                     b->stream));
    pr_internal_count_launches(1);
    FCUDA(b, cudaStreamSynchronize(b->stream));
    FCUDA(b, cudaMemcpy(out, b->d_tmp, sizeof(double) * n, cudaMemcpyDeviceToHost));
    return prf::take_status(b);
}

int pr_force_sync(pr_force* b)
{
    if (!b) return PR_EINVAL;
    return prf::take_status(b);
}

int pr_force_set_lift_order(pr_force* b, int order)
{
    if (!b) return PR_EINVAL;
    if (order != 0 && order != 1) return ffail(b, PR_EINVAL, "lift order must be 0 or 1");
    if (order == 1)
        for (const prk::FInst& I : b->h)
            if (!I.collide) return ffail(b, PR_EINVAL, "the first-order lift needs a finite eps");
    b->lift_order = order;
    return PR_OK;
}

int pr_force_config(const pr_force* b, int* cluster, int* chunk)
{
    if (!b) return PR_EINVAL;
    if (cluster) *cluster = b->g.C;
    if (chunk) *chunk = b->g.rows * b->nvp * b->nvp;
    return PR_OK;
}

// Geometry for C CTAs per column with the requested walk (-1 automatic, 0
// clustered step): the fused step where it applies, else the clustered one;
// false (with a message) when neither fits.
static bool pick_geometry(pr_force* b, int C, int max_threads, int walk_req, prk::FGeom* g, size_t* sm)
{
    if (walk_req != 0 && fused_geometry(b, C, max_threads, walk_req, g, sm)) return true;
    if (walk_req >= 1) {
        ffail(b, PR_EINVAL, "the fused step does not apply to this geometry");
        return false;
    }
    if (!geometry(b->precision, b->scheme, b->nvx, b->nvp, C, max_threads, g, sm)) {
        ffail(b, PR_EINVAL, "no layout with %d CTAs of at most %d threads for this column", C, max_threads);
        return false;
    }
    int clusters = 0;
    if (prk::force_step_occupancy(b->precision, b->scheme, g->vec, C, g->threads, *sm, &clusters) != 0 ||
        clusters < 1) {
        ffail(b, PR_EINVAL, "no cluster of %d CTAs fits the device", C);
        return false;
    }
    return true;
}

// Switch to geometry g once the stream has drained: the partials follow the
// fused step's geometry and the descriptors are uploaded again.
static int apply_geometry(pr_force* b, const prk::FGeom& g, size_t sm)
{
    FCUDA(b, cudaStreamSynchronize(b->stream));
    const prk::FGeom old = b->g;
    const size_t old_sm = b->smem;
    b->g = g;
    b->smem = sm;
    if (!ensure_partials(b)) {
        b->g = old;
        b->smem = old_sm;
        return ffail(b, PR_ENOMEM, "fused-step partials: out of device memory");
    }
    std::fill(b->sums_ok.begin(), b->sums_ok.end(), 0);
    FCUDA(b, prf::upload(b, 0, b->n, b->stream));
    FCUDA(b, cudaStreamSynchronize(b->stream));
    return PR_OK;
}

int pr_force_set_cluster(pr_force* b, int cluster)
{
    if (!b) return PR_EINVAL;
    prk::FGeom g;
    size_t sm;
    // an explicit walk that does not apply to the new size falls back to the clustered step
    if (!pick_geometry(b, cluster, b->max_threads, b->march_req, &g, &sm) &&
        (b->march_req < 1 || !pick_geometry(b, cluster, b->max_threads, 0, &g, &sm)))
        return PR_EINVAL;
    return apply_geometry(b, g, sm);
}

int pr_force_set_threads(pr_force* b, int threads)
{
    if (!b) return PR_EINVAL;
    if (threads < 32 || threads > 1024 || threads % 32) return ffail(b, PR_EINVAL, "threads must be 32..1024, a multiple of 32");
    prk::FGeom g;
    size_t sm;
    if (!pick_geometry(b, b->g.C, threads, b->march_req, &g, &sm) &&
        (b->march_req < 1 || !pick_geometry(b, b->g.C, threads, 0, &g, &sm)))
        return PR_EINVAL;
    int rc = apply_geometry(b, g, sm);
    if (rc == PR_OK) b->max_threads = threads;
    return rc;
}

int pr_force_set_march(pr_force* b, int columns)
{
    if (!b) return PR_EINVAL;
    if (columns < -1) return ffail(b, PR_EINVAL, "columns must be -1, 0 or a walk length");
    prk::FGeom g;
    size_t sm;
    if (!pick_geometry(b, b->g.C, b->max_threads, columns, &g, &sm)) return PR_EINVAL;
    int rc = apply_geometry(b, g, sm);
    if (rc == PR_OK) b->march_req = columns;
    return rc;
}

int pr_force_set_persistent(pr_force* b, int mode)
{
    if (!b) return PR_EINVAL;
    if (mode < -1 || mode > 1) return ffail(b, PR_EINVAL, "mode must be -1, 0 or 1");
    FCUDA(b, cudaStreamSynchronize(b->stream));
    b->persist_req = mode;
    return PR_OK;
}

int pr_force_get_persistent(const pr_force* b, int nsteps, int* on)
{
    if (!b || !on) return PR_EINVAL;
    *on = fused_persistent(b, b->n, nsteps) ? 1 : 0;
    return PR_OK;
}

int pr_force_get_march(const pr_force* b, int* columns)
{
    if (!b || !columns) return PR_EINVAL;
    *columns = b->g.march;
    return PR_OK;
}

int pr_force_kernel_time(pr_force* b, double* avg_ms, int* steps, int reset)
{
    if (!b) return PR_EINVAL;
    FCUDA(b, cudaStreamSynchronize(b->stream));
    fold_events(b);
    if (avg_ms) *avg_ms = b->steps_timed ? b->step_ms_sum / b->steps_timed : 0.0;
    if (steps) *steps = b->steps_timed;
    if (reset) {
        b->step_ms_sum = 0.0;
        b->steps_timed = 0;
    }
    return PR_OK;
}

int pr_force_inject_wait_timeout(pr_force* b, int wait_ms)
{
    if (!b) return PR_EINVAL;
    if (!b->g.bulk || wait_ms < 1) return ffail(b, PR_EINVAL, "needs bulk-copy staging and wait_ms >= 1");
    cudaStream_t s = b->stream;
    FCUDA(b, cudaStreamSynchronize(s));
    FCUDA(b, set_active(b, 0, b->n, s));
    if (b->g.march > 0) {  // the fused step reads the partials of the current states
        FCUDA(b, prk::launch_force_sums(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->g, b->nx, b->n, b->d_active, b->d_cur, s));
        pr_internal_count_launches(1);
    }
    if (b->g.march > 0 && b->persist_req == 1) {
        // a two-step persistent run whose step-1 dependency waits run out
        const long long walks = (b->nx + b->g.march - 1) / b->g.march;
        const int ctas = (int)std::min<long long>(fused_resident(b), 2LL * b->n * walks * b->g.C);
        FCUDA(b, prk::launch_force_fused_run(b->precision == PR_FP64 ? 0 : 1, b->d_inst, b->g, b->n, b->d_active, b->d_cur, 2, b->d_fsync,
                                             b->fsync_words, b->d_status, b->smem, s, ctas,
                                             (long long)wait_ms * 1000000LL, 1));
        pr_internal_count_launches(1);
    } else {
        FCUDA(b, prk::launch_force_step(b->precision == PR_FP64 ? 0 : 1, b->scheme, b->d_inst, b->g, b->nx, b->n,
                                        b->d_active, b->d_cur, 0, 1, b->d_status, b->smem, s,
                                        (long long)wait_ms * 1000000LL, 1));
        FCUDA(b, prk::launch_force_advance(b->d_active, b->d_cur, 1, b->n, s));
        pr_internal_count_launches(2);
    }
    std::fill(b->sums_ok.begin(), b->sums_ok.end(), 0);
    return prf::take_status(b);
}

int pr_force_dt_stab(const pr_force_instance* inst, double cfl, double* dt)
{
    if (!inst || !dt || inst->nx < 1 || inst->nvx < 1 || !(inst->L > 0) || !(inst->x1 > inst->x0) || !(cfl > 0))
        return PR_EINVAL;
    *dt = dt_stab(*inst, cfl);
    return PR_OK;
}

// Time candidate step layouts on the current states and keep the fastest:
// every CTA count per column for which the fused step applies, each with the
// automatic walk and half and twice it, and the clustered step at its
// default cluster size.  Each candidate runs nsteps steps twice from the
// saved states (CUDA events on the stream, the second run counts); the
// states and moments are restored afterwards.
int pr_force_autotune(pr_force* b, int nsteps)
{
    if (!b) return PR_EINVAL;
    if (nsteps < 1) return ffail(b, PR_EINVAL, "nsteps must be >= 1");
    cudaStream_t s = b->stream;
    FCUDA(b, cudaStreamSynchronize(s));
    int rc = prf::take_status(b);
    if (rc) return rc;
    const size_t state = (size_t)b->nx * b->g.ncol * elem(b->precision);
    std::vector<int> cur(b->n);
    FCUDA(b, cudaMemcpy(cur.data(), b->d_cur, sizeof(int) * b->n, cudaMemcpyDeviceToHost));
    void* save = nullptr;
    double* saveU = nullptr;
    if (cudaMalloc(&save, state * b->n) != cudaSuccess || cudaMalloc(&saveU, sizeof(double) * 5 * b->nx * b->n) != cudaSuccess) {
        cudaFree(save);
        cudaGetLastError();
        return ffail(b, PR_ENOMEM, "autotune needs %zu bytes of scratch", state * b->n);
    }
    auto copy_states = [&](bool to_save) -> cudaError_t {
        for (int i = 0; i < b->n; ++i) {
            char* sv = static_cast<char*>(save) + state * i;
            void* f = b->bufs[2 * i + cur[i]];
            cudaError_t e = to_save ? prk::copy_now(sv, f, state, cudaMemcpyDeviceToDevice, s)
                                    : prk::copy_now(f, sv, state, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
        }
        const size_t ub = sizeof(double) * 5 * b->nx * b->n;
        cudaError_t e = to_save ? prk::copy_now(saveU, b->d_U, ub, cudaMemcpyDeviceToDevice, s)
                                : prk::copy_now(b->d_U, saveU, ub, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = prk::copy_now(b->d_cur, cur.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, s);
        return e;
    };
    struct Cand {
        prk::FGeom g;
        size_t sm;
    };
    std::vector<Cand> cands;
    auto add = [&](const prk::FGeom& g, size_t sm) {
        for (const Cand& c : cands)
            if (c.g.C == g.C && c.g.march == g.march) return;
        cands.push_back({g, sm});
    };
    for (int C = 1; C <= prk::FORCE_MAX_CLUSTER; ++C) {
        prk::FGeom g;
        size_t sm;
        if (!fused_geometry(b, C, b->max_threads, -1, &g, &sm) &&
            !fused_geometry(b, C, b->max_threads, std::min(8, b->nx), &g, &sm))
            continue;
        add(g, sm);
        const int S0 = g.march;
        for (int S : {std::max(1, S0 / 2), std::min(b->nx, 2 * S0)}) {
            prk::FGeom g2;
            size_t sm2;
            if (fused_geometry(b, C, b->max_threads, S, &g2, &sm2)) add(g2, sm2);
        }
    }
    {
        const int Cd = default_cluster(b->precision, b->scheme, b->nvx, b->nvp);
        prk::FGeom g;
        size_t sm;
        if (Cd > 0 && pick_geometry(b, Cd, b->max_threads, 0, &g, &sm)) add(g, sm);
    }
    const prk::FGeom g_old = b->g;
    const size_t sm_old = b->smem;
    const int march_old = b->march_req;
    double best_ms = 1e300;
    int best = -1;
    cudaError_t ce = copy_states(true);
    for (size_t ci = 0; ci < cands.size() && ce == cudaSuccess && rc == PR_OK; ++ci) {
        if (apply_geometry(b, cands[ci].g, cands[ci].sm) != PR_OK) continue;  // e.g. no room for its partials
        double ms = 0.0;
        for (int rep = 0; rep < 2 && rc == PR_OK; ++rep) {
            if ((ce = copy_states(false)) != cudaSuccess) break;
            std::fill(b->sums_ok.begin(), b->sums_ok.end(), 0);
            fold_events(b);
            b->step_ms_sum = 0.0;
            b->steps_timed = 0;
            rc = prf::enqueue_run(b, 0, b->n, nsteps, s, true);
            if (rc == PR_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = ffail(b, PR_ECUDA, "autotune run");
            if (rc == PR_OK) rc = prf::take_status(b);
            fold_events(b);
            ms = b->steps_timed ? b->step_ms_sum / b->steps_timed : 1e300;
        }
        if (rc == PR_OK && ms < best_ms) {
            best_ms = ms;
            best = (int)ci;
        }
    }
    b->step_ms_sum = 0.0;
    b->steps_timed = 0;
    int rc2 = best >= 0 ? apply_geometry(b, cands[best].g, cands[best].sm) : apply_geometry(b, g_old, sm_old);
    if (rc2 == PR_OK) b->march_req = best >= 0 ? cands[best].g.march : march_old;
    if (ce == cudaSuccess) ce = copy_states(false);
    std::fill(b->sums_ok.begin(), b->sums_ok.end(), 0);
    cudaFree(save);
    cudaFree(saveU);
    if (ce != cudaSuccess) return ffail(b, PR_ECUDA, "autotune state copies: %s", cudaGetErrorString(ce));
    if (rc) return rc;
    if (rc2) return rc2;
    FCUDA(b, cudaStreamSynchronize(s));
    return PR_OK;
}

}  // extern "C"
