// Device-side descriptors and launch wrappers shared by the kernels (fine.cu,
// coarse.cu) and the host runtime (runtime.cu).  Internal to libpr.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace prk {

constexpr int THREADS = 256;             // threads per fine-step CTA
constexpr int VPT = 4;                   // velocities per thread (one 16-byte f32 vector)
constexpr int CHUNK = THREADS * VPT;     // velocities per work item
constexpr int WARPS = THREADS / 32;
constexpr int MAXDEP = 8;                // neighbour tiles an item may wait on
constexpr int MAX_TX = 64;               // largest tile width (x cells per item)

constexpr long long WAIT_LIMIT_NS = 4000000000LL;  // a dependency wait gives up after 4 s
constexpr int ST_OK = 0;
constexpr int ST_TIMEOUT = -4;           // = PR_ETIMEOUT
constexpr int ST_NONPHYS = -5;           // = PR_ENONPHYS

// Static description of one fine-solve instance (written once by the host).
struct Inst {
    int nx, nv, nv3, ldv;      // ldv: column stride of f in elements (multiple of 4)
    int bc, scheme;
    int tx, n_xt, n_vc;        // tile width, x tiles, v chunks of CHUNK velocities
    int pad0;
    double L, dv, dv3, dx, dt, eps;
    double a, b;               // f^{n+1} = a f* + b M  (a = eps/(eps+dt), b = dt/(eps+dt))
    double nu;                 // dt/dx
    void* g[2];                // stored transported state f* (T*), [nx][ldv], ping-pong
    void* tab[2];              // Maxwellian factor tables (T*), [nx][3][nv]
    double* part;              // velocity-chunk partial moments [nx][n_vc][5]
    double* Ucur;              // conserved moments of the current state [5][nx]
    const double* Uin;         // lift source, conserved [5][nx] (device)
    double* Uout;              // projection destination after the last step (or null)
    unsigned int* done;        // [n_xt] last finalised step of each tile (reset per launch)
    unsigned int* arrive;      // [n_xt] arrivals of v chunks in the current step
    const int* deps;           // [n_xt][MAXDEP] tiles an item must wait on (-1 padded)
    long long item0;           // prefix: first item of this instance within a step
    double* trace;             // float64 only, or null: f* of step s of a launch at [s-1][nx][ldv]
    double* trace_m;           // float64 only, or null: its moment sums (grid units) at [s-1][nx][5]
};

// Per-instance dynamic state, updated on the device between launches.
struct InstState {
    int cur;                   // buffer index of the state at launch start
    int pad;
    double a0;                 // weight of g in that state (0 after a lift, 1 after set_f)
};

// Work range of one launch.
struct Active {
    int begin, end;            // instances [begin, end)
};

// ---- fine propagator (fine.cu) ----
// Persistent fused fine-step kernel over the active instances for nsteps steps.
// vpt: velocities per thread (4, or 8 in float32 when every nv is a multiple
// of 8); the CTA has CHUNK / vpt threads.
// wait_ns: limit of each dependency wait (<= 0: no waits, for one-step launches);
// poison = 1 makes the items of step 2 wait for a step that never completes
// (failure-detection check: the wait runs out and the launch reports PR_ETIMEOUT).
cudaError_t launch_fine_run(int precision, int scheme, int vpt, const Inst* insts, InstState* st,
                            const long long* prefix, const Active* active, int nsteps,
                            unsigned long long* ticket, int* status, long long wait_ns, int grid,
                            size_t smem, cudaStream_t s, int poison = 0);
int fine_run_occupancy(int precision, int scheme, int vpt, size_t smem, int* blocks_per_sm);
size_t fine_run_smem(int precision, int vpt, int tx, int nv, int H);

// Cluster-resident fine run (float32 f, nv = 8 or 16): one thread-block
// cluster of C CTAs per active instance, w x cells per CTA, keeps the
// instance in shared memory for lift (from Uin), nsteps steps and the
// projection into Uout (and Ucur).  The batch's g, tab and state are not used.
bool fine_cluster_plan(int nx, int nv, int max_smem, int* C, int* w, size_t* smem);
int fine_cluster_resident(int scheme, int nv, int C, size_t smem);  // co-resident clusters
cudaError_t launch_fine_cluster(int scheme, int nv, const Inst* insts, const Active* active, int n_inst_max,
                                int nsteps, int C, int w, size_t smem, int* status, cudaStream_t s);

// Set the dynamic shared-memory limit of the kernels (called once).
void prepare_fine_kernels(int max_smem);
void prepare_coarse_kernels(int max_smem);

// Lift (Eq. 17) into tab[cur], Ucur; st.a0 = 0. One CTA per (active instance, tile).
cudaError_t launch_lift(int precision, const Inst* insts, InstState* st, const Active* active,
                        int max_tiles, int n_inst_max, size_t smem, int* status, cudaStream_t s);
size_t lift_smem(int precision, int tx, int nv);

// After a run: cur <- (cur + nsteps) & 1, a0 <- a.
cudaError_t launch_advance(const Inst* insts, InstState* st, const Active* active, int nsteps,
                           int n_inst_max, cudaStream_t s);

// Materialise f = a0 g + M into out (double) [nx][nv3] for instance b.
cudaError_t launch_materialize(int precision, const Inst* insts, const InstState* st, int b,
                               const Inst& hinst, double* out, cudaStream_t s);

// Load f (double) into g[cur] of instance b, zero its tables, a0 = 1, Ucur = P(f).
cudaError_t launch_set_f(int precision, const Inst* insts, InstState* st, int b,
                         const Inst& hinst, const double* f, cudaStream_t s);

// ---- adjoint of the float64 upwind fine run (adjoint.cu) ----
cudaError_t adj_seed(const Inst& I, const double* lamV, double* lam, cudaStream_t s);
// One reverse step: lam_out = T^T (a lam_in + b dv^3 (c0 + c.v + c4 |v|^2)),
// the coefficients from the moments of the step's transported state g.
cudaError_t adj_step(const Inst& I, const double* lam_in, const double* g, const double* msum, double* coef,
                     double* eps_acc, double* lam_out, cudaStream_t s);
cudaError_t adj_lift(const Inst& I, const double* lam, const double* Uin, double* dU0, cudaStream_t s);

// ---- fine propagator with an exterior force (force.cu) ----
constexpr int FORCE_THREADS = 256;       // threads per CTA of the force kernels
constexpr int FORCE_MAX_CLUSTER = 16;    // CTAs per x column (8 portable, 16 opt-in)
constexpr int FORCE_MAX_CHUNK_BYTES = 96 * 1024;  // f* of one CTA's v_x rows, staged in shared memory

// One instance of the force path.  f[buf] is [nx][ncol] of T (float or double).
struct FInst {
    int nx, bc, collide;
    int hpos;                  // first v_x row whose node is > 0 (in the element type)
    double L, dx, dvx, dvp, dv3, dt, eps;
    double a, b;               // f^{n+1} = a f* + b M
    double nu, nuv;            // dt/dx, dt/dv_x
    double Emax;               // max_i |E_i|
    const double* E;           // [nx] exterior force at the cell centres (device)
    const float* Ef;           // the same in float (the float path converts nothing per thread)
    float fa, fb, fnu, fnuv, fEmax, fdv3;
    void* f[2];                // ping-pong state
    void* part[2];             // fused step: column sums of f[k], [nx][C][17], double-float (float) or double
    const void* vtab;          // T: v_x[nvx], v_y[nvp2], v_z[nvp2], v_y^2+v_z^2[nvp2]
    const float* vpair;        // float path: the nodes as float pairs, v_x[nvx][2], v_p[nvp][2]
    const double* Uin;         // lift source, conserved [5][nx] (device) or null
    double* Uout;              // projection destination after the last step (or null)
    double* Ucur;              // conserved moments of the current state [5][nx]
};

// Geometry shared by the instances of one force batch.
struct FGeom {
    int nvx, nvp;
    long long ncol;            // nvx * nvp^2
    int C;                     // CTAs (cluster size) per x column
    int rows;                  // v_x rows per CTA (the last CTA may have fewer)
    int vec;                   // (v_y, v_z) cells per thread: 16 bytes when bulk, else 1
    int groups;                // row groups per CTA (nvp^2/vec threads each)
    int threads;               // threads per CTA of the step kernel
    int bulk;                  // rows are 16-byte multiples: stage them with bulk copies
    int buf_off;               // shared-memory offset of the staging buffers
    int march;                 // > 0: fused single-pass step, a CTA walks this many x columns; 0: clustered step
    int scheme;                // x fluxes: 0 upwind, 1 MUSCL-minmod
};

cudaError_t prepare_force_kernels(int max_smem);
size_t force_step_smem(int precision, int scheme, int nvx, int nvp, int rows);
size_t force_step_buf_off(int precision, int nvx, int nvp);
// The fused single-pass step (upwind or MUSCL, 16-byte lanes, <= 256
// threads; float or double): its shared memory for a walk of `walk` columns,
// whether geometry g can use it (MUSCL: at most force_fused_muscl_rows v_x
// rows per thread), the partials it keeps per column (8 bytes each), and its
// resident CTAs per SM.
size_t force_fused_smem(int precision, int scheme, int nvp, int rows, int walk);
bool force_fused_fits(int precision, int scheme, const FGeom& g);
int force_fused_muscl_rows(int precision);
int force_partials_per_column(const FGeom& g);
int force_fused_occupancy(int precision, int scheme, int threads, size_t smem, int* per_sm);
// All nsteps fused steps of the active instances in one persistent launch of
// `ctas` CTAs (at most the resident count); sync (sync_words ints: a ticket
// and one done count per instance and walk) is zeroed on the stream first.
cudaError_t launch_force_fused_run(int precision, const FInst* insts, const FGeom& g, int n_inst, const Active* act,
                                   int* cur, int nsteps, int* sync, int sync_words, int* status, size_t smem,
                                   cudaStream_t s, int ctas, long long wait_ns = WAIT_LIMIT_NS, int poison = 0);
// Partials of the current state of the active instances (fused step input).
cudaError_t launch_force_sums(int precision, const FInst* insts, const FGeom& g, int nx, int n_inst,
                              const Active* act, const int* cur, cudaStream_t s);
// Ucur / Uout of the active instances from the partials of their current state.
cudaError_t launch_force_finalize(int precision, const FInst* insts, const FGeom& g, int nx, int n_inst,
                                  const Active* act, const int* cur, cudaStream_t s);
void force_step_layout(int nvp, int vec, int rows, int max_threads, int* groups, int* threads);
size_t force_lift_smem(int precision, int nvx, int nvp);
// Resident clusters of C CTAs of the clustered step kernel.
int force_step_occupancy(int precision, int scheme, int vec, int C, int threads, size_t smem, int* clusters);
// One fine step of every active instance; input buffer cur[b] ^ (step & 1);
// last != 0 also writes P(f^{n+1}) into Ucur (and Uout).
// Each CTA stages its input rows with bulk copies and waits on an mbarrier
// for at most wait_ns (then PR_ETIMEOUT).  poison = 1 adds a wait on a second
// mbarrier that no copy completes (failure-detection check: PR_ETIMEOUT).
cudaError_t launch_force_step(int precision, int scheme, const FInst* insts, const FGeom& g, int nx, int n_inst,
                              const Active* act, int* cur, int step, int last, int* status, size_t smem,
                              cudaStream_t s, long long wait_ns = WAIT_LIMIT_NS, int poison = 0);
// Lift Uin into f[0] of the active instances, cur <- 0.
cudaError_t launch_force_lift(int precision, const FInst* insts, const FGeom& g, int nx, int n_inst,
                              const Active* act, int* cur, int* status, cudaStream_t s);
cudaError_t launch_force_moments(int precision, const FInst* insts, const FGeom& g, int nx, int b0, int b1,
                                 const int* cur, cudaStream_t s);
cudaError_t launch_force_load(int precision, const FInst* insts, int b, const int* cur, const double* src,
                              long long n, cudaStream_t s);
cudaError_t launch_force_store(int precision, const FInst* insts, int b, const int* cur, double* dst,
                               long long n, cudaStream_t s);
// cur[b] ^= nsteps & 1 for the active instances (after a run of nsteps steps).
cudaError_t launch_force_advance(const Active* act, int* cur, int nsteps, int n_inst, cudaStream_t s);
cudaError_t launch_force_set_cur(int* cur, int b, int v, cudaStream_t s);

// ---- first-order (Chapman-Enskog) lifting, Def. 3 with L = 1 (lift_ce.cu) ----
// E = 0 path: g[cur] = M (1 - eps P(c)) from Uin, tab[cur] = 0, a0 = 1 for
// the active instances (grid over nx_max cells); with_moments also writes
// P(f) into Ucur.
cudaError_t launch_lift_ce(int precision, const Inst* insts, InstState* st, const Active* active, int nx_max,
                           int n_inst_max, int with_moments, int* status, cudaStream_t s);
// Force path: f[0] of the active instances, cur <- 0.
cudaError_t launch_force_lift_ce(int precision, const FInst* insts, const FGeom& g, int nx, int n_inst,
                                 const Active* act, int* cur, int* status, cudaStream_t s);

// ---- coarse propagator and parareal sweep (coarse.cu) ----
struct CoarseParams {
    int nx, bc, sound;
    double x0, x1, dx, cfl;
    const double* E = nullptr; // exterior force [nx] (device) or null: source (0, rho E, 0, 0, rho u_x E)
    double visc = 0.0;         // Knudsen number of the Navier-Stokes model (Eq. 8); 0: Euler
};

// G over dT for one state (Vin/Vout device [5][nx], may alias).
cudaError_t launch_coarse(const CoarseParams& p, const double* Vin, double* Vout, double dT,
                          double* work, int* status, cudaStream_t s);

// Sequential sweep of Algorithm 2 for n = k..N (k read from *dk on the device):
//   Gv = G(U[n-1]); U[n] = Gv + (k > 0 ? PFL[n] - Gs[n] : 0); Gs[n] = Gv;
//   err[k] = max |U[n]_new - U[n]_old|.  Then *dk <- k + 1 if bump.
// Doubles of global workspace a coarse step needs when its state does not fit
// shared memory (state, next state, per-cell cache).
size_t coarse_work_doubles(int nx);
cudaError_t launch_sweep(const CoarseParams& p, int N, double dT, const int* dk, double* U,
                         const double* PFL, double* Gs, double* err, double* work, int* status,
                         int bump, int* dk_mut, cudaStream_t s);

// Active range for the parareal fine phase: instances [k-1, N) -> wave window.
cudaError_t launch_set_active(const int* dk, Active* active, int first_slice, int n_inst,
                              int N, cudaStream_t s);
// Lockstep problems sharing one batch: slices nidx[i] (ascending) for
// i < n_sl, independent instances after them; run / lift ranges from k.
cudaError_t launch_set_active_multi(const int* dk, const int* nidx, int n_sl, int n_inst, Active* run, Active* lift,
                                    cudaStream_t s);

// Host copy that is complete when it returns and ordered after the work
// already queued on stream s.  A plain cudaMemcpy from pageable host memory,
// or between device buffers, may return before its transfer lands, and the
// transfer runs on the legacy default stream, which the runtime's
// non-blocking streams neither wait for nor hold back: a kernel queued next on
// s could read the buffer before the data arrives.
inline cudaError_t copy_now(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s)
{
    if (bytes == 0) return cudaSuccess;
    const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, s);
    return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
}

// cudaMemset's counterpart: zeroes ordered after the work queued on s and
// complete when it returns.
inline cudaError_t zero_now(void* dst, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) return cudaSuccess;
    const cudaError_t e = cudaMemsetAsync(dst, 0, bytes, s);
    return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
}

}  // namespace prk
