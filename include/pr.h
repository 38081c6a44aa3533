/*
 * libpr — GB300 (sm_103a) kinetic-fluid parareal library for the collisional
 * Vlasov-BGK equation in the hyperbolic scaling (alpha = 0), 1D in x and 3D in
 * v, after Laidin & Rey, arXiv 2502.02704: without a force field (E = 0, the
 * pr_init / pr_batch_* path) and with one (the pr_force_* / pr_init_force path).
 *
 * C ABI: every entry point takes plain pointers and sizes and returns an int
 * status (PR_OK = 0, negative on error).  Nothing aborts or exits.  Objects are
 * opaque and library-owned; the library allocates its own device memory
 * (cudaMalloc) when an object is created and frees it in the matching destroy
 * call.  Host arrays are caller-owned: they are read or written before the call
 * returns and never retained.  "stream" arguments are cudaStream_t values
 * passed as void*; NULL selects the object's own stream.  Calls that return
 * host data synchronise that stream.  Calls that only enqueue work report
 * device-side errors (time-outs, non-physical states) at the next synchronising
 * call on the same object.  Calls that upload host data into an object (initial
 * states, f, a resumed iterate, layouts) queue the copy on the object's own
 * stream ahead of the work they enqueue, so work queued next on that stream
 * sees the data; the host array may be reused as soon as the call returns.  A
 * caller that passes its own stream after calls that used the object's stream
 * (set-up, uploads) orders the two itself, e.g. with an event or a
 * synchronisation; the library does not join streams.
 *
 * Layouts (row-major, float64 unless stated):
 *   primitive state  U[5][nx] = (rho, u_x, u_y, u_z, theta)         (Def. 1)
 *   conserved state  V[5][nx] = (rho, rho u_x, rho u_y, rho u_z, E),
 *                    E = rho |u|^2 / 2 + 3 rho theta / 2             (Eq. 14)
 *   distribution     f[nx][nv^3], velocity index (jx*nv + jy)*nv + jz, nodes
 *                    v_j = -L + (j + 1/2) 2L/nv (cube centres, Sec. 3)
 * x cells are uniform on [x0, x1].  nv must be a multiple of 4 (the kernels move
 * four consecutive v_z nodes per 16-byte access).
 *
 * Readings of the paper that the library implements (same as its oracle):
 * upwind flux F_{i+1/2} = v+ f_i - v- f_{i+1} (Eq. 13 with v- = -min(v,0) and
 * the sign that makes it upwind); the 1/dx of Eq. (12) and dt/dx of Eq. (15);
 * BGK rate 1/eps (tau = 1 in Eq. 7); Rusanov flux (h_i + h_{i+1})/2 -
 * S (V_{i+1} - V_i)/2 on conserved V (Eq. 16); sound speed sqrt(5 theta/3) by
 * default; MUSCL = minmod slopes with forward-Euler time stepping; ghost
 * cells: periodic wrap, outflow copy, specular reflection with v_x reversed.
 */
#ifndef PR_H
#define PR_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define PR_OK 0
#define PR_EINVAL -1     /* bad argument or unsupported combination            */
#define PR_ENOMEM -2     /* device or host allocation failed                   */
#define PR_ECUDA -3      /* a CUDA runtime call failed (see pr_*_last_error)   */
#define PR_ETIMEOUT -4   /* a device-side wait ran out; the launch was aborted */
#define PR_ENONPHYS -5   /* a density or temperature became <= 0 or NaN        */
#define PR_ENOTCONV -6   /* parareal reached K iterations above the tolerance  */

/* ---- enumerations ---- */
#define PR_BC_PERIODIC 0
#define PR_BC_OUTFLOW 1  /* zero-gradient; the paper's "absorbing" walls        */
#define PR_BC_REFLECT 2  /* specular walls                                      */

#define PR_UPWIND 0      /* first-order upwind flux, Eq. (13)                   */
#define PR_MUSCL 1       /* minmod-limited slopes (flux limiter, Sec. 3.1)      */

#define PR_FP64 0        /* f, tables and all arithmetic in float64             */
#define PR_MIXED 1       /* f and its per-cell arithmetic in float32; velocity
                            moments beyond a warp, Maxwellian parameters,
                            projection and parareal sums in float64             */

#define PR_SOUND_GAMMA53 0     /* c = sqrt(5 theta / 3) in the Rusanov speed   */
#define PR_SOUND_SQRT_THETA 1  /* c = sqrt(theta) as printed below Eq. (16)    */

#define PR_PRIMITIVE 0
#define PR_CONSERVED 1

#define PR_COARSE_EULER 0      /* Euler system, Eqs. (14)-(16)                 */
#define PR_COARSE_CNS 1        /* compressible Navier-Stokes, Eq. (8): the Euler
                                  scheme plus viscous fluxes with mu = rho theta,
                                  kappa = 5 rho theta / 2 (first-order
                                  Chapman-Enskog coefficients of BGK, tau = 1),
                                  central face gradients, local steps also
                                  limited by dx^2 / (2 eps (5/3) max theta)    */

#define PR_FINE_AUTO 0         /* fine phase of a parareal iteration: chosen   */
#define PR_FINE_TILED 1        /* the persistent tiled kernel (any instance)   */
#define PR_FINE_CLUSTER 2      /* one thread-block cluster per slice, the slice
                                  kept in shared memory for all its steps
                                  (mixed precision, Maxwellian lifting, no
                                  force, nv = 8 or 16, small nx)               */

/* ---- parameter blocks ---- */
typedef struct {
    int nx;            /* x cells (>= 1)                                       */
    double x0, x1;     /* domain, x1 > x0                                      */
    int bc;            /* PR_BC_*                                              */
} pr_grid;

typedef struct {
    int nv;            /* velocity cells per direction, multiple of 4          */
    double L;          /* velocity box [-L, L]^3, L > 0                        */
} pr_velocity;

typedef struct {
    double T;          /* final time                                           */
    int n_slices;      /* N_g coarse slices (>= 1)                             */
    double cfl_f;      /* fine CFL: dt_stab = cfl_f dx / max|v_x| (Sec. 2.2)   */
    double cfl_g;      /* coarse CFL for the Rusanov local steps               */
    int scheme;        /* PR_UPWIND or PR_MUSCL                                */
    int precision;     /* PR_FP64 or PR_MIXED                                  */
    int sound_speed;   /* PR_SOUND_*                                           */
    int max_batch;     /* slices whose fine states are resident at once;
                          0 = all N (the fine phase runs in waves otherwise)  */
    int nf;            /* fine steps per slice; 0 = ceil(dT_g / dt_stab)       */
    int coarse_model;  /* PR_COARSE_EULER (0) or PR_COARSE_CNS                 */
    int lift_order;    /* 0: Maxwellian lifting (Def. 2); 1: first-order
                          lifting L^(1) of Def. 3, f = M (1 - eps P(c)) with the
                          Chapman-Enskog term of BGK, gradients of u and theta
                          by central differences through the ghosts           */
} pr_time;

/* One fine-solve instance of a batch (independent problem). */
typedef struct {
    int nx;
    double x0, x1;
    int bc;
    int nv;
    double L;
    double eps;        /* Knudsen number > 0; +INFINITY = collisionless        */
    double dt;         /* fine time step > 0                                   */
    int scheme;        /* PR_UPWIND or PR_MUSCL                                */
} pr_instance;

typedef struct pr_ctx pr_ctx;      /* one parareal problem (Algorithm 2)       */
typedef struct pr_batch pr_batch;  /* independent fine-solve instances         */
typedef struct pr_multi pr_multi;  /* problems iterated together in one launch  */

/* ======================= parareal problem (Sec. 2) ======================= */

/* Create a parareal problem: grid, velocity box, Knudsen number eps and the
 * time grid T^n = n T/N (Sec. 2.2).  Allocates every device buffer: N slice
 * states (or max_batch of them), the iterates U^{n,k} (conserved), the fine
 * results P F L(U^{n-1}) and the coarse results G(U^{n-1}).  *out is NULL on
 * failure.  Errors: PR_EINVAL, PR_ENOMEM, PR_ECUDA. */
int pr_init(pr_ctx** out, const pr_grid* g, const pr_velocity* v, double eps,
            const pr_time* t);

/* Free everything owned by ctx (NULL is accepted). */
int pr_destroy(pr_ctx* ctx);

/* Last error message of ctx, or of the last failed pr_init when ctx is NULL.
 * The string stays valid until the next call on ctx. */
const char* pr_last_error(const pr_ctx* ctx);

/* Set U^{0} from a host primitive state U0[5][nx] and run the first coarse
 * guess U^{n,0} = G(U^{n-1,0}), n = 1..N (Algorithm 2, before the loop).
 * Resets the iteration counter k to 0.  Synchronous.
 * Errors: PR_EINVAL, PR_ENONPHYS, PR_ECUDA. */
int pr_set_initial(pr_ctx* ctx, const double* U0);

/* Coarse propagator G (Eqs. 14-16) over a time dT >= 0 on host conserved
 * states Vin/Vout[5][nx] (may alias): explicit Rusanov updates with local steps
 * dt = min(cfl_g dx / max S, remaining).  Synchronous.
 * Errors: PR_EINVAL, PR_ENONPHYS, PR_ECUDA. */
int pr_coarse_step(pr_ctx* ctx, const double* Vin, double* Vout, double dT);

/* Advance the live distribution of slice n (1..N) by nsteps fine steps of
 * dt = (T/N)/n_f (Eqs. 11-13).  A slice without a live distribution is first
 * lifted (Eq. 17) from the current iterate U^{n-1}.  Enqueued on stream.
 * Errors: PR_EINVAL, PR_ECUDA (PR_ETIMEOUT/PR_ENONPHYS at the next sync). */
int pr_fine_step(pr_ctx* ctx, int slice, int nsteps, void* stream);

/* Moments (Eq. 18) of slice n's live distribution into host out[5][nx], kind
 * PR_PRIMITIVE or PR_CONSERVED.  Synchronous. */
int pr_fine_moments(pr_ctx* ctx, int slice, int kind, double* out);

/* Slice n's live distribution f[nx][nv^3] as float64 on the host. */
int pr_fine_get_f(pr_ctx* ctx, int slice, double* out);

/* One iteration of Algorithm 2 (k <- k+1): lift U^{n-1,k-1}, run n_f fine steps
 * and project for every slice n = k..N in one launch (the tiled persistent
 * kernel, or one cluster per slice: pr_set_fine_path), form
 * the jumps P F L(U^{n-1,k-1}) - G(U^{n-1,k-1}), then the sequential correction
 * U^{n,k} = G(U^{n-1,k}) + jump for n = k..N on the device.  *err_out (may be
 * NULL) receives max_n |U^{n,k} - U^{n,k-1}| over cells and the 5 conserved
 * components (Eq. 10).  Synchronous when err_out is not NULL.
 * Errors: PR_EINVAL (called before pr_set_initial), PR_ETIMEOUT, PR_ENONPHYS,
 * PR_ECUDA. */
int pr_parareal_iter(pr_ctx* ctx, double* err_out);

/* Iterate until k == K or the error drops below tol (tol <= 0: fixed K).
 * errs (may be NULL) receives one error per iteration run (length >= K);
 * *k_done the number of iterations run.  Iterations of the fixed-K loop are
 * replayed from one captured CUDA graph.  Returns PR_ENOTCONV when tol > 0 and
 * the last error is still >= tol (the iterates are valid). */
int pr_parareal_run(pr_ctx* ctx, int K, double tol, int* k_done, double* errs);

/* Current iterate U^{n,k} (n = 0..N) into host out[5][nx]. Synchronous. */
int pr_moments(pr_ctx* ctx, int n, int kind, double* out);

/* Number of fine steps per slice n_f and the fine step dt (either may be NULL). */
int pr_fine_steps_per_slice(const pr_ctx* ctx, int* nf, double* dt);

/* Iterations completed since pr_set_initial. */
int pr_iterations(const pr_ctx* ctx, int* k);

/* Parareal resume.  pr_save writes the state Algorithm 2 carries from one
 * iteration to the next (Sec. 2.2): the iterates U^{n,k} (n = 0..N), the
 * coarse values G(U^{n-1,k}) the next correction reuses, k and the errors of
 * the iterations run, with a header of the problem's sizes and settings (and
 * its force field), to the file at path (binary, host byte order; about
 * 80 (N+1) nx bytes).  pr_load reads such a file into a problem created with
 * the same sizes and settings (max_batch may differ): the next
 * pr_parareal_iter continues with iteration k+1 and gives the bits the
 * uninterrupted run gives.  Synchronous.  Errors: PR_EINVAL (called before
 * pr_set_initial (save), a file that cannot be opened or written, another
 * problem's file, a truncated file), PR_ENONPHYS (a loaded iterate with
 * rho <= 0, theta <= 0 or a non-finite value: nothing is changed), PR_ECUDA. */
int pr_save(pr_ctx* ctx, const char* path);
int pr_load(pr_ctx* ctx, const char* path);

/* ============ several parareal problems and instances per launch ============ */

/* Algorithm 2 for several problems at once (the batching of Sec. 2.2 across
 * problems): every slice of every problem (pr_init problems, no exterior
 * force; one precision, scheme, lifting order and n_f, other sizes, eps and
 * boundaries free) and n_extra independent instances (pr_instance, the same
 * scheme and precision, each with its own dt) become instances of one batch,
 * so one persistent launch per iteration runs the lift, the n_f fine steps
 * and the projection of every active slice together with n_f steps of every
 * independent instance; then each problem's sequential correction sweep
 * (Eq. 10) runs on a stream of its own, concurrently with the others.  One
 * iteration is one replay of a captured CUDA graph.  The problems are
 * borrowed (they must outlive the object) and iterate in lockstep.  *out is
 * NULL on failure (message: pr_multi_last_error(NULL)).
 * Errors: PR_EINVAL, PR_ENOMEM, PR_ECUDA. */
int pr_multi_create(pr_multi** out, pr_ctx* const* ctxs, int n_ctx, const pr_instance* extra, int n_extra);
int pr_multi_destroy(pr_multi* m);
const char* pr_multi_last_error(const pr_multi* m);

/* The batch that holds the instances: instances 0 .. *first_independent - 1
 * are the problems' slices (owned by the object), the rest the independent
 * instances in the order given, which the pr_batch_* calls set and read
 * (pr_batch_set_initial, pr_batch_get_f, pr_batch_moments ...). */
int pr_multi_batch(pr_multi* m, pr_batch** batch, int* first_independent);

/* count iterations (k <- k + count) of every problem, each initialised
 * (pr_set_initial, or pr_load) and all at the same k, with k + count at most
 * the smallest N; the independent instances advance count x n_f steps.
 * errs (may be NULL) receives errs[it * n_ctx + p], the error of Eq. 10 of
 * problem p in iteration it.  Synchronous.
 * Errors: PR_EINVAL, PR_ETIMEOUT, PR_ENONPHYS, PR_ECUDA. */
int pr_multi_iterate(pr_multi* m, int count, double* errs);

/* ================== batched fine solves (many instances) ================== */

/* Create a batch of n independent fine-solve instances of uneven sizes, all in
 * one precision.  Each fine step of every instance is the fused transport +
 * moments + Maxwellian + implicit BGK update of Eqs. (11)-(13).  Allocates two
 * state buffers per instance plus small tables.  Errors: PR_EINVAL, PR_ENOMEM,
 * PR_ECUDA. */
int pr_batch_create(pr_batch** out, const pr_instance* inst, int n, int precision);

int pr_batch_destroy(pr_batch* b);

const char* pr_batch_last_error(const pr_batch* b);

/* Lift instance i from host state U[5][nx_i] (kind PR_PRIMITIVE or
 * PR_CONSERVED): f = L(U), the pointwise Maxwellian of Eq. (17).  Enqueued on
 * the batch stream after the host copy. */
int pr_batch_set_initial(pr_batch* b, int i, const double* U, int kind);

/* Same with a device pointer U_dev[5][nx_i], enqueued on stream. */
int pr_batch_set_initial_device(pr_batch* b, int i, const double* U_dev, int kind, void* stream);

/* Load an arbitrary distribution f[nx_i][nv_i^3] (host, float64; rounded to
 * float32 in PR_MIXED). Synchronous. */
int pr_batch_set_f(pr_batch* b, int i, const double* f);

/* Advance every instance by nsteps fine steps in ONE persistent launch whose
 * CTAs pull (step, instance, x-tile, v-chunk) work items in step order and
 * wait on neighbouring tiles of the previous step only.  Enqueued on stream. */
int pr_batch_run(pr_batch* b, int nsteps, void* stream);

/* The same for the instances [first, first + count) only (the others keep
 * their state): one persistent launch over that range, e.g. the slices a
 * rank holds at a late parareal iteration (Algorithm 2 recomputes fewer
 * slices each iteration).  Enqueued on stream.  Errors: PR_EINVAL (range
 * outside the batch, nsteps < 0), PR_ECUDA. */
int pr_batch_run_range(pr_batch* b, int first, int count, int nsteps, void* stream);

/* The fine propagation P F L of Algorithm 2 for every instance (Eqs. 17,
 * 11-13, 18): lift from a conserved state (U_dev: the instances' states one
 * after another, [5][nx_i] each, device memory; NULL: the lift sources of the
 * last pr_batch_set_initial calls), run nsteps >= 1 fine steps and project;
 * read the moments with pr_batch_moments or pr_batch_moments_device.  When
 * every instance has one shape whose slice fits a thread-block cluster's
 * shared memory (mixed precision, the Maxwellian lifting, nv = 8 or 16) the
 * run is cluster-resident (one cluster per instance, f never leaves shared
 * memory), else the tiled persistent run.  The stored distributions are
 * unspecified afterwards (set them again before pr_batch_run).  Enqueued on
 * stream.  Errors: PR_EINVAL, PR_ECUDA (PR_ETIMEOUT, PR_ENONPHYS at the next
 * synchronising call). */
int pr_batch_propagate(pr_batch* b, const double* U_dev, int nsteps, void* stream);

/* Moments (Eq. 18) of instance i into host out[5][nx_i]. Synchronous. */
int pr_batch_moments(pr_batch* b, int i, int kind, double* out);

/* Conserved moments of instance i into device out_dev[5][nx_i] on stream. */
int pr_batch_moments_device(pr_batch* b, int i, double* out_dev, void* stream);

/* Distribution of instance i as float64 host f[nx_i][nv_i^3]. Synchronous. */
int pr_batch_get_f(pr_batch* b, int i, double* out);

/* Failure-detection check (not in the paper): one persistent launch of nsteps
 * >= 2 steps in which the dependency waits of step 2 wait for a step that no
 * item ever completes, with the wait limit shortened to wait_ms.  The waiting
 * CTAs give up, record PR_ETIMEOUT and every CTA leaves the launch; the call
 * returns that status after clearing it (PR_ETIMEOUT is the expected result).
 * The batch stays usable; its instance states are unspecified until they are
 * set again.  No GPU fault is involved.  Synchronous. */
int pr_batch_inject_wait_timeout(pr_batch* b, int nsteps, int wait_ms);

/* Wait for the batch stream and report any device-side error. */
int pr_batch_sync(pr_batch* b);

/* Lifting order of the batch's later lifts (pr_batch_set_initial*): 0
 * (Maxwellian, Eq. 17) or 1 (first-order, Def. 3; every instance needs a
 * finite eps).  The first-order lift writes f as a general state (one extra
 * pass instead of the lift fused into the first step).  Errors: PR_EINVAL. */
int pr_batch_set_lift_order(pr_batch* b, int order);

/* Tile width (x cells per work item) used for instance i, and whether it came
 * from the autotuner (1) or the default (0).  The default is 32 cells (capped at
 * nx), narrowed to 16 and then 8 while the batch has fewer work items than the
 * fine kernel has resident CTAs. */
int pr_batch_tile(const pr_batch* b, int i, int* tx, int* tuned);

/* Set the tile width (x cells per work item, 1..64; capped at each instance's
 * nx, and widths below 8 are raised to 8) of every instance, replacing the
 * default or tuned width.  Synchronous. */
int pr_batch_set_tile(pr_batch* b, int tx);

/* Time candidate layouts on the current data with CUDA events and keep the
 * fastest: tile widths 8, 16, 32, 64 (capped at each nx) times velocities
 * per thread of the fine kernel, 8 and 4 when every nv is a multiple of 8
 * (else 4).  The state is saved and restored.  Synchronous. */
int pr_batch_autotune(pr_batch* b);

/* Velocities per thread of the fine kernel in use (4 or 8). */
int pr_batch_vpt(const pr_batch* b, int* vpt);

/* Average duration in ms of the persistent fine kernel over the launches since
 * the last reset, measured with CUDA events on the launching stream; reset=1
 * clears the accumulator.  *launches (may be NULL) gets the launch count. */
int pr_batch_kernel_time(pr_batch* b, double* avg_ms, int* launches, int reset);

/* Gradient of a scalar J(V(T)) of the final conserved moments V(T)[5][nx_i] of
 * instance i after nsteps fine steps from its lifted initial state (the state
 * set by the last pr_batch_set_initial), for the float64 upwind scheme with
 * periodic or outflow boundaries (PR_EINVAL otherwise).  Input lamV = dJ/dV(T)
 * (host [5][nx_i]).  Output dU0 = dJ/dU0 with respect to the primitive initial
 * state U0 = (rho, u_x, u_y, u_z, theta) (host [5][nx_i]) and *dlogeps =
 * dJ/d(log eps).  The hand-written adjoint of each fine step (transposed
 * transport, BGK relaxation differentiated through rho, u, theta of the
 * transported column, Eqs. 11-13, 17, 18) runs backwards from checkpoints of
 * f stored every `checkpoint` steps; each segment is recomputed forward.  Not
 * in the paper.  Allocates and frees its work buffers; synchronous.  The
 * instance's state afterwards is unspecified (set it again before reuse). */
int pr_batch_adjoint(pr_batch* b, int i, int nsteps, int checkpoint, const double* lamV, double* dU0,
                     double* dlogeps);

/* Stable fine step of the E = 0 propagator for the grid of *inst (Sec. 2.2):
 * dt_stab = cfl dx / max|v_x|, dx = (x1 - x0)/nx, max|v_x| = L - dv/2 (the
 * outermost velocity node).  inst->eps, inst->dt and inst->scheme are not
 * read.  Errors: PR_EINVAL (null pointers, nx < 1, x1 <= x0, L <= 0, nv < 1,
 * cfl not finite and > 0). */
int pr_fine_dt_stab(const pr_instance* inst, double cfl, double* dt);

/* Measured FP64 fused multiply-add throughput of the current device in
 * TFLOP/s (2 flops per DFMA): independent DFMA chains on every SM, best of
 * five launches timed with CUDA events after a warm-up.  Not in the paper:
 * the denominator of the plain-FP64 fine step's roofline, which this part's
 * FP64 pipe bounds.  Allocates and frees 8 bytes and a stream; synchronous.
 * Errors: PR_EINVAL (null out), PR_ECUDA. */
int pr_probe_fp64_peak(double* tflops);

/* Number of kernels the library launched since the last reset (any object). */
long long pr_kernel_launches(int reset);

/* ============== one fine step without any memory allocation ============== */

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory themselves or let a library do it --
 * for example an application whose GPU memory is entirely owned by another
 * allocator or pool, or code that must not allocate once it is set up.
 *
 * Computes one fused float64 fine step of the instance *inst (transport,
 * moments, Maxwellian and implicit BGK, the same arithmetic as pr_batch_run):
 * f_out = F(f_in), both caller-owned device arrays [nx][nv^3] of float64,
 * 16-byte aligned, distinct (no in-place update).  It calls no cudaMalloc,
 * cudaFree or other allocating routine.  All scratch (descriptor, factor
 * tables, moment partials, counters, status) lives in one static device array
 * of 4 MiB that every GPU which loads libpr holds until the process exits;
 * instances needing more (about nx * (6 nv + 5 ceil(nv^3/1024)) * 8 bytes plus
 * a few KiB), or more shared memory per CTA than the device allows, are
 * rejected with PR_EINVAL and a message.  The first call on each device does a
 * one-time set-up there: with that device current it looks up the array's
 * device address and sets the fine kernel's shared-memory limit; make that
 * first call before any stream capture.  Every call copies its small
 * descriptors from host memory into the array, clears what must start at
 * zero, and ends by reading the device status back and synchronising the
 * stream.  Calls share the array, so calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Enqueued on stream (NULL: the legacy default stream); returns the device
 * status (PR_ENONPHYS for a non-physical state, PR_ECUDA on a runtime error;
 * the message is in pr_batch_last_error(NULL)). */
int pr_fine_step_noalloc(const pr_instance* inst, const double* f_in, double* f_out, void* stream);

/* ============ exterior force E != 0 (Eqs. 5, 11-13; Test 3) ============ */

/* The collisional Vlasov equation with a force field E(x) along x:
 * d_t f + v_x d_x f + E d_{v_x} f = (M[f] - f)/eps, and the Euler system with
 * the source (0, rho E, 0, 0, rho u_x E) of Eq. (5) as coarse model.
 * Readings (the same as the oracle's): the force enters with the + sign of
 * Eqs. (5), (11) and the flux of Eq. (13) (Eq. 1 prints -E.grad_v f); the v_x
 * flux is the Rusanov flux G_{i,a+1/2} = E_i/2 (f_a + f_{a+1}) - E_max/2
 * (f_{a+1} - f_a), E_max = max_i |E_i|, with no flux through v_x = -L or +L
 * (Eq. 13 prints a viscosity term that vanishes identically); the 1/dv_x of the
 * divergence is inserted; the coarse solver adds the source forward-Euler on
 * the state before each local step; the stable fine step is
 * dt_stab = cfl / (max|v_x| / dx + E_max / dv_x).
 * Velocity grid: nvx cells along v_x and nvp along each of v_y and v_z, all on
 * [-L, L] (Test 3 refines v_x only).  f[nx][nvx nvp^2], velocity index
 * (jx*nvp + jy)*nvp + jz.  No 16-byte rule on nvp here.
 * Each fine step is one kernel launch in which a cluster of CTAs owns one x
 * column: transport in x and v_x, velocity moments exchanged through
 * distributed shared memory, Maxwellian and implicit BGK. */

typedef struct pr_force pr_force;  /* independent force-path instances        */

typedef struct {
    int nx;
    double x0, x1;
    int bc;            /* PR_BC_*                                              */
    int nvx;           /* velocity cells along v_x (>= 2)                      */
    int nvp;           /* velocity cells along each of v_y, v_z (1..32)        */
    double L;          /* velocity box [-L, L]^3                               */
    double eps;        /* Knudsen number > 0; +INFINITY = collisionless        */
    double dt;         /* fine time step > 0                                   */
    const double* E;   /* host [nx]: force at the cell centres, copied at
                          creation; NULL means E = 0                           */
} pr_force_instance;

/* Create n instances that share nx, nvx, nvp (the other fields may differ),
 * one x-transport scheme (PR_UPWIND or PR_MUSCL) and one precision.  Allocates
 * two state buffers per instance.  The v_x rows of a column are split over at
 * most 16 CTAs of nvp^2 threads (rounded up to 32), each thread owning one
 * (v_y, v_z) cell and each CTA staging its rows of f* in shared memory; columns
 * above 16 x 96 KiB (393,216 cells in PR_MIXED, 196,608 in PR_FP64) are
 * rejected with PR_EINVAL.  Errors: PR_EINVAL, PR_ENOMEM, PR_ECUDA. */
int pr_force_create(pr_force** out, const pr_force_instance* inst, int n, int scheme, int precision);

int pr_force_destroy(pr_force* b);

const char* pr_force_last_error(const pr_force* b);

/* Lift instance i from host U[5][nx] (kind PR_PRIMITIVE or PR_CONSERVED):
 * the pointwise Maxwellian of Eq. (17).  Synchronous.
 * Errors: PR_EINVAL, PR_ENONPHYS, PR_ECUDA. */
int pr_force_set_initial(pr_force* b, int i, const double* U, int kind);

/* Load an arbitrary distribution f[nx][nvx nvp^2] (host float64, rounded to
 * float32 in PR_MIXED), e.g. Test 3's two beams.  Synchronous. */
int pr_force_set_f(pr_force* b, int i, const double* f);

/* Advance every instance by nsteps fine steps (one launch per step), enqueued
 * on stream (NULL: the object's stream). */
int pr_force_run(pr_force* b, int nsteps, void* stream);

/* Moments (Eq. 18) of instance i's current state into host out[5][nx].
 * Synchronous; reports device-side errors of earlier runs. */
int pr_force_moments(pr_force* b, int i, int kind, double* out);

/* Instance i's distribution as float64 host f[nx][nvx nvp^2]. Synchronous. */
int pr_force_get_f(pr_force* b, int i, double* out);

/* Wait for the object's stream and report any device-side error. */
int pr_force_sync(pr_force* b);

/* Lifting order of later pr_force_set_initial calls (0 or 1, as
 * pr_batch_set_lift_order).  Errors: PR_EINVAL. */
int pr_force_set_lift_order(pr_force* b, int order);

/* CTAs per x column (the cluster size) and velocities per CTA (v_x rows per
 * CTA times nvp^2) in use. */
int pr_force_config(const pr_force* b, int* cluster, int* chunk);

/* Use `cluster` CTAs per x column (1..16) if the chunk fits shared memory;
 * PR_EINVAL otherwise (the previous setting stays).  Synchronous. */
int pr_force_set_cluster(pr_force* b, int cluster);

/* Cap the threads of the step kernel's CTAs (32..1024, a multiple of 32;
 * default 256): fewer threads per CTA means fewer row groups and more CTAs
 * resident per SM.  A column row always gets its nvp^2 / vec threads.
 * Applies to the current cluster size; PR_EINVAL when no layout fits.
 * Synchronous. */
int pr_force_set_threads(pr_force* b, int threads);

/* Step kernel of the force path.  Two implementations give the same scheme:
 * the clustered step (a cluster of CTAs per x column: transport, exchange of
 * the moments of f* over distributed shared memory, relaxation) and the fused
 * single-pass step (either precision): the moments of f* follow from 17 sums
 * per column of f^n (the upwind-side half sums of v_x f, end-row densities;
 * the v_x fluxes telescope), which every step writes next to f^{n+1}, so each
 * cell is read, relaxed and written in one pass and a CTA walks `columns`
 * consecutive x columns with the next column's bulk copy in flight.  With
 * MUSCL the half sums are of f +- s/2 (s the minmod slope, Eq. 13 with the
 * limiter): a walk also computes, without storing, the column next to each
 * of its ends to form the slopes of f^{n+1}, every walk has at least three
 * columns, a thread holds at most 4 (float) or 8 (double) v_x rows, and a
 * reflecting wall keeps the clustered step.  The fused step needs rows that
 * are 16-byte multiples, at most 256 threads per CTA, and no CTA whose rows
 * straddle v_x = 0.  columns = -1:
 * automatic (the default: the fused step where it applies and there are at
 * least two columns per resident CTA group, walks of that many columns,
 * capped where longer walks would cost a resident CTA per SM and at 32); 0:
 * the clustered step; >= 1: the fused step with walks of about that length
 * (the columns split into equal walks), PR_EINVAL where it does not apply
 * (the previous setting stays).  Results agree to rounding (the moments of f* are
 * summed in another order).  Synchronous. */
int pr_force_set_march(pr_force* b, int columns);

/* Runs of the fused step in one persistent launch.  mode = 1: every run of
 * the fused step is one launch whose CTAs take work items (step, instance,
 * walk, CTA row block) in step order, each waiting (bounded; PR_ETIMEOUT)
 * until its own and its two neighbour walks have finished the previous step;
 * 0: one launch per step; -1 (the default): persistent for runs of two
 * steps or more.  Same results bit for bit.  Synchronous. */
int pr_force_set_persistent(pr_force* b, int mode);

/* Whether a run of nsteps steps of all instances would take one persistent
 * launch (*on = 1) under the current settings. */
int pr_force_get_persistent(const pr_force* b, int nsteps, int* on);

/* Walk length of the fused step in use (0: the clustered step). */
int pr_force_get_march(const pr_force* b, int* columns);

/* Time candidate step layouts on the current states with CUDA events and
 * keep the fastest: every CTA count per column for which the fused step
 * applies, each with its automatic walk length and half and twice it, and
 * the clustered step at its default cluster size (each candidate runs nsteps
 * >= 1 steps twice from the saved states; the second run counts).  The
 * states and moments are restored; the chosen cluster size and walk stay
 * set (pr_force_config, pr_force_get_march).  Synchronous.
 * Errors: PR_EINVAL, PR_ENOMEM (scratch for one copy of the states),
 * PR_ETIMEOUT, PR_ENONPHYS, PR_ECUDA. */
int pr_force_autotune(pr_force* b, int nsteps);

/* Average duration in ms of one step launch over the runs since the last
 * reset (CUDA events on the launching stream around each run, divided by its
 * steps); reset = 1 clears the accumulator. */
int pr_force_kernel_time(pr_force* b, double* avg_ms, int* steps, int reset);

/* Failure-detection check (not in the paper): one fine step of every
 * instance in which each CTA, besides its real staging copies, waits on a
 * second mbarrier that expects bytes no copy delivers, with the wait limit
 * shortened to wait_ms.  The waits run out, record PR_ETIMEOUT, then each CTA
 * waits for its real copies before it leaves; the call returns that status
 * after clearing it (PR_ETIMEOUT is the expected result).  The object stays
 * usable; the instance states are unspecified until they are set again.
 * With the fused step forced persistent (pr_force_set_persistent(b, 1)) the
 * check is instead a two-step persistent run whose step-2 items wait for a
 * completion count no walk reaches: those dependency waits run out the same
 * way.  PR_EINVAL when the rows are not staged by bulk copies (nvp^2 x
 * element size not a multiple of 16 bytes).  No GPU fault is involved.
 * Synchronous. */
int pr_force_inject_wait_timeout(pr_force* b, int wait_ms);

/* dt_stab of the reading above for inst (E read from the host array).
 * Errors: PR_EINVAL. */
int pr_force_dt_stab(const pr_force_instance* inst, double cfl, double* dt);

/* A parareal problem with the force: as pr_init, with v->nv cells along v_y
 * and v_z, nvx along v_x, and E (host [nx], copied; NULL = 0).  The fine
 * propagator is the force path above (scheme and precision from t), the
 * coarse propagator the Euler system with the source, n_f (t->nf = 0) from
 * dt_stab with the force.  Every pr_* call on a parareal problem works on the
 * result.  Errors: PR_EINVAL, PR_ENOMEM, PR_ECUDA. */
int pr_init_force(pr_ctx** out, const pr_grid* g, const pr_velocity* v, double eps, const pr_time* t, int nvx,
                  const double* E);

/* Kernel of the fine phase of a parareal iteration (pr_init problems):
 * PR_FINE_AUTO takes the cluster-resident run when it applies (mixed
 * precision, Maxwellian lifting, nv = 8 or 16, a slice's cells fit the
 * shared memory of a cluster of <= 16 CTAs) and the resident slices'
 * clusters run in at most two waves, else the tiled persistent kernel; PR_FINE_TILED and
 * PR_FINE_CLUSTER force one (PR_EINVAL when the cluster run does not apply or
 * the problem has a force).  The cluster run lifts, steps and projects a
 * slice without the batch's global state: it serves pr_parareal_iter / _run;
 * pr_fine_step always uses the tiled kernel.  The next iteration rebuilds its
 * captured graph.  Synchronous. */
int pr_set_fine_path(pr_ctx* ctx, int mode);

/* The kernel the fine phase of an iteration uses: PR_FINE_TILED or
 * PR_FINE_CLUSTER (never PR_FINE_AUTO). */
int pr_get_fine_path(const pr_ctx* ctx, int* path);

/* Layout of the cluster-resident fine run for this problem's slices: CTAs
 * per cluster, x cells per CTA and how many clusters (slices) the device runs
 * at once; all 0 (and PR_OK) when the run does not apply. */
int pr_fine_cluster_shape(const pr_ctx* ctx, int* cluster, int* cells_per_cta, int* resident);

/* Step kernel of a pr_init_force problem's fine propagator (its slices are
 * the instances of an internal pr_force): cluster > 0 sets the CTAs per x
 * column (pr_force_set_cluster; 0 keeps them), then columns and persistent as
 * pr_force_set_march and pr_force_set_persistent.  The next iteration
 * rebuilds its captured graph.  PR_EINVAL for a problem without a force or a
 * setting that does not apply (earlier settings of the call stay).
 * Synchronous. */
int pr_set_force_step(pr_ctx* ctx, int cluster, int columns, int persistent);

#ifdef __cplusplus
}
#endif
#endif
