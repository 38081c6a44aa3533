// Internal interface between the force-path batch (force_runtime.cu) and the
// parareal context (runtime.cu).  Internal to libpr.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "pr.h"
#include "pr_kernels.h"

struct pr_force {
    int n = 0, precision = 0, scheme = 0, nx = 0, nvx = 0, nvp = 0;
    int lift_order = 0;                 // 0: Maxwellian lift; 1: first-order lift (lift_ce.cu)
    int max_threads = 256;              // thread cap of the step kernel's CTAs
    int march_req = -1;                 // fused step walk length: -1 automatic, 0 clustered step
    void* d_part = nullptr;             // fused step partials, [2][n][nx][C][17] double-float
    size_t part_bytes = 0;
    std::vector<char> sums_ok;          // per instance: the partials match the current state
    int persist_req = -1;               // fused runs in one persistent launch: -1 automatic, 0 never, 1 always
    int* d_fsync = nullptr;             // persistent run: ticket + done count per instance and walk
    int fsync_words = 0;
    prk::FGeom g{};
    size_t smem = 0;
    std::vector<prk::FInst> h;          // host copy of the descriptors
    prk::FInst* d_inst = nullptr;
    prk::Active* d_active = nullptr;
    int* d_cur = nullptr;               // [n] buffer index of each instance's state
    int* d_status = nullptr;
    double* d_E = nullptr;              // [n][nx]
    float* d_Ef = nullptr;              // [n][nx] float copy
    double* d_U = nullptr;              // [n][5][nx] moments of the current states
    double* d_Ulift = nullptr;          // [n][5][nx] lift sources of pr_force_set_initial
    void* d_vtab = nullptr;             // [n][nvx + 3 nvp^2] velocity tables (element type of f)
    std::vector<void*> bufs;            // two state buffers per instance
    double* d_tmp = nullptr;            // float64 staging of one instance's f (lazy)
    cudaStream_t stream = nullptr;
    // CUDA-event timing of the step launches
    struct Pending {
        cudaEvent_t a, b;
        int steps;
    };
    std::vector<Pending> pending;
    double step_ms_sum = 0.0;
    int steps_timed = 0;
    std::string err;
};

// Adds n to the library-wide kernel launch counter (runtime.cu).
void pr_internal_count_launches(long long n);

namespace prf {

int create(pr_force** out, const pr_force_instance* inst, int n, int scheme, int precision, std::string& err);
void destroy(pr_force* b);
// Point instance b's lift source and projection target at device buffers.
void bind(pr_force* b, int i, const double* Uin, double* Uout);
cudaError_t upload(pr_force* b, int b0, int b1, cudaStream_t s);
// Lift instances [b0, b1) from their Uin, run nsteps steps (the last writes
// Ucur and Uout; with nsteps = 0 the moments of the lifted state go to Ucur),
// advance their buffer indices.  Active range restored to all.
int enqueue_lift_run(pr_force* b, int b0, int b1, int nsteps, cudaStream_t s, bool timing);
// Run nsteps steps of instances [b0, b1) from their current states.
int enqueue_run(pr_force* b, int b0, int b1, int nsteps, cudaStream_t s, bool timing);
// The body of one graph-captured parareal iteration: active slices from the
// device counter dk (slices max(k,1)..N on instances first_slice-1..), lift,
// nsteps steps with projection, advance.
cudaError_t enqueue_graph_body(pr_force* b, const int* dk, int N, int nsteps, cudaStream_t s);
// Device status: 0 or a PR_* code (cleared).  Synchronises b->stream.
// Kernel launches enqueue_graph_body makes for a run of nsteps steps.
int graph_body_launches(const pr_force* b, int nsteps);
int take_status(pr_force* b);
double emax(const pr_force* b, int i);
int launches_per_step();

}  // namespace prf
