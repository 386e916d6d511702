// Host-side state of one simulation, shared by the single-simulation entry points and the
// batch / serving entry points.
#pragma once
#include <cstdint>
#include <utility>
#include <vector>
#include <cuda_runtime.h>
#include "../../include/wmcd.h"
#include "wmcd_internal.h"

namespace wmcd {

// Bump allocation of a simulation's device state inside one block of a batch's pool. In
// counting mode nothing is placed: `used` only sums the 256-byte-aligned sizes.
struct Arena {
    char* base = nullptr;
    size_t size = 0, used = 0;
    bool count_only = false;
};

struct Handle {
    wmcd_params P;
    SimView v;                   // host copy of the view
    SimView* dview = nullptr;    // device copy read by every kernel
    GroupDims g;                 // launch bounds of this one simulation
    int dev = 0;
    int64_t N = 0;
    int nL = 0;
    double expect[kMaxLayers] = {0};
    int Mmax[kMaxLayers] = {0};
    double p_fourier = 0.0, dt_move = 0.0, R = 1.0;
    uint64_t sweep = 0, pw_calls = 0;
    int64_t tr_pw_count = 0;
    int64_t launches = 0;        // kernels launched by this handle
    std::vector<void*> allocs;   // cudaMalloc'd blocks owned by the handle
    size_t bytes = 0;
    double* staging = nullptr;   // 3N doubles
    Arena* arena = nullptr;      // set while a batch places the state in its pool
    void* batch = nullptr;       // owning batch, if any
    ForkJoin fj;                 // side stream and events: launches of a phase that run side by side
    // profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    int64_t prof_launches[8] = {0};
    double prof_ms[8] = {0};
};

int last_cuda_status();
// WMCD_OK, or WMCD_EINVAL for parameters wmcd_create refuses (the checks listed in wmcd.h)
int validate_params(const wmcd_params* p);
int64_t slot_count(const Handle* h, uint32_t kind, int l, uint64_t ctr, double x);
int64_t enqueue_sweep(const SimView* d, const GroupDims& g, const int64_t* hc, Handle* prof, cudaStream_t s,
                      const ForkJoin* fj = nullptr);
// Set up a simulation in *H (tables, device state, cell list). With an arena the device state
// is placed in it; a counting arena only sizes it (nothing is launched or copied). On failure
// the caller releases H with destroy_handle.
int create_handle(struct ::wmcd_handle* H, const wmcd_params* params, const double* pos, const int32_t* chain_len,
                  int64_t n_chains, cudaStream_t s, Arena* arena);
void destroy_handle(struct ::wmcd_handle* H);
void prof_harvest(Handle* h);
int take_kernel_times(Handle* h, int64_t* launches, double* ms, int n_classes);
// a batch is told when a member's view changed (its copy in the batch is refreshed)
void batch_view_changed(void* batch);

}  // namespace wmcd

struct wmcd_handle { wmcd::Handle h; };
