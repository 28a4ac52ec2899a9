// plan.h — host-side plan object of the photoacoustic operator library.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "pat.h"
#include "pat_internal.h"

namespace patgpu {

constexpr uint64_t kPlanMagic = 0x5041545f504c414eull; // "PAT_PLAN"

struct Plan {
    uint64_t magic = kPlanMagic;
    int device = 0;
    int num_sms = 0;
    int n_inst = 0;
    int band_budget_bytes = 110 * 1024;  // default shared memory of a circular-mean CTA (2 per SM)
    int max_smem_optin = 227 * 1024;
    pat_options_t opt{};
    std::vector<pat_geometry_t> geoms;
    std::vector<int64_t> f_offsets, g_offsets;
    void* d_tables = nullptr;
    size_t tables_bytes = 0;
    float* d_work = nullptr;
    int64_t work_floats = 0;
    int32_t* d_counters = nullptr;     // arrival counters + work queues (zero between calls)
    size_t counters_bytes = 0;
    void* d_lists = nullptr;           // adjoint sample lists (list mode)
    float* d_resid = nullptr;          // data residual of the fused TV step (inside d_work)
    int code_bits_max = 0;             // bits of a packed (j, m, q) sample code, largest instance
    int64_t list_budget_bytes = 24ll << 30;
    int fwd_smem = 0;
    DevPlan dp{};
    pat_plan_info_t info{};
    // tracing: recorded (start, end) event pairs per kernel kind, and a pool
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> recorded[PAT_K_COUNT];
    std::vector<cudaEvent_t> event_pool;
};

// Builds all tables, schedules and tiles of P for the given geometries and
// (already defaulted and validated) options; uploads them on `st` and waits.
pat_status_t build_plan(Plan& P, const pat_geometry_t* geoms, int n_inst, const pat_options_t& opt,
                        cudaStream_t st);
void free_plan_memory(Plan& P);

// Every device allocation of plan creation (and of the autotuner) goes
// through dev_malloc.  Test hook: after set_alloc_failure(n), the n-th next
// such allocation (0 = the next one) fails as if the device were out of
// memory, once; n < 0 disarms it.
cudaError_t dev_malloc(void** p, size_t bytes);
void set_alloc_failure(int32_t n);

// Builds the plan with the fastest of a set of candidate tile shapes, timed on
// the plan's geometries (tune = 1); results are cached per process.
pat_status_t autotune_plan(Plan** out, const pat_geometry_t* geoms, int n_inst, const pat_options_t& opt,
                           cudaStream_t st);

} // namespace patgpu
