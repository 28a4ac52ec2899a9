// capi.cpp — the extern "C" entry points declared in include/pat.h.
// Validation happens here, before anything is enqueued; the kernels are in
// kernels.cu and the plan builder in plan.cpp.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <set>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "kernels.h"
#include "pat.h"
#include "plan.h"

using namespace patgpu;

namespace {

std::mutex g_mu;
std::set<const Plan*> g_live;

Plan* lookup(pat_plan_t h)
{
    std::lock_guard<std::mutex> lk(g_mu);
    const Plan* p = reinterpret_cast<const Plan*>(h);
    if (!p || !g_live.count(p) || p->magic != kPlanMagic) return nullptr;
    return const_cast<Plan*>(p);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// true when the byte ranges [a, a + na) and [b, b + nb) overlap
bool overlap(const void* a, size_t na, const void* b, size_t nb)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

// Makes the plan's device current for the duration of a call.
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            prev = -1;
            return;
        }
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceScope()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

pat_status_t cuda_status(cudaError_t e) { return e == cudaSuccess ? PAT_OK : PAT_ERR_CUDA; }

// NVTX range named after the entry point, for the host-side timeline of a
// profiler (header-only NVTX: a no-op unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

cudaEvent_t take_event(Plan& p)
{
    if (!p.event_pool.empty()) {
        cudaEvent_t e = p.event_pool.back();
        p.event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Enqueues `fn` on `st`; with tracing on, brackets it with two events.
template <typename F>
cudaError_t timed(Plan& p, int kind, cudaStream_t st, F&& fn)
{
    if (!p.timing) return fn();
    cudaEvent_t a = take_event(p), b = take_event(p);
    if (!a || !b) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) p.recorded[kind].emplace_back(a, b);
    else {
        p.event_pool.push_back(a);
        p.event_pool.push_back(b);
    }
    return e;
}

// The circular-mean launch; a wait probe armed by pat_plan_set_wait_probe
// goes with this one launch only.
cudaError_t circmean(Plan& p, const void* f, cudaStream_t st, bool msum = true)
{
    const cudaError_t e = launch_circmean(p.dp, f, st, msum);
    p.dp.wait_probe = 0;
    return e;
}

// The adjoint gather launch (list or cell form; f == nullptr: cell sums only,
// for the fused steps); a bounds probe armed by pat_plan_set_bounds_probe
// goes with this one launch only.
cudaError_t gather(Plan& p, void* f, cudaStream_t st)
{
    const cudaError_t e = f ? launch_adjoint_gather(p.dp, f, st) : launch_adjoint_cells(p.dp, st);
    p.dp.bounds_probe = 0;
    return e;
}

bool valid_geometry(const pat_geometry_t& g, bool bf16)
{
    if (g.n < 8 || g.n > 4096 || (g.n % (bf16 ? 8 : 4)) != 0) return false;
    if (g.n_det < 1 || g.n_det > 16384) return false;
    if (!(g.arc_span > 0.0) || g.arc_span > 6.283185307179586 * (1.0 + 1e-12) || !std::isfinite(g.arc_start))
        return false;
    if (g.n_t < 1 || g.n_t > 16384) return false;
    if (!(g.t_max > 0.0) || !std::isfinite(g.t_max) || g.t_max > 64.0) return false;
    if (g.n_angles < 3 || g.n_angles > 65536) return false;
    return true;
}

} // namespace

extern "C" {

const char* pat_status_string(pat_status_t s)
{
    switch (s) {
    case PAT_OK: return "PAT_OK";
    case PAT_ERR_INVALID_ARG: return "PAT_ERR_INVALID_ARG";
    case PAT_ERR_CUDA: return "PAT_ERR_CUDA";
    case PAT_ERR_OOM: return "PAT_ERR_OOM";
    case PAT_ERR_UNSUPPORTED: return "PAT_ERR_UNSUPPORTED";
    case PAT_ERR_TIMEOUT: return "PAT_ERR_TIMEOUT";
    case PAT_ERR_BAD_PLAN: return "PAT_ERR_BAD_PLAN";
    case PAT_ERR_BOUNDS: return "PAT_ERR_BOUNDS";
    }
    return "PAT_ERR_UNKNOWN";
}

pat_status_t pat_plan_create(const pat_geometry_t* geoms, int32_t n_instances, const pat_options_t* opt_in,
                             void* stream, pat_plan_t* out)
{
    NvtxRange nvtx("pat_plan_create");
    if (!geoms || n_instances < 1 || n_instances > (1 << 20) || !out) return PAT_ERR_INVALID_ARG;
    pat_options_t opt;
    if (opt_in) opt = *opt_in;
    else std::memset(&opt, 0, sizeof(opt));
    if (opt.image_dtype != PAT_F32 && opt.image_dtype != PAT_BF16) return PAT_ERR_INVALID_ARG;
    if (opt.schedule != PAT_SCHED_STAGED && opt.schedule != PAT_SCHED_PERSISTENT) return PAT_ERR_INVALID_ARG;
    if (opt.schedule == PAT_SCHED_PERSISTENT) return PAT_ERR_UNSUPPORTED;
    if (opt.tune < 0 || opt.tune > 2) return PAT_ERR_INVALID_ARG;
    if (opt.m_lanes == 0) opt.m_lanes = 32;
    if (opt.m_lanes != 32 && opt.m_lanes != 16 && opt.m_lanes != 8) return PAT_ERR_INVALID_ARG;
    if (opt.q_piece == 0) opt.q_piece = 128;
    if (opt.q_piece < 4 || opt.q_piece % 4 != 0) return PAT_ERR_INVALID_ARG;
    if (opt.band_rows != 0 && (opt.band_rows < 1 || opt.band_rows > 8192)) return PAT_ERR_INVALID_ARG;
    if (opt.tile_cols != 0 && (opt.tile_cols < 1 || opt.tile_cols > 8192)) return PAT_ERR_INVALID_ARG;
    if (opt.adj_groups < 0 || opt.adj_groups > 16) return PAT_ERR_INVALID_ARG;
    if (opt.time_pair != 0 && opt.time_pair != 1) return PAT_ERR_INVALID_ARG;
    if (opt.adj_mode < 0 || opt.adj_mode > 4) return PAT_ERR_INVALID_ARG;
    if (opt.adj_jblock < 0 || opt.adj_jblock > 16384) return PAT_ERR_INVALID_ARG;
    if (opt.abel_split != 0 && opt.abel_split != 1 && opt.abel_split != 2 && opt.abel_split != 4 &&
        opt.abel_split != 8)
        return PAT_ERR_INVALID_ARG;
    const bool bf16 = opt.image_dtype == PAT_BF16;
    for (int i = 0; i < n_instances; ++i)
        if (!valid_geometry(geoms[i], bf16)) return PAT_ERR_INVALID_ARG;

    Plan* p = nullptr;
    pat_status_t s;
    if (opt.tune == 1) {
        try {
            s = autotune_plan(&p, geoms, n_instances, opt, static_cast<cudaStream_t>(stream));
        } catch (const std::bad_alloc&) {
            s = PAT_ERR_OOM;
        }
        if (s != PAT_OK) return s;
    } else {
        p = new (std::nothrow) Plan();
        if (!p) return PAT_ERR_OOM;
        try {
            s = build_plan(*p, geoms, n_instances, opt, static_cast<cudaStream_t>(stream));
        } catch (const std::bad_alloc&) {
            s = PAT_ERR_OOM;
        } catch (...) {
            s = PAT_ERR_INVALID_ARG;
        }
        if (s != PAT_OK) {
            free_plan_memory(*p);
            delete p;
            return s;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_live.insert(p);
    }
    *out = reinterpret_cast<pat_plan_t>(p);
    return PAT_OK;
}

pat_status_t pat_plan_destroy(pat_plan_t h)
{
    NvtxRange nvtx("pat_plan_destroy");
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_live.erase(p);
    }
    {
        DeviceScope ds(p->device);
        free_plan_memory(*p);
    }
    p->magic = 0;
    delete p;
    return PAT_OK;
}

pat_status_t pat_plan_layout(pat_plan_t h, int64_t* f_offsets, int64_t* g_offsets)
{
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    if (f_offsets) std::memcpy(f_offsets, p->f_offsets.data(), sizeof(int64_t) * p->f_offsets.size());
    if (g_offsets) std::memcpy(g_offsets, p->g_offsets.data(), sizeof(int64_t) * p->g_offsets.size());
    return PAT_OK;
}

pat_status_t pat_plan_info(pat_plan_t h, pat_plan_info_t* info)
{
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    if (!info) return PAT_ERR_INVALID_ARG;
    *info = p->info;
    return PAT_OK;
}

pat_status_t pat_forward(pat_plan_t h, const void* d_f, float* d_g, void* stream)
{
    NvtxRange nvtx("pat_forward");
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    if (!d_f || !d_g || !aligned16(d_f) || !aligned16(d_g)) return PAT_ERR_INVALID_ARG;
    DeviceScope ds(p->device);
    if (!ds.ok) return PAT_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = timed(*p, PAT_K_CIRCMEAN, st, [&] { return circmean(*p, d_f, st); });
    if (e == cudaSuccess) e = timed(*p, PAT_K_ABEL_FWD, st, [&] { return launch_abel_fwd(p->dp, d_g, st); });
    return cuda_status(e);
}

pat_status_t pat_adjoint(pat_plan_t h, const float* d_g, void* d_f, void* stream)
{
    NvtxRange nvtx("pat_adjoint");
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    if (!d_f || !d_g || !aligned16(d_f) || !aligned16(d_g)) return PAT_ERR_INVALID_ARG;
    DeviceScope ds(p->device);
    if (!ds.ok) return PAT_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = timed(*p, PAT_K_ABEL_ADJ, st, [&] { return launch_abel_adj(p->dp, d_g, st); });
    if (e == cudaSuccess) e = timed(*p, PAT_K_ADJ_GATHER, st, [&] { return gather(*p, d_f, st); });
    return cuda_status(e);
}

pat_status_t pat_tv_grad(pat_plan_t h, const float* d_f, float eps, float* d_grad, float* d_value, void* stream)
{
    NvtxRange nvtx("pat_tv_grad");
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    if (p->dp.bf16) return PAT_ERR_UNSUPPORTED;
    if (!d_f || !aligned16(d_f) || !(eps > 0.f) || !std::isfinite(eps)) return PAT_ERR_INVALID_ARG;
    if (!d_grad && !d_value) return PAT_ERR_INVALID_ARG;
    if ((d_grad && !aligned16(d_grad)) || (d_value && (reinterpret_cast<uintptr_t>(d_value) & 3u)))
        return PAT_ERR_INVALID_ARG;
    // the stencil reads neighbours other threads may already have written
    const size_t fb = sizeof(float) * (size_t)p->f_offsets.back(), vb = sizeof(float) * (size_t)p->n_inst;
    if (d_grad && overlap(d_f, fb, d_grad, fb)) return PAT_ERR_INVALID_ARG;
    if (d_value && (overlap(d_f, fb, d_value, vb) || (d_grad && overlap(d_grad, fb, d_value, vb))))
        return PAT_ERR_INVALID_ARG;
    DeviceScope ds(p->device);
    if (!ds.ok) return PAT_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return cuda_status(timed(*p, PAT_K_TV, st, [&] { return launch_tv(p->dp, d_f, eps, d_grad, d_value, st); }));
}

pat_status_t pat_residual(pat_plan_t h, const float* d_Af, const float* d_g, float* d_r, float scale, void* stream)
{
    NvtxRange nvtx("pat_residual");
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    if (!d_Af || !d_g || !d_r || !aligned16(d_Af) || !aligned16(d_g) || !aligned16(d_r) || !std::isfinite(scale))
        return PAT_ERR_INVALID_ARG;
    DeviceScope ds(p->device);
    if (!ds.ok) return PAT_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return cuda_status(timed(*p, PAT_K_RESIDUAL, st,
                             [&] { return launch_residual(d_Af, d_g, d_r, scale, p->g_offsets.back(), st); }));
}

pat_status_t pat_descent_step(pat_plan_t h, float* d_f, const float* d_adj, const float* d_tvgrad, float tau,
                              float lam, int32_t nonneg, float* d_delta, void* stream)
{
    NvtxRange nvtx("pat_descent_step");
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    if (p->dp.bf16) return PAT_ERR_UNSUPPORTED;
    if (!d_f || !d_adj || !aligned16(d_f) || !aligned16(d_adj) || (d_tvgrad && !aligned16(d_tvgrad)))
        return PAT_ERR_INVALID_ARG;
    if (!std::isfinite(tau) || !std::isfinite(lam)) return PAT_ERR_INVALID_ARG;
    DeviceScope ds(p->device);
    if (!ds.ok) return PAT_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return cuda_status(timed(*p, PAT_K_DESCENT, st, [&] {
        return launch_descent(p->dp, d_f, d_adj, d_tvgrad, tau, lam, nonneg, d_delta, st);
    }));
}

pat_status_t pat_tv_step(pat_plan_t h, const float* d_f_in, float* d_f_out, const float* d_g, float tau, float lam,
                         float eps, int32_t nonneg, float* d_delta, void* stream)
{
    NvtxRange nvtx("pat_tv_step");
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    if (p->dp.bf16) return PAT_ERR_UNSUPPORTED;
    if (!d_f_in || !d_f_out || !d_g || !aligned16(d_f_in) || !aligned16(d_f_out) || !aligned16(d_g))
        return PAT_ERR_INVALID_ARG;
    if (d_f_in == d_f_out) return PAT_ERR_INVALID_ARG;
    if (!std::isfinite(tau) || !std::isfinite(lam) || !(eps > 0.f) || !std::isfinite(eps)) return PAT_ERR_INVALID_ARG;
    DeviceScope ds(p->device);
    if (!ds.ok) return PAT_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const DevPlan& dp = p->dp;
    const bool pair = dp.time_chunks > 0;
    cudaError_t e = timed(*p, PAT_K_CIRCMEAN, st, [&] { return circmean(*p, d_f_in, st, !pair); });
    if (pair) {
        if (e == cudaSuccess)
            e = timed(*p, PAT_K_TIME_PAIR, st,
                      [&] { return launch_time_pair(dp, d_g, nullptr, false, 0.f, 1.f, st); });
    } else {
        if (e == cudaSuccess)
            e = timed(*p, PAT_K_ABEL_FWD, st, [&] { return launch_abel_fwd(dp, p->d_resid, st, d_g); });
        if (e == cudaSuccess)
            e = timed(*p, PAT_K_ABEL_ADJ, st, [&] { return launch_abel_adj(dp, p->d_resid, st); });
    }
    if (e == cudaSuccess) e = timed(*p, PAT_K_ADJ_GATHER, st, [&] { return gather(*p, nullptr, st); });
    if (e == cudaSuccess)
        e = timed(*p, PAT_K_TV_UPDATE, st,
                  [&] { return launch_tv_update(dp, d_f_in, d_f_out, tau, lam, eps, nonneg, d_delta, st); });
    return cuda_status(e);
}

pat_status_t pat_pdhg_step(pat_plan_t h, float* d_f, float* d_fbar, float* d_y, float* d_px, float* d_py,
                           const float* d_g, float sigma, float tau, float alpha, int32_t nonneg, float beta,
                           float mean_target, float* d_fmean, float* d_delta, void* stream)
{
    NvtxRange nvtx("pat_pdhg_step");
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    if (p->dp.bf16) return PAT_ERR_UNSUPPORTED;
    float* img[4] = {d_f, d_fbar, d_px, d_py};
    for (float* q : img)
        if (!q || !aligned16(q)) return PAT_ERR_INVALID_ARG;
    if (!d_y || !d_g || !aligned16(d_y) || !aligned16(d_g)) return PAT_ERR_INVALID_ARG;
    const size_t fb = sizeof(float) * (size_t)p->f_offsets.back(), gb = sizeof(float) * (size_t)p->g_offsets.back();
    for (int a = 0; a < 4; ++a) {
        for (int b = a + 1; b < 4; ++b)
            if (overlap(img[a], fb, img[b], fb)) return PAT_ERR_INVALID_ARG;
        if (overlap(img[a], fb, d_y, gb) || overlap(img[a], fb, d_g, gb)) return PAT_ERR_INVALID_ARG;
    }
    if (overlap(d_y, gb, d_g, gb)) return PAT_ERR_INVALID_ARG;
    if (!(sigma > 0.f) || !std::isfinite(sigma) || !(tau > 0.f) || !std::isfinite(tau) || !(alpha >= 0.f) ||
        !std::isfinite(alpha) || !(beta >= 0.f) || !std::isfinite(beta) || !std::isfinite(mean_target))
        return PAT_ERR_INVALID_ARG;
    if (beta > 0.f && !d_fmean) return PAT_ERR_INVALID_ARG;
    if (d_delta) {
        const size_t db = 2 * sizeof(float) * (size_t)p->n_inst;
        if (reinterpret_cast<uintptr_t>(d_delta) & 3u) return PAT_ERR_INVALID_ARG;
        for (float* q : img)
            if (overlap(q, fb, d_delta, db)) return PAT_ERR_INVALID_ARG;
        if (overlap(d_y, gb, d_delta, db) || overlap(d_g, gb, d_delta, db)) return PAT_ERR_INVALID_ARG;
    }
    if (d_fmean) {
        const size_t mb = sizeof(float) * (size_t)p->n_inst;
        if (reinterpret_cast<uintptr_t>(d_fmean) & 3u) return PAT_ERR_INVALID_ARG;
        for (float* q : img)
            if (overlap(q, fb, d_fmean, mb)) return PAT_ERR_INVALID_ARG;
        if (overlap(d_y, gb, d_fmean, mb) || overlap(d_g, gb, d_fmean, mb)) return PAT_ERR_INVALID_ARG;
        if (d_delta && overlap(d_delta, 2 * mb, d_fmean, mb)) return PAT_ERR_INVALID_ARG;
    }
    DeviceScope ds(p->device);
    if (!ds.ok) return PAT_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const DevPlan& dp = p->dp;
    const float inv1ps = 1.f / (1.f + sigma);
    cudaError_t e = timed(*p, PAT_K_PDHG_DUAL, st,
                          [&] { return launch_pdhg_dual_tv(dp, d_fbar, d_px, d_py, sigma, alpha, st); });
    const bool pair = dp.time_chunks > 0;
    if (e == cudaSuccess) e = timed(*p, PAT_K_CIRCMEAN, st, [&] { return circmean(*p, d_fbar, st, !pair); });
    if (pair) {
        if (e == cudaSuccess)
            e = timed(*p, PAT_K_TIME_PAIR, st,
                      [&] { return launch_time_pair(dp, d_g, d_y, true, sigma, inv1ps, st); });
    } else {
        if (e == cudaSuccess)
            e = timed(*p, PAT_K_ABEL_FWD, st,
                      [&] { return launch_abel_fwd_dual(dp, d_y, d_g, sigma, inv1ps, st); });
        if (e == cudaSuccess) e = timed(*p, PAT_K_ABEL_ADJ, st, [&] { return launch_abel_adj(dp, d_y, st); });
    }
    if (e == cudaSuccess) e = timed(*p, PAT_K_ADJ_GATHER, st, [&] { return gather(*p, nullptr, st); });
    if (e == cudaSuccess)
        e = timed(*p, PAT_K_PDHG_PRIMAL, st,
                  [&] {
                      return launch_pdhg_primal(dp, d_f, d_fbar, d_px, d_py, tau, nonneg, d_fmean, beta, mean_target,
                                                d_delta, st);
                  });
    return cuda_status(e);
}

pat_status_t pat_plan_sync_status(pat_plan_t h, void* stream)
{
    NvtxRange nvtx("pat_plan_sync_status");
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    DeviceScope ds(p->device);
    if (!ds.ok) return PAT_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t word = 0;
    if (cudaMemcpyAsync(&word, p->dp.status, sizeof(word), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return PAT_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PAT_ERR_CUDA;
    if (word == 0) return PAT_OK;
    // a launch that gave up may have left counters armed: clear them with the word
    // (a failed bounds check of a debug build is reported the same way)
    if (cudaMemsetAsync(p->dp.status, 0, sizeof(int32_t), st) != cudaSuccess) return PAT_ERR_CUDA;
    if (cudaMemsetAsync(p->d_counters, 0, p->counters_bytes, st) != cudaSuccess) return PAT_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PAT_ERR_CUDA;
    return (word & kBoundsFlag) ? PAT_ERR_BOUNDS : PAT_ERR_TIMEOUT;
}

pat_status_t pat_plan_set_bounds_probe(pat_plan_t h, int32_t enable)
{
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
#ifdef PAT_DEBUG
    p->dp.bounds_probe = enable ? 1 : 0;
    return PAT_OK;
#else
    (void)enable;
    return PAT_ERR_UNSUPPORTED;
#endif
}

pat_status_t pat_debug_fail_alloc(int32_t n)
{
    set_alloc_failure(n);
    return PAT_OK;
}

int32_t pat_debug_build(void)
{
#ifdef PAT_DEBUG
    return 1;
#else
    return 0;
#endif
}

pat_status_t pat_plan_set_wait_probe(pat_plan_t h, int32_t clocks)
{
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    if (clocks < 0) return PAT_ERR_INVALID_ARG;
    p->dp.wait_probe = clocks;
    return PAT_OK;
}

pat_status_t pat_plan_set_timing(pat_plan_t h, int32_t enable)
{
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    p->timing = enable != 0;
    return PAT_OK;
}

pat_status_t pat_plan_kernel_times(pat_plan_t h, double* total_ms, int64_t* launches, int32_t n_kinds)
{
    Plan* p = lookup(h);
    if (!p) return PAT_ERR_BAD_PLAN;
    if (n_kinds < 0) return PAT_ERR_INVALID_ARG;
    DeviceScope ds(p->device);
    if (!ds.ok) return PAT_ERR_CUDA;
    pat_status_t st = PAT_OK;
    for (int k = 0; k < PAT_K_COUNT; ++k) {
        double sum = 0.0;
        int64_t cnt = 0;
        for (auto& pr : p->recorded[k]) {
            float ms = 0.f;
            if (cudaEventSynchronize(pr.second) != cudaSuccess ||
                cudaEventElapsedTime(&ms, pr.first, pr.second) != cudaSuccess)
                st = PAT_ERR_CUDA;
            sum += ms;
            ++cnt;
            p->event_pool.push_back(pr.first);
            p->event_pool.push_back(pr.second);
        }
        p->recorded[k].clear();
        if (k < n_kinds) {
            if (total_ms) total_ms[k] = sum;
            if (launches) launches[k] = cnt;
        }
    }
    return st;
}

} // extern "C"
