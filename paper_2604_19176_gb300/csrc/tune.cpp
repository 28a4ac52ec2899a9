// tune.cpp — autotuner for the tile shapes of a plan.
//
// Candidates for the circular-mean kernel (radii per warp, angles per unit,
// tile width) are timed on the plan's own geometries with
// CUDA events, then the cluster split of the two time stages, then candidates
// for the adjoint gather (list format, list parts) with the best shapes so
// far; the fastest plan is kept.  Results are cached per
// process by geometry list and image dtype, so a second plan with the same
// geometries skips the search.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.h"
#include "plan.h"

namespace patgpu {

namespace {

std::mutex g_tune_mu;
std::map<std::string, pat_options_t> g_tune_cache;

// Cache key from the geometries' fields (not their struct bytes, whose
// padding a C caller may leave uninitialised), the image dtype and the device.
std::string tune_key(const pat_geometry_t* geoms, int n, const pat_options_t& opt, int device)
{
    std::string k;
    auto put = [&k](const void* p, size_t b) { k.append(static_cast<const char*>(p), b); };
    for (int i = 0; i < n; ++i) {
        const pat_geometry_t& g = geoms[i];
        put(&g.n, sizeof g.n);
        put(&g.n_det, sizeof g.n_det);
        put(&g.arc_start, sizeof g.arc_start);
        put(&g.arc_span, sizeof g.arc_span);
        put(&g.n_t, sizeof g.n_t);
        put(&g.t_max, sizeof g.t_max);
        put(&g.n_angles, sizeof g.n_angles);
    }
    // the requested fields the tuner keeps (it searches the tile shapes and groups)
    put(&opt.image_dtype, sizeof opt.image_dtype);
    put(&opt.adj_mode, sizeof opt.adj_mode);
    put(&opt.time_pair, sizeof opt.time_pair);
    put(&opt.adj_jblock, sizeof opt.adj_jblock);
    put(&device, sizeof device);
    return k;
}

template <typename F>
float time_ms(cudaStream_t st, int warm, int reps, F&& fn)
{
    for (int i = 0; i < warm; ++i)
        if (fn() != cudaSuccess) return -1.f;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.f;
    }
    float ms = -1.f;
    bool ok = cudaEventRecord(a, st) == cudaSuccess;
    for (int i = 0; i < reps && ok; ++i) ok = fn() == cudaSuccess;
    if (ok && cudaEventRecord(b, st) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
        cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
        ms /= reps;
    else
        ms = -1.f;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

Plan* try_build(const pat_geometry_t* geoms, int n, const pat_options_t& opt, cudaStream_t st)
{
    Plan* p = new (std::nothrow) Plan();
    if (!p) return nullptr;
    pat_status_t s;
    try {
        s = build_plan(*p, geoms, n, opt, st);
    } catch (...) {
        s = PAT_ERR_OOM;
    }
    if (s != PAT_OK) {
        free_plan_memory(*p);
        delete p;
        return nullptr;
    }
    return p;
}

void drop(Plan* p)
{
    if (!p) return;
    free_plan_memory(*p);
    delete p;
}

} // namespace

pat_status_t autotune_plan(Plan** out, const pat_geometry_t* geoms, int n_inst, const pat_options_t& opt_in,
                           cudaStream_t st)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PAT_ERR_CUDA;
    pat_options_t opt = opt_in;
    opt.tune = 0;
    const std::string key = tune_key(geoms, n_inst, opt, dev);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            Plan* p = try_build(geoms, n_inst, it->second, st);
            if (!p) return PAT_ERR_CUDA;
            *out = p;
            return PAT_OK;
        }
    }
    const bool bf16 = opt.image_dtype == PAT_BF16;
    int64_t f_elems = 0, g_elems = 0;
    int n_max = 0;
    for (int i = 0; i < n_inst; ++i) {
        f_elems += (int64_t)geoms[i].n * geoms[i].n;
        g_elems += (int64_t)geoms[i].n_det * geoms[i].n_t;
        n_max = std::max(n_max, geoms[i].n);
    }
    void* d_f = nullptr;
    float* d_g = nullptr;
    if (dev_malloc(reinterpret_cast<void**>(&d_f), (size_t)f_elems * (bf16 ? 2 : 4)) != cudaSuccess) {
        cudaGetLastError();
        return PAT_ERR_OOM;
    }
    if (dev_malloc(reinterpret_cast<void**>(&d_g), (size_t)g_elems * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_f);
        return PAT_ERR_OOM;
    }
    cudaMemsetAsync(d_f, 0, (size_t)f_elems * (bf16 ? 2 : 4), st);
    cudaMemsetAsync(d_g, 0, (size_t)g_elems * 4, st);

    // ---- forward candidates ---------------------------------------------
    // tile widths: automatic (fewest tile edges), full width, half, quarter
    const bool large = f_elems > (1 << 20);   // keep the search short on big plans
    std::vector<int> cols_cands = {0};
    for (int div : large ? std::vector<int>{2} : std::vector<int>{1, 2, 4})
        if (n_max / div >= 32) cols_cands.push_back((n_max + div - 1) / div);
    Plan* best = nullptr;
    float best_ms = 1e30f;
    pat_options_t best_opt = opt;
    const std::vector<int> ml_c = large ? std::vector<int>{16, 8} : std::vector<int>{32, 16, 8};
    const std::vector<int> qp_c = large ? std::vector<int>{256} : std::vector<int>{64, 128, 256};
    for (int ml : ml_c) {
        for (int qp : qp_c) {
            for (int cols : cols_cands) {
                pat_options_t o = opt;
                o.m_lanes = ml;
                o.q_piece = qp;
                o.tile_cols = cols;
                o.band_rows = 0;
                o.adj_mode = 2;      // the adjoint is tuned below; skip list building here
                o.adj_groups = 1;
                Plan* p = try_build(geoms, n_inst, o, st);
                if (!p) continue;
                const float ms = time_ms(st, 2, 5, [&] {
                    cudaError_t e = launch_circmean(p->dp, d_f, st);
                    return e == cudaSuccess ? launch_abel_fwd(p->dp, d_g, st) : e;
                });
                drop(p);
                if (ms > 0.f && ms < best_ms) {
                    best_ms = ms;
                    best_opt = o;
                }
            }
        }
    }
    // ---- time-stage cluster split (with the best forward shape) ------------
    if (opt.abel_split == 0) {
        best_ms = 1e30f;
        pat_options_t split_opt = best_opt;
        for (int cs : {1, 2, 4, 8}) {
            pat_options_t o = best_opt;
            o.abel_split = cs;
            Plan* p = try_build(geoms, n_inst, o, st);
            if (!p) continue;
            const float ms = time_ms(st, 2, 5, [&] {
                cudaError_t e = launch_abel_fwd(p->dp, d_g, st);
                return e == cudaSuccess ? launch_abel_adj(p->dp, d_g, st) : e;
            });
            drop(p);
            if (ms > 0.f && ms < best_ms) {
                best_ms = ms;
                split_opt = o;
            }
        }
        best_opt = split_opt;
    }
    // ---- adjoint candidates (with the best forward shape) ------------------
    best_ms = 1e30f;
    pat_options_t fwd_opt = best_opt;
    // the list modes cut each cell's list into groups, the enumeration mode its detectors
    // (and, when not fixed, the detector block size of the aligned code lists)
    struct AdjCand {
        int groups, jblock;
    };
    std::vector<AdjCand> adj_cands;
    // (16384: one block, i.e. every lane's list from the patch's first position)
    const std::vector<int> jb_c = opt.adj_jblock > 0 ? std::vector<int>{opt.adj_jblock}
                                  : large           ? std::vector<int>{8, 16}
                                                    : std::vector<int>{4, 8, 16, 16384};
    const std::vector<int> g_c = large ? std::vector<int>{0, 4, 8} : std::vector<int>{0, 1, 2, 4, 8};
    for (int gcount : g_c)
        for (int jb : jb_c) adj_cands.push_back({gcount, jb});
    for (auto& ac : adj_cands) {
        pat_options_t o = fwd_opt;
        o.adj_mode = opt.adj_mode;
        o.adj_groups = ac.groups;
        o.adj_jblock = ac.jblock;
        Plan* p = try_build(geoms, n_inst, o, st);
        if (!p) continue;
        const float ms = time_ms(st, 2, 5, [&] {
            cudaError_t e = launch_abel_adj(p->dp, d_g, st);
            return e == cudaSuccess ? launch_adjoint_gather(p->dp, d_f, st) : e;
        });
        if (ms > 0.f && ms < best_ms) {
            best_ms = ms;
            drop(best);
            best = p;
            best_opt = o;
        } else {
            drop(p);
        }
    }
    cudaFree(d_f);
    cudaFree(d_g);
    if (!best) return PAT_ERR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best_opt;
    }
    best->opt.tune = 1;
    *out = best;
    return PAT_OK;
}

} // namespace patgpu
