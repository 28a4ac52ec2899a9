// kernels.h — launchers of the device kernels (host-callable, enqueue only).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pat_internal.h"

namespace patgpu {

constexpr int kCircThreads = 512;   // threads per circular-mean CTA (16 warps)

// Launches fn<<<grid, block, smem, st>>>(args...) with programmatic stream
// serialization (the kernel must call pdl_wait before it reads or writes
// memory that earlier work in the stream touches), and optionally as
// clusters of `cluster` CTAs along x.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, int cluster,
                       Args&&... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    int na = 1;
    if (cluster > 1) {
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = (unsigned)cluster;
        attr[1].val.clusterDim.y = 1;
        attr[1].val.clusterDim.z = 1;
        na = 2;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, fn, static_cast<KArgs>(args)...);
}

cudaError_t launch_circmean(const DevPlan& dp, const void* f, cudaStream_t st, bool msum = true);
cudaError_t launch_abel_fwd(const DevPlan& dp, float* g, cudaStream_t st, const float* gsub = nullptr);
cudaError_t launch_abel_adj(const DevPlan& dp, const float* g, cudaStream_t st);
// Fused time stage (radius sums, forward, residual or dual update, adjoint)
// of the steps: Mbar from the circular-mean partial slots in one launch.
cudaError_t launch_time_pair(const DevPlan& dp, const float* g, float* y, bool dual, float sigma, float inv1ps,
                             cudaStream_t st);
// Clusters of the fused time stage that fit the GPU at once (0: cannot run).
int time_pair_clusters(int smem_bytes);
cudaError_t launch_adjoint_gather(const DevPlan& dp, void* f, cudaStream_t st);
// Adjoint cell sums only (no combine), for the fused TV step.
cudaError_t launch_adjoint_cells(const DevPlan& dp, cudaStream_t st);
// Fused combine + TV gradient + projected update:
// f_out = [f_in - tau (A^T r + lam grad TV_eps(f_in))]_+ ; delta as pat_descent_step.
cudaError_t launch_tv_update(const DevPlan& dp, const float* f_in, float* f_out, float tau, float lam, float eps,
                             int nonneg, float* delta, cudaStream_t st);
// Primal-dual TV iteration (Eq. (4)): dual step of the TV term, in place,
// p <- proj_{|p_i| <= alpha}(p + sigma grad fbar); and the primal step with
// extrapolation from the adjoint cell sums, f <- max(0, f - tau (A^T y +
// grad^T p + beta (mean f - c) / P)), fbar <- 2 f_new - f_old; delta as
// pat_descent_step; fmean (nullable, per instance) read as the mean of f and
// overwritten with the mean of f_new (the penalty term needs it).
cudaError_t launch_pdhg_dual_tv(const DevPlan& dp, const float* fbar, float* px, float* py, float sigma, float alpha,
                                cudaStream_t st);
cudaError_t launch_pdhg_primal(const DevPlan& dp, float* f, float* fbar, const float* px, const float* py, float tau,
                               int nonneg, float* fmean, float beta, float mean_target, float* delta, cudaStream_t st);
// Time stage of A with the data-term dual step of the primal-dual iteration
// as its epilogue: y <- (y + sigma (A fbar - g)) * inv1ps, inv1ps = 1/(1+sigma).
cudaError_t launch_abel_fwd_dual(const DevPlan& dp, float* y, const float* g, float sigma, float inv1ps,
                                 cudaStream_t st);
cudaError_t launch_tv(const DevPlan& dp, const float* f, float eps, float* grad, float* value, cudaStream_t st);
cudaError_t launch_residual(const float* a, const float* b, float* r, float scale, int64_t n, cudaStream_t st);
cudaError_t launch_descent(const DevPlan& dp, float* f, const float* adj, const float* tvg, float tau, float lam,
                           int nonneg, float* delta, cudaStream_t st);
cudaError_t launch_count_samples(const DevPlan& dp, int inst_idx, int n_det, unsigned long long* out,
                                 cudaStream_t st);

// Occupancy of the circular-mean kernel for the plan's tile shape, and of the
// adjoint cell kernel (256-thread CTAs).
int circmean_blocks_per_sm(int m_lanes, bool bf16, int smem_bytes);
int adj_cells_blocks_per_sm();
// Resident CTAs per SM of the list gather: lm 0 = code lists, 1 = fraction
// lists, 2 = run-pair code lists.
int adj_list_blocks_per_sm(int lm);

// Fraction-list building at plan creation (layouts in pat_internal.h):
// counts the samples of every cell of instance inst_idx into `counts`
// (out == nullptr), or fills the lists given the (patch, part) block bases.
cudaError_t launch_adj_frac_build(const DevPlan& dp, int inst_idx, int n, int32_t* counts, const int64_t* pbase,
                                  uint32_t* out, cudaStream_t st);

// Code-list building: with out == nullptr, atomicMax of every cell's entry
// count per detector block into seg (per patch: nblk blocks + 1, zeroed by
// the caller); else writes every entry at its aligned position (seg holding
// the segment starts and each patch's length in vectors, out pre-filled
// with null codes).  pairs: run-pair codes.
cudaError_t launch_adj_seg(const DevPlan& dp, int inst_idx, int n, bool pairs, int jblock, int nblk, int32_t* seg,
                           const int64_t* pbase, uint32_t* out, cudaStream_t st);

// p[0 .. n) = v
cudaError_t launch_fill_u32(uint32_t* p, int64_t n, uint32_t v, cudaStream_t st);

} // namespace patgpu
