// abel.cu — the time stage of A and of A^T.
//
// Forward:  g[j][kk] = (1/K) sum_{m <= kk+2} P[kk][m] M[j][m]
// Adjoint:  Mbar[j][m] = sum_{kk >= m-2} P[kk][m] gbar[j][kk]
//
// P is the product-integrated Abel kernel followed by the midpoint time
// derivative (the 2D Poisson formula of the wave problem Eq. (1)-(2)); it is
// lower triangular plus one super-diagonal.  A CTA computes 32 outputs (one
// per lane) for 4 detectors.  The 32-column slice of P^T (forward) or P
// (adjoint) that the tile needs is staged in shared memory in chunks of rows
// by 16-byte asynchronous copies spread over the CTA; the 4 detectors' rows
// of M (or gbar) are staged by plain loads.  The 8 warps
// split each chunk's rows and their partial sums are added in warp order
// (deterministic).  The triangle is skipped: rows stop (forward) or start
// (adjoint) where the tile's band of P ends.
#include "device_common.cuh"
#include "kernels.h"

namespace patgpu {

static_assert(kAbelJ == 4, "the Abel kernels keep 4 detectors in a float4");

namespace {
// Adds the per-warp partials in warp order; returns the total in warp 0.
__device__ __forceinline__ float4 reduce_warps(float4 acc, float4 (*red)[kWarp])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    red[w][lane] = acc;
    __syncthreads();
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < kAbelWarps; ++i) {
            const float4 v = red[i][lane];
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
    }
    return s;
}

// Copies rows [r0, r0 + nrows) of a 32-column slice (row pitch `pitch`
// floats, slice starting at column c0, both multiples of 32) into
// sP[nrows][32] with 16-byte asynchronous copies spread over the CTA.
__device__ __forceinline__ void stage_slice(float* sP, const float* src, int pitch, int c0, int r0, int nrows)
{
    for (int e = threadIdx.x; e < nrows * 8; e += blockDim.x) {
        const int r = e >> 3, c = (e & 7) * 4;
        cp_async16(sP + r * kWarp + c, src + (size_t)(r0 + r) * pitch + c0 + c);
    }
}
} // namespace

// gsub (nullable): when given, the output is A f - gsub (the data residual).
__global__ void __launch_bounds__(kAbelWarps * kWarp) k_abel_fwd(DevPlan dp, float* __restrict__ g,
                                                                 const float* __restrict__ gsub)
{
    extern __shared__ __align__(128) float smem_f[];
    float* sP = smem_f;                           // [kAbelChunk][32]
    float4* sM4 = reinterpret_cast<float4*>(smem_f + kAbelChunk * kWarp); // [kAbelChunk]
    __shared__ float4 red[kAbelWarps][kWarp];
    const TimeTile t = dp.fwd_tiles[blockIdx.x];
    const InstDev in = dp.inst[t.inst];
    const int n_r = in.n_r, n_t = in.n_t;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int kk = t.x0 + lane;
    const int m_end = min(n_r, t.x0 + kAbelX + 2);
    const float* PT = dp.P + in.p_off + (size_t)n_t * in.n_rp; // P^T: [m][kk], pitch n_tp
    const float* M = dp.msum + in.mbar_off;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int mc = 0; mc < m_end; mc += kAbelChunk) {
        const int len = min(kAbelChunk, m_end - mc);
        __syncthreads(); // previous chunk consumed
        stage_slice(sP, PT, in.n_tp, t.x0, mc, len);
        for (int e = threadIdx.x; e < len; e += blockDim.x) {
            const int m = mc + e;
            float4 v;
            v.x = (t.j0 + 0 < in.n_det) ? __ldg(M + (size_t)(t.j0 + 0) * in.n_rp + m) : 0.f;
            v.y = (t.j0 + 1 < in.n_det) ? __ldg(M + (size_t)(t.j0 + 1) * in.n_rp + m) : 0.f;
            v.z = (t.j0 + 2 < in.n_det) ? __ldg(M + (size_t)(t.j0 + 2) * in.n_rp + m) : 0.f;
            v.w = (t.j0 + 3 < in.n_det) ? __ldg(M + (size_t)(t.j0 + 3) * in.n_rp + m) : 0.f;
            sM4[e] = v;
        }
        cp_async_wait_all();
        __syncthreads();
        for (int m = w; m < len; m += kAbelWarps) {
            const float p = sP[m * kWarp + lane];
            const float4 v = sM4[m];
            acc.x = fmaf(p, v.x, acc.x);
            acc.y = fmaf(p, v.y, acc.y);
            acc.z = fmaf(p, v.z, acc.z);
            acc.w = fmaf(p, v.w, acc.w);
        }
    }
    const float4 s = reduce_warps(acc, red);
    if (w == 0 && kk < n_t) {
        const float sc = in.inv_K;
        const size_t o = in.g_off + kk;
        float* out = g + o;
        const float r[4] = {s.x * sc, s.y * sc, s.z * sc, s.w * sc};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (t.j0 + i >= in.n_det) break;
            const size_t jo = (size_t)(t.j0 + i) * n_t;
            out[jo] = gsub ? r[i] - gsub[o + jo] : r[i];
        }
    }
}

__global__ void __launch_bounds__(kAbelWarps * kWarp) k_abel_adj(DevPlan dp, const float* __restrict__ g)
{
    extern __shared__ __align__(128) float smem_f[];
    float* sP = smem_f;                           // [kAbelChunk][32]
    float4* sG4 = reinterpret_cast<float4*>(smem_f + kAbelChunk * kWarp); // [kAbelChunk]
    __shared__ float4 red[kAbelWarps][kWarp];
    const TimeTile t = dp.adj_tiles[blockIdx.x];
    const InstDev in = dp.inst[t.inst];
    const int n_r = in.n_r, n_t = in.n_t;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m = t.x0 + lane;
    const int k_begin = max(0, t.x0 - 2);
    const float* P = dp.P + in.p_off; // [kk][m], pitch n_rp
    const float* gi = g + in.g_off;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int kc = k_begin; kc < n_t; kc += kAbelChunk) {
        const int len = min(kAbelChunk, n_t - kc);
        __syncthreads();
        stage_slice(sP, P, in.n_rp, t.x0, kc, len);
        for (int e = threadIdx.x; e < len; e += blockDim.x) {
            const int kk = kc + e;
            float4 v;
            v.x = (t.j0 + 0 < in.n_det) ? __ldg(gi + (size_t)(t.j0 + 0) * n_t + kk) : 0.f;
            v.y = (t.j0 + 1 < in.n_det) ? __ldg(gi + (size_t)(t.j0 + 1) * n_t + kk) : 0.f;
            v.z = (t.j0 + 2 < in.n_det) ? __ldg(gi + (size_t)(t.j0 + 2) * n_t + kk) : 0.f;
            v.w = (t.j0 + 3 < in.n_det) ? __ldg(gi + (size_t)(t.j0 + 3) * n_t + kk) : 0.f;
            sG4[e] = v;
        }
        cp_async_wait_all();
        __syncthreads();
        for (int k = w; k < len; k += kAbelWarps) {
            const float p = sP[k * kWarp + lane];
            const float4 v = sG4[k];
            acc.x = fmaf(p, v.x, acc.x);
            acc.y = fmaf(p, v.y, acc.y);
            acc.z = fmaf(p, v.z, acc.z);
            acc.w = fmaf(p, v.w, acc.w);
        }
    }
    const float4 s = reduce_warps(acc, red);
    if (w == 0 && m < n_r) {
        float* out = dp.mbar + in.mbar_off + m;
        if (t.j0 + 0 < in.n_det) out[(size_t)(t.j0 + 0) * in.n_rp] = s.x;
        if (t.j0 + 1 < in.n_det) out[(size_t)(t.j0 + 1) * in.n_rp] = s.y;
        if (t.j0 + 2 < in.n_det) out[(size_t)(t.j0 + 2) * in.n_rp] = s.z;
        if (t.j0 + 3 < in.n_det) out[(size_t)(t.j0 + 3) * in.n_rp] = s.w;
    }
}

static cudaError_t set_abel_smem(const void* fn, int bytes)
{
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_abel_fwd(const DevPlan& dp, float* g, cudaStream_t st, const float* gsub)
{
    if (dp.n_fwd_tiles == 0) return cudaSuccess;
    cudaError_t e = set_abel_smem(reinterpret_cast<const void*>(k_abel_fwd), dp.abel_smem_bytes);
    if (e != cudaSuccess) return e;
    k_abel_fwd<<<dp.n_fwd_tiles, kAbelWarps * kWarp, dp.abel_smem_bytes, st>>>(dp, g, gsub);
    return cudaGetLastError();
}

cudaError_t launch_abel_adj(const DevPlan& dp, const float* g, cudaStream_t st)
{
    if (dp.n_adj_tiles == 0) return cudaSuccess;
    cudaError_t e = set_abel_smem(reinterpret_cast<const void*>(k_abel_adj), dp.abel_smem_bytes);
    if (e != cudaSuccess) return e;
    k_abel_adj<<<dp.n_adj_tiles, kAbelWarps * kWarp, dp.abel_smem_bytes, st>>>(dp, g);
    return cudaGetLastError();
}

} // namespace patgpu
