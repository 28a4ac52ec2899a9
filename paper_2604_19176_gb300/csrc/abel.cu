// abel.cu — the time stage of A and of A^T.
//
// Forward:  g[j][kk] = (1/K) sum_{m <= kk+2} P[kk][m] M[j][m]
// Adjoint:  Mbar[j][m] = sum_{kk >= m-2} P[kk][m] gbar[j][kk]
//
// P is the product-integrated Abel kernel followed by the midpoint time
// derivative (the 2D Poisson formula of the wave problem Eq. (1)-(2)); it is
// lower triangular plus one super-diagonal.  A CTA computes 32 outputs (one
// per lane) for 4 detectors; its 8 warps split the contracted index into
// contiguous ranges (so each SM keeps many independent loads of P in flight),
// each lane streams its column of P (P^T for the forward: a warp reads 128
// contiguous bytes per step), the 4 detectors' rows sit in shared memory as
// float4, and the 8 partial sums are added in warp order (deterministic).
// The triangle is skipped: the contracted range stops (forward) or starts
// (adjoint) where the tile's band of P ends.
#include "device_common.cuh"
#include "kernels.h"

namespace patgpu {

static_assert(kAbelJ == 4, "the Abel kernels keep 4 detectors in a float4");

namespace {
__device__ __forceinline__ void fma4(float4& acc, float p, const float4 v)
{
    acc.x = fmaf(p, v.x, acc.x);
    acc.y = fmaf(p, v.y, acc.y);
    acc.z = fmaf(p, v.z, acc.z);
    acc.w = fmaf(p, v.w, acc.w);
}

// Adds the per-warp partials in warp order; returns the total in warp 0.
__device__ __forceinline__ float4 reduce_warps(float4 acc, float4 (*red)[kWarp])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
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
} // namespace

__global__ void __launch_bounds__(kAbelWarps * kWarp) k_abel_fwd(DevPlan dp, float* __restrict__ g)
{
    extern __shared__ float4 sM4[]; // [kAbelChunk]: M of the 4 detectors at one radius
    __shared__ float4 red[kAbelWarps][kWarp];
    const TimeTile t = dp.fwd_tiles[blockIdx.x];
    const InstDev in = dp.inst[t.inst];
    const int n_r = in.n_r, n_t = in.n_t;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int kk = t.x0 + lane;
    const int m_end = min(n_r, t.x0 + kAbelX + 2);
    const float* PT = dp.P + in.p_off + (size_t)n_t * n_r; // P^T: [m][kk]
    const float* M = dp.msum + in.mbar_off;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int mc = 0; mc < m_end; mc += kAbelChunk) {
        const int len = min(kAbelChunk, m_end - mc);
        __syncthreads();
        for (int e = threadIdx.x; e < len; e += blockDim.x) {
            const int m = mc + e;
            float4 v;
            v.x = (t.j0 + 0 < in.n_det) ? M[(size_t)(t.j0 + 0) * n_r + m] : 0.f;
            v.y = (t.j0 + 1 < in.n_det) ? M[(size_t)(t.j0 + 1) * n_r + m] : 0.f;
            v.z = (t.j0 + 2 < in.n_det) ? M[(size_t)(t.j0 + 2) * n_r + m] : 0.f;
            v.w = (t.j0 + 3 < in.n_det) ? M[(size_t)(t.j0 + 3) * n_r + m] : 0.f;
            sM4[e] = v;
        }
        __syncthreads();
        const int per = (len + kAbelWarps - 1) / kAbelWarps;
        const int mb = w * per, me = min(len, mb + per);
        if (kk < n_t) {
            const float* pc = PT + (size_t)mc * n_t + kk;
#pragma unroll 8
            for (int m = mb; m < me; ++m) fma4(acc, __ldg(pc + (size_t)m * n_t), sM4[m]);
        }
    }
    const float4 s = reduce_warps(acc, red);
    if (w == 0 && kk < n_t) {
        const float sc = in.inv_K;
        float* out = g + in.g_off + kk;
        if (t.j0 + 0 < in.n_det) out[(size_t)(t.j0 + 0) * n_t] = s.x * sc;
        if (t.j0 + 1 < in.n_det) out[(size_t)(t.j0 + 1) * n_t] = s.y * sc;
        if (t.j0 + 2 < in.n_det) out[(size_t)(t.j0 + 2) * n_t] = s.z * sc;
        if (t.j0 + 3 < in.n_det) out[(size_t)(t.j0 + 3) * n_t] = s.w * sc;
    }
}

__global__ void __launch_bounds__(kAbelWarps * kWarp) k_abel_adj(DevPlan dp, const float* __restrict__ g)
{
    extern __shared__ float4 sG4[]; // [kAbelChunk]: gbar of the 4 detectors at one time
    __shared__ float4 red[kAbelWarps][kWarp];
    const TimeTile t = dp.adj_tiles[blockIdx.x];
    const InstDev in = dp.inst[t.inst];
    const int n_r = in.n_r, n_t = in.n_t;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m = t.x0 + lane;
    const int k_begin = max(0, t.x0 - 2);
    const float* P = dp.P + in.p_off; // [kk][m]
    const float* gi = g + in.g_off;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int kc = k_begin; kc < n_t; kc += kAbelChunk) {
        const int len = min(kAbelChunk, n_t - kc);
        __syncthreads();
        for (int e = threadIdx.x; e < len; e += blockDim.x) {
            const int kk = kc + e;
            float4 v;
            v.x = (t.j0 + 0 < in.n_det) ? __ldg(gi + (size_t)(t.j0 + 0) * n_t + kk) : 0.f;
            v.y = (t.j0 + 1 < in.n_det) ? __ldg(gi + (size_t)(t.j0 + 1) * n_t + kk) : 0.f;
            v.z = (t.j0 + 2 < in.n_det) ? __ldg(gi + (size_t)(t.j0 + 2) * n_t + kk) : 0.f;
            v.w = (t.j0 + 3 < in.n_det) ? __ldg(gi + (size_t)(t.j0 + 3) * n_t + kk) : 0.f;
            sG4[e] = v;
        }
        __syncthreads();
        const int per = (len + kAbelWarps - 1) / kAbelWarps;
        const int kb = w * per, ke = min(len, kb + per);
        if (m < n_r) {
            const float* pc = P + (size_t)kc * n_r + m;
#pragma unroll 8
            for (int k = kb; k < ke; ++k) fma4(acc, __ldg(pc + (size_t)k * n_r), sG4[k]);
        }
    }
    const float4 s = reduce_warps(acc, red);
    if (w == 0 && m < n_r) {
        float* out = dp.mbar + in.mbar_off + m;
        if (t.j0 + 0 < in.n_det) out[(size_t)(t.j0 + 0) * n_r] = s.x;
        if (t.j0 + 1 < in.n_det) out[(size_t)(t.j0 + 1) * n_r] = s.y;
        if (t.j0 + 2 < in.n_det) out[(size_t)(t.j0 + 2) * n_r] = s.z;
        if (t.j0 + 3 < in.n_det) out[(size_t)(t.j0 + 3) * n_r] = s.w;
    }
}

cudaError_t launch_abel_fwd(const DevPlan& dp, float* g, cudaStream_t st)
{
    if (dp.n_fwd_tiles == 0) return cudaSuccess;
    k_abel_fwd<<<dp.n_fwd_tiles, kAbelWarps * kWarp, dp.abel_smem_bytes, st>>>(dp, g);
    return cudaGetLastError();
}

cudaError_t launch_abel_adj(const DevPlan& dp, const float* g, cudaStream_t st)
{
    if (dp.n_adj_tiles == 0) return cudaSuccess;
    k_abel_adj<<<dp.n_adj_tiles, kAbelWarps * kWarp, dp.abel_smem_bytes, st>>>(dp, g);
    return cudaGetLastError();
}

} // namespace patgpu
