// abel.cu — the time stage of A and of A^T.
//
// Forward:  g[j][kk] = (1/K) sum_{m <= kk+2} P[kk][m] M[j][m]
// Adjoint:  Mbar[j][m] = sum_{kk >= m-2} P[kk][m] gbar[j][kk]
//
// P is the product-integrated Abel kernel followed by the midpoint time
// derivative (the 2D Poisson formula of the wave problem Eq. (1)-(2)); it is
// lower triangular plus one super-diagonal, so a tile of outputs only needs
// the band of the contraction where its slice of P is nonzero.
//
// Both stages are C[j][x] = sum_k A[j][k] B[k][x] over a 32 x 32 output tile
// (32 detectors, 32 times or radii): A = M and B = P^T for the forward,
// A = gbar and B = P for the adjoint.  Warp w owns detectors 4w .. 4w+3 and
// lane l output x0 + l, so each thread keeps four FP32 accumulators and each
// staged element of P serves 32 detectors.  Every output is a sequential
// FMA chain over k in increasing order.
//
// The contraction runs in chunks of 32 rows through a ring of kStages
// shared-memory stages filled by asynchronous copies (16-byte copies for the
// chunk of P, 4-byte zero-filling copies that write the chunk of A already
// transposed, so that a warp reads its four detectors as one broadcast
// 16-byte load), kStages - 1 chunks ahead of the FMAs: a CTA's loads are all
// in flight at once for short contractions.
//
// When a plan has fewer tiles than SMs, a thread-block cluster of 2, 4 or 8 CTAs
// shares each tile: rank r takes the r-th share of the chunks, and rank 0
// adds the partial tiles in rank order through distributed shared memory
// (deterministic; no global atomics).
#include <cooperative_groups.h>

#include "device_common.cuh"
#include "kernels.h"

namespace patgpu {

namespace cg = cooperative_groups;

static_assert(kAbelJ == 4 * kAbelWarps && kAbelX == kWarp && kAbelKC == 32, "Abel tile shape");

namespace {
constexpr int kStages = 6;
struct AbelSmem {
    float A[kStages][kAbelKC][kAbelJ + 4];   // [stage][k][detector], rows 16-byte aligned
    float B[kStages][kAbelKC][kAbelX];       // [stage][k][output]
    float part[kAbelJ][kAbelX];              // partial tile read by cluster rank 0
};
} // namespace

// FWD: gin unused, gout = g (gsub nullable: gout = A f - gsub).
// FWD && DUAL: gout = y (read and written), gsub = g:
//   y <- (y + sigma (A f - g)) * inv1ps, the data-term dual step of the
//   primal-dual iteration (the proximal map of the conjugate of
//   1/2 ||. - g||^2), with inv1ps = 1 / (1 + sigma).
// ADJ: gin = gbar, gout unused (writes Mbar in the plan workspace).
template <bool FWD, bool DUAL>
__global__ void __launch_bounds__(kAbelWarps * kWarp) k_abel(DevPlan dp, const float* __restrict__ gin,
                                                             float* __restrict__ gout,
                                                             const float* __restrict__ gsub, int cs, float sigma,
                                                             float inv1ps)
{
    extern __shared__ __align__(16) unsigned char abel_smem[];
    AbelSmem& sm = *reinterpret_cast<AbelSmem*>(abel_smem);
    const int rank = (int)(blockIdx.x % (unsigned)cs);
    const TimeTile t = (FWD ? dp.fwd_tiles : dp.adj_tiles)[blockIdx.x / cs];
    const InstDev in = dp.inst[t.inst];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;

    const float* A;   // A[j][k] with row pitch a_pitch, valid for k < a_len
    const float* B;   // B[k][x] with row pitch b_pitch (zero padded to the chunk grid)
    int a_pitch, a_len, b_pitch, k_begin, k_end;
    if (FWD) {
        A = dp.msum + in.mbar_off;
        a_pitch = in.m_pitch;
        a_len = in.n_r;
        B = dp.P + in.p_off + (size_t)in.n_tp * in.n_rp;
        b_pitch = in.n_tp;
        k_begin = 0;
        k_end = min(in.n_r, t.x0 + kAbelX + 2);
    } else {
        A = gin + in.g_off;
        a_pitch = in.n_t;
        a_len = in.n_t;
        B = dp.P + in.p_off;
        b_pitch = in.n_rp;
        k_begin = max(0, t.x0 - 2) & ~(kAbelKC - 1);
        k_end = in.n_t;
    }
    const int nchunks = (k_end - k_begin + kAbelKC - 1) / kAbelKC;
    const int per = (nchunks + cs - 1) / cs;
    const int c_lo = min(nchunks, rank * per), c_hi = min(nchunks, c_lo + per);

    // copy roles: A elements (detector ja, rows ka .. ka+3); B (row rb, columns cb .. cb+3)
    const int ja = tid >> 3, ka = (tid & 7) * 4;
    const int rb = tid >> 3, cb = (tid & 7) * 4;
    const bool ja_ok = t.j0 + ja < in.n_det;
    const float* Arow = A + (size_t)(ja_ok ? t.j0 + ja : 0) * a_pitch;
    // issues chunk c into its stage; always commits one group (empty past the end)
    auto issue = [&](int c) {
        if (c < c_hi) {
            const int st = (c - c_lo) % kStages;
            const int k0 = k_begin + c * kAbelKC;
            cp_async16(&sm.B[st][rb][cb], B + (size_t)(k0 + rb) * b_pitch + t.x0 + cb);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = k0 + ka + i;
                const bool ok = ja_ok && k < a_len;
                cp_async4_zfill(&sm.A[st][ka + i][ja], ok ? Arow + k : Arow, ok);
            }
        }
        cp_async_commit();
    };

    pdl_wait();   // M (forward) or gbar (adjoint) come from the previous kernel
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int i = 0; i < kStages - 1; ++i) issue(c_lo + i);
    for (int c = c_lo; c < c_hi; ++c) {
        const int st = (c - c_lo) % kStages;
        cp_async_wait_group<kStages - 2>();   // chunk c has landed (this thread's copies)
        __syncthreads();                      // ... and every thread's
#pragma unroll 8
        for (int k = 0; k < kAbelKC; ++k) {
            const float b = sm.B[st][k][lane];
            const float4 a = *reinterpret_cast<const float4*>(&sm.A[st][k][4 * w]);
            acc.x = fmaf(b, a.x, acc.x);
            acc.y = fmaf(b, a.y, acc.y);
            acc.z = fmaf(b, a.z, acc.z);
            acc.w = fmaf(b, a.w, acc.w);
        }
        __syncthreads();                      // stage st is free again
        issue(c + kStages - 1);
    }
    cp_async_wait_group<0>();

    if (cs > 1) {
        cg::cluster_group cluster = cg::this_cluster();
        sm.part[4 * w + 0][lane] = acc.x;
        sm.part[4 * w + 1][lane] = acc.y;
        sm.part[4 * w + 2][lane] = acc.z;
        sm.part[4 * w + 3][lane] = acc.w;
        cluster.sync();
        if (rank == 0) {
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int r = 0; r < cs; ++r) {
                const float* pr = cluster.map_shared_rank(&sm.part[0][0], r);
                s.x += pr[(4 * w + 0) * kAbelX + lane];
                s.y += pr[(4 * w + 1) * kAbelX + lane];
                s.z += pr[(4 * w + 2) * kAbelX + lane];
                s.w += pr[(4 * w + 3) * kAbelX + lane];
            }
            acc = s;
        }
        cluster.sync();   // keep every rank's partial alive until rank 0 has read it
        if (rank != 0) return;
    }

    const float r4[4] = {acc.x, acc.y, acc.z, acc.w};
    const int x = t.x0 + lane;
    if (FWD) {
        if (x < in.n_t) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int j = t.j0 + 4 * w + i;
                if (j >= in.n_det) break;
                const size_t o = in.g_off + (size_t)j * in.n_t + x;
                const float v = r4[i] * in.inv_K;
                if (DUAL)
                    gout[o] = fmaf(sigma, v - gsub[o], gout[o]) * inv1ps;
                else
                    gout[o] = gsub ? v - gsub[o] : v;
            }
        }
    } else {
        if (x < in.n_r) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int j = t.j0 + 4 * w + i;
                if (j >= in.n_det) break;
                dp.mbar[in.mbar_off + (size_t)j * in.m_pitch + x] = r4[i];
            }
        }
    }
}

namespace {
template <bool FWD, bool DUAL = false>
cudaError_t launch_abel(const DevPlan& dp, int tiles, int cs, const float* gin, float* gout, const float* gsub,
                        cudaStream_t st, float sigma = 0.f, float inv1ps = 1.f)
{
    if (tiles == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_abel<FWD, DUAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(AbelSmem));
    if (e != cudaSuccess) return e;
    return launch_pdl(k_abel<FWD, DUAL>, dim3((unsigned)(tiles * cs)), dim3(kAbelWarps * kWarp), sizeof(AbelSmem),
                      st, cs, dp, gin, gout, gsub, cs, sigma, inv1ps);
}
} // namespace

cudaError_t launch_abel_fwd(const DevPlan& dp, float* g, cudaStream_t st, const float* gsub)
{
    return launch_abel<true>(dp, dp.n_fwd_tiles, dp.abel_cluster_fwd, nullptr, g, gsub, st);
}

cudaError_t launch_abel_fwd_dual(const DevPlan& dp, float* y, const float* g, float sigma, float inv1ps,
                                 cudaStream_t st)
{
    return launch_abel<true, true>(dp, dp.n_fwd_tiles, dp.abel_cluster_fwd, nullptr, y, g, st, sigma, inv1ps);
}

cudaError_t launch_abel_adj(const DevPlan& dp, const float* g, cudaStream_t st)
{
    return launch_abel<false>(dp, dp.n_adj_tiles, dp.abel_cluster_adj, g, nullptr, nullptr, st);
}

} // namespace patgpu
