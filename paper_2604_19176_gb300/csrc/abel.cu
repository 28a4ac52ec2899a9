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


// ---------------------------------------------------------------------------
// Fused time stage of the TV and primal-dual steps: radius sums M, forward
// g = M P^T / K, residual, adjoint Mbar = r P, for kTimeJ detectors per
// thread-block cluster of kTimeCS CTAs, in one launch.
//
// Every step is row-local (a detector's outputs need only that detector's
// rows), so a cluster owns whole rows and nothing synchronises across the
// grid:
//   1. each CTA adds the circular-mean partial slots of its share of the
//      radius chunks (in slot order, as k_msum) into its shared copy of M;
//      cluster barrier; it copies the other shares from the other CTAs'
//      shared memory, so each CTA holds the group's rows of M;
//   2. forward: each CTA computes its time chunks of g and the residual
//      r = g - data (or the dual update of y), kept in shared memory;
//   3. cluster barrier; each CTA copies the other CTAs' residual chunks;
//   4. adjoint: each CTA computes its radius chunks of Mbar.
// Chunks of 32 outputs go to the ranks in boustrophedon order (0..7, 7..0,
// 0..7, ...), which evens out the triangle of P (late forward chunks and
// early adjoint chunks are the long ones).  The contraction of a chunk is
// cut into blocks of 32 rows; warp w takes blocks w, w + 8, ... of each of
// its CTA's chunks and walks them without CTA-wide synchronisation: a lane
// owns one output for all kTimeJ detectors (kTimeJ accumulators; a row's
// detector values are broadcast 16-byte shared-memory loads), and the block's 32
// values of P for that output sit in registers, loaded one block ahead
// from the plan's blocked copy of P (8 warp-wide 512-byte loads per block;
// the loads of the first block are issued before the dependency wait: P
// does not depend on the data).  After a phase the warps' partial sums are
// added in warp order (deterministic) and the epilogue runs.
// ---------------------------------------------------------------------------
namespace {
constexpr int kTimeThreads = kTimeWarps * kWarp;
constexpr int kTimeSub = kTimeWarps / kTimeJ;   // warps per detector in the sums and epilogues
static_assert(kTimeJ % 4 == 0 && kTimeWarps % kTimeJ == 0, "fused time stage shape");

// chunk p of a rank (p = 0, 1, ...) and the rank that owns chunk c
__device__ __forceinline__ int time_chunk(int p, int rank)
{
    return p * kTimeCS + ((p & 1) ? kTimeCS - 1 - rank : rank);
}
__device__ __forceinline__ int time_owner(int c)
{
    const int p = c / kTimeCS, r = c - p * kTimeCS;
    return (p & 1) ? kTimeCS - 1 - r : r;
}

// Contraction blocks [lo, hi) (32 rows each) of output chunk c: forward chunk
// c contracts radii [0, min(n_r, 32 c + 34)), adjoint chunk c times
// [max(0, 32 c - 2), n_t) (P is zero elsewhere; the padded rows of P, P^T and
// of the staged operands are zero).
__device__ __forceinline__ void time_blocks(int phase, int c, int n_r, int n_tc, int& lo, int& hi)
{
    lo = phase == 0 ? 0 : max(0, 32 * c - 2) >> 5;
    hi = phase == 0 ? (min(n_r, 32 * c + 34) + 31) >> 5 : n_tc;
}

struct TItem {
    int phase;   // 0 forward, 1 adjoint
    int p;       // the CTA's chunk index (slot of the partial sums)
    int c;       // output chunk
    int kc;      // contraction block
    bool last;   // this warp's last block of the chunk
};

// The blocks of one warp: for each of its CTA's forward chunks, then each
// adjoint chunk, blocks lo + w, lo + w + kTimeWarps, ... below hi.
struct TWalk {
    int phase = 0, p = 0, kc = -1;
    int rank, w, n_tc, n_rc, n_r;
    __device__ TWalk(int rank_, int w_, int n_tc_, int n_rc_, int n_r_)
        : rank(rank_), w(w_), n_tc(n_tc_), n_rc(n_rc_), n_r(n_r_) {}
    __device__ bool next(TItem& it)
    {
        for (;;) {
            if (phase > 1) return false;
            const int c = time_chunk(p, rank);
            if (c >= (phase == 0 ? n_tc : n_rc)) {
                ++phase;
                p = 0;
                kc = -1;
                continue;
            }
            int lo, hi;
            time_blocks(phase, c, n_r, n_tc, lo, hi);
            const int k = kc < 0 ? lo + w : kc + kTimeWarps;
            if (k >= hi) {
                ++p;
                kc = -1;
                continue;
            }
            kc = k;
            it.phase = phase;
            it.p = p;
            it.c = c;
            it.kc = k;
            it.last = k + kTimeWarps >= hi;
            return true;
        }
    }
};

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }
} // namespace

// DUAL = false: r = A f - g (y, if not null, receives r).
// DUAL = true:  y <- (y + sigma (A f - g)) * inv1ps and r = the new y.
template <bool DUAL>
__global__ void __launch_bounds__(kTimeThreads, 2) k_time_pair(DevPlan dp, const float* __restrict__ gdata,
                                                              float* __restrict__ y, float sigma, float inv1ps)
{
    extern __shared__ __align__(16) unsigned char tp_smem[];
    const int nch = dp.time_chunks;                                  // most chunks of a CTA in one phase
    float* Ms = reinterpret_cast<float*>(tp_smem);                   // [radius][detector]
    float* rs = Ms + (size_t)dp.time_rows_r * kTimeJ;                // [time][detector]
    float* red = rs + (size_t)dp.time_rows_t * kTimeJ;               // [chunk p][warp][detector][lane]
    float* gs = red + (size_t)nch * kTimeWarps * kTimeJ * kWarp;     // [chunk p][data, y][detector][lane]

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const TimeGroup grp = dp.time_groups[blockIdx.x / kTimeCS];
    const InstDev in = dp.inst[grp.inst];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int jd = w % kTimeJ, sub = w / kTimeJ;   // sums and epilogues: detector, and chunks p = sub (mod kTimeSub)
    const int n_tc = in.n_tp >> 5, n_rc = in.n_rp >> 5;
    // the staged rows hold the group's instance (the same for every CTA of the
    // cluster, so all of them return here together and no cluster barrier waits)
    if (!dbg_ok(dp, 32 * n_rc <= dp.time_rows_r && 32 * n_tc <= dp.time_rows_t, kSiteTimeRows)) return;
    // P in 32 x 32 blocks (after P and P^T): forward [time chunk][radius
    // block], then adjoint [radius chunk][time block]; float4 q of a block
    // holds contraction rows 4q .. 4q + 3 of its 32 outputs in lane order
    const size_t pplane = (size_t)in.n_tp * in.n_rp;
    const float* PBF = dp.P + in.p_off + 2 * pplane;
    const float* PBA = PBF + pplane;

    // this lane's 32 values of P for block it (output 32 c + lane, rows 32 kc ..): 8 16-byte loads,
    // each a warp-wide 512-byte contiguous read
    auto load_block = [&](const TItem& it, float(&pv)[32]) {
        const int nkc = it.phase == 0 ? n_rc : n_tc;   // contraction blocks per output chunk
        const float4* src = reinterpret_cast<const float4*>(
            (it.phase == 0 ? PBF : PBA) + ((size_t)it.c * nkc + it.kc) * 1024) + lane;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 v = __ldg(src + q * 32);
            pv[4 * q] = v.x;
            pv[4 * q + 1] = v.y;
            pv[4 * q + 2] = v.z;
            pv[4 * q + 3] = v.w;
        }
    };
    float acc[kTimeJ];
#pragma unroll
    for (int j = 0; j < kTimeJ; ++j) acc[j] = 0.f;
    auto run_block = [&](const TItem& it, const float(&pv)[32]) {
        const float* ab = (it.phase == 0 ? Ms : rs) + (size_t)(32 * it.kc) * kTimeJ;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
#pragma unroll
            for (int h = 0; h < kTimeJ / 4; ++h) {
                const float4 a = *reinterpret_cast<const float4*>(ab + r * kTimeJ + 4 * h);
                acc[4 * h + 0] = fmaf(pv[r], a.x, acc[4 * h + 0]);
                acc[4 * h + 1] = fmaf(pv[r], a.y, acc[4 * h + 1]);
                acc[4 * h + 2] = fmaf(pv[r], a.z, acc[4 * h + 2]);
                acc[4 * h + 3] = fmaf(pv[r], a.w, acc[4 * h + 3]);
            }
        }
        if (it.last) {   // this warp's partial sums of the chunk
            float* dst = red + (size_t)((it.p * kTimeWarps + w) * kTimeJ) * kWarp + lane;
#pragma unroll
            for (int j = 0; j < kTimeJ; ++j) {
                dst[j * kWarp] = acc[j];
                acc[j] = 0.f;
            }
        }
    };

    TWalk walk(rank, w, n_tc, n_rc, in.n_r);
    float pa[32], pb[32];
    TItem cur, nxt;
    bool have = walk.next(cur);
    if (have) load_block(cur, pa);
    bool in_b = false;   // the current block's values are in pb
    // this warp's blocks of phase ph, the next block's loads in flight during each
    auto run_phase = [&](int ph) {
        while (have && cur.phase == ph) {
            const bool more = walk.next(nxt);
            if (!in_b) {
                if (more) load_block(nxt, pb);
                run_block(cur, pa);
            } else {
                if (more) load_block(nxt, pa);
                run_block(cur, pb);
            }
            in_b = !in_b;
            have = more;
            cur = nxt;
        }
    };

    pdl_wait();   // the partial slots come from the circular-mean kernel; g and y from earlier work

    // the data (and y) of this CTA's time chunks, for the forward epilogue
    for (int p = sub; time_chunk(p, rank) < n_tc; p += kTimeSub) {
        const int x = 32 * time_chunk(p, rank) + lane;
        const bool ok = jd < grp.jn && x < in.n_t;
        const size_t o = ok ? in.g_off + (size_t)(grp.j0 + jd) * in.n_t + x : 0;
        float* d = gs + (size_t)(p * 2 * kTimeJ + jd) * kWarp + lane;
        cp_async4_zfill(d, gdata + o, ok);
        if (DUAL) cp_async4_zfill(d + kTimeJ * kWarp, y + o, ok);
    }
    cp_async_commit();

    // 1. M of this CTA's radius chunks: thread = (detector jd, radius lane of the chunk)
    //    for chunks p = sub (mod kTimeSub), kU chunks at a time with 8 slots of each in flight
    {
        constexpr int kU = 2;
        const bool jok = jd < grp.jn;
        const int jj = grp.j0 + (jok ? jd : 0);
        const size_t plane = (size_t)in.n_det * in.n_r;
        const float* src = dp.mpart + in.mpart_off + (size_t)jj * in.n_r;
        const int32_t* cnt_row = reinterpret_cast<const int32_t*>(dp.slotcnt + in.slotcnt_off) + (size_t)jj * in.nmb;
        for (int p0 = sub; time_chunk(p0, rank) < n_rc; p0 += kU * kTimeSub) {
            int m[kU], cnt[kU], cmax = 0;
            float s[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int c = time_chunk(p0 + u * kTimeSub, rank);
                m[u] = 32 * c + lane;
                cnt[u] = (c < n_rc && jok && m[u] < in.n_r) ? __ldg(cnt_row + m[u] / dp.m_lanes) : 0;
                if (!dbg_ok(dp, cnt[u] <= in.n_slots, kSiteTimeRows)) cnt[u] = 0;
                cmax = max(cmax, cnt[u]);
                s[u] = 0.f;
            }
            for (int sl = 0; sl < cmax; sl += 8) {
                float v[kU][8];
#pragma unroll
                for (int u = 0; u < kU; ++u)
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        v[u][k] = sl + k < cnt[u] ? __ldcg(src + (size_t)(sl + k) * plane + m[u]) : 0.f;
#pragma unroll
                for (int u = 0; u < kU; ++u)
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (sl + k < cnt[u]) s[u] += v[u][k];
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (time_chunk(p0 + u * kTimeSub, rank) < n_rc) Ms[m[u] * kTimeJ + jd] = s[u];
        }
    }
    cluster_arrive();
    cluster_wait();   // every CTA's share of M is in place
    constexpr int kChunkF4 = 32 * kTimeJ / 4;   // float4s of one chunk of rows
    for (int idx = tid; idx < n_rc * kChunkF4; idx += kTimeThreads) {
        const int own = time_owner(idx / kChunkF4);
        if (own != rank)
            reinterpret_cast<float4*>(Ms)[idx] = reinterpret_cast<const float4*>(cluster.map_shared_rank(Ms, own))[idx];
    }
    __syncthreads();

    // 2. forward blocks, then the CTA's time chunks: g = sum / K and the residual
    run_phase(0);
    cp_async_wait_group<0>();   // this thread's data (and y) of its outputs
    __syncthreads();            // every warp's partial sums are in place
    for (int p = sub; time_chunk(p, rank) < n_tc; p += kTimeSub) {   // thread = (detector jd, output lane)
        const int c = time_chunk(p, rank);
        int lo, hi;
        time_blocks(0, c, in.n_r, n_tc, lo, hi);
        const int nw = min(kTimeWarps, hi - lo);   // warps that had blocks of this chunk
        float sum = 0.f;
        for (int ww = 0; ww < nw; ++ww) sum += red[(size_t)((p * kTimeWarps + ww) * kTimeJ + jd) * kWarp + lane];
        const int x = 32 * c + lane;
        float r = 0.f;
        if (jd < grp.jn && x < in.n_t) {
            const float* d = gs + (size_t)(p * 2 * kTimeJ + jd) * kWarp + lane;
            const size_t o = in.g_off + (size_t)(grp.j0 + jd) * in.n_t + x;
            const float g = sum * in.inv_K;
            if (DUAL) {
                r = fmaf(sigma, g - d[0], d[kTimeJ * kWarp]) * inv1ps;
                y[o] = r;
            } else {
                r = g - d[0];
                if (y) y[o] = r;
            }
        }
        rs[x * kTimeJ + jd] = r;   // zero for absent detectors and padded times
    }

    // 3. exchange of the residual chunks
    cluster_arrive();
    cluster_wait();   // every CTA's residual chunks are in place
    for (int idx = tid; idx < n_tc * kChunkF4; idx += kTimeThreads) {
        const int own = time_owner(idx / kChunkF4);
        if (own != rank)
            reinterpret_cast<float4*>(rs)[idx] = reinterpret_cast<const float4*>(cluster.map_shared_rank(rs, own))[idx];
    }
    cluster_arrive();   // this CTA has read the others' shared memory (waited for at exit)
    __syncthreads();    // the copies are visible to the CTA; the forward partial sums are consumed

    // 4. adjoint blocks, then the CTA's radius chunks of Mbar
    run_phase(1);
    __syncthreads();
    for (int p = sub; time_chunk(p, rank) < n_rc; p += kTimeSub) {
        const int c = time_chunk(p, rank);
        int lo, hi;
        time_blocks(1, c, in.n_r, n_tc, lo, hi);
        const int nw = min(kTimeWarps, hi - lo);
        float sum = 0.f;
        for (int ww = 0; ww < nw; ++ww) sum += red[(size_t)((p * kTimeWarps + ww) * kTimeJ + jd) * kWarp + lane];
        const int x = 32 * c + lane;
        if (jd < grp.jn && x < in.n_r) dp.mbar[in.mbar_off + (size_t)(grp.j0 + jd) * in.m_pitch + x] = sum;
    }
    cluster_wait();   // no CTA leaves while another may still read its shared memory
}

namespace {
template <bool DUAL>
cudaError_t launch_time_pair_t(const DevPlan& dp, const float* g, float* y, float sigma, float inv1ps,
                               cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(k_time_pair<DUAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         dp.time_smem_bytes);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_time_pair<DUAL>, dim3((unsigned)(dp.n_time_groups * kTimeCS)), dim3(kTimeThreads),
                      (size_t)dp.time_smem_bytes, st, kTimeCS, dp, g, y, sigma, inv1ps);
}
} // namespace

cudaError_t launch_time_pair(const DevPlan& dp, const float* g, float* y, bool dual, float sigma, float inv1ps,
                             cudaStream_t st)
{
    if (dp.n_time_groups == 0) return cudaSuccess;
    if (dp.time_chunks <= 0) return cudaErrorInvalidValue;
    return dual ? launch_time_pair_t<true>(dp, g, y, sigma, inv1ps, st)
                : launch_time_pair_t<false>(dp, g, y, sigma, inv1ps, st);
}

int time_pair_clusters(int smem_bytes)
{
    const void* fn = reinterpret_cast<const void*>(k_time_pair<false>);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(kTimeCS);
    cfg.blockDim = dim3(kTimeThreads);
    cfg.dynamicSmemBytes = (size_t)smem_bytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kTimeCS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

} // namespace patgpu
