// gather.cu — adjoint circular means f = C^T Mbar as a gather over pixels.
//
// C^T scatters every sample's bilinear weights; here every output is instead
// summed by the one warp or thread that owns it, in a fixed order (no atomics,
// deterministic).  Work happens per cell [cx, cx+1) x [cy, cy+1): a sample
// that lands in the cell adds w (1-a)(1-b), w a(1-b), w (1-a)b, w ab to the
// cell's four corner sums Z (w = Mbar[j][m]); pixel (px, py) then sums
// Z00(px,py) + Z10(px-1,py) + Z01(px,py-1) + Z11(px-1,py-1) (times 1/K).
//
// Finding a cell's samples.  For each detector, a cell can only receive
// samples from rays q whose direction passes within R = sqrt(2)/2 (+ margin)
// of its centre; each such ray is intersected with the cell (slab test,
// widened by a margin that covers FP32 rounding) to get the run of radii m
// that can land in it, and each candidate's cell is re-evaluated with exactly
// the forward's split-form expression.  Hits come out in the order (j, q, m).
//
// Three ways to run this:
//   code lists (when 4 B per sample fits the list budget and a (q, j, m)
//     code fits 32 bits): at plan creation the enumeration runs twice
//     (count, then fill) to store every cell's hits as packed codes, the 32
//     cells of an 8 x 4 patch interleaved vector by vector so that a warp
//     streams them with full 512-byte loads; each call recomputes a and b
//     from the codes with the forward's expressions (k_adj_list).  The
//     default form is run pairs: most hits of a cell come in runs of two
//     consecutive radii on one ray (a cell is about two radius steps wide),
//     and one code then stands for both, so the pair shares its detector and
//     ray loads and the code stream shrinks by about 40 %.
//   fraction lists (12 B per sample): the hits as (Mbar index, a, b), a and b
//     the exact FP32 values the forward computes (one table load per sample,
//     no coordinate arithmetic, but a 3x larger stream).
//   compute mode: the enumeration runs on every call (k_adj_cells), one warp
//     per 8 x 4 patch of cells and detector group, partial Z per group.
#include <algorithm>

#include "device_common.cuh"
#include "kernels.h"

namespace patgpu {

namespace {
constexpr float kRcell = 0.70710678f + 0.004f;  // half cell diagonal + rounding margin (pixels)
constexpr float kSlabEps = 0.01f;                // slab widening (pixels)
constexpr float kAngMargin = 1.0e-5f;            // > 5x the atan2_approx error (radians)

// Calls hit(j, m, q, a, b) for every sample (j in j0, j0 + dj, ...) that
// lands in centred cell (cxf, cyf), (a, b) its fractions in the cell, in
// (j, q, m) order; q in [0, K).
template <typename Hit>
__device__ __forceinline__ void enumerate_cell(const DevPlan& dp, const InstDev& in, float cxf, float cyf, int j0,
                                               int dj, Hit&& hit)
{
    const float ccx = cxf + 0.5f, ccy = cyf + 0.5f;
    const float4* det = dp.det + in.det_off;
    const float4* rays = dp.rays + in.ray_off;
    const float2* rtrig = dp.rtrig + in.ray_off;
    const int K = in.K;
    for (int j = j0; j < in.n_det; j += dj) {
        const float4 d = __ldg(det + j);
        const float U = d.x + d.z, V = d.y + d.w;   // approximate U, V for the candidate search
        const float du = ccx - U, dv = ccy - V;
        const float rc = sqrtf(fmaf(du, du, dv * dv));
        const int mlo = max(0, (int)ceilf((rc - kRcell) * in.inv_delta));
        const int mhi = min(in.n_r - 1, (int)floorf((rc + kRcell) * in.inv_delta));
        if (mlo > mhi) continue;
        int qlo = 0, qn = K;
        if (rc > 1.25f * kRcell) {
            const float phic = atan2_approx(dv, du);
            const float alpha = asin_upper(__fdividef(kRcell, rc)) + kAngMargin;
            qlo = (int)ceilf((phic - alpha) * in.inv_dphi);
            qn = min((int)floorf((phic + alpha) * in.inv_dphi) - qlo + 1, K);
            if (qlo < 0) qlo += K;
        }
        const float ax0 = (cxf - kSlabEps) - U, ax1 = (cxf + 1.f + kSlabEps) - U;
        const float ay0 = (cyf - kSlabEps) - V, ay1 = (cyf + 1.f + kSlabEps) - V;
        // the cell relative to the detector's integer part (exact: small integers)
        const float cxr = cxf - d.x, cyr = cyf - d.y;
        for (int i = 0; i < qn; ++i) {
            const int q = qlo + i;
            const float2 ri = __ldg(rtrig + q);
            const float tx0 = ax0 * ri.x, tx1 = ax1 * ri.x;
            const float ty0 = ay0 * ri.y, ty1 = ay1 * ri.y;
            const float lo = fmaxf(fminf(tx0, tx1), fminf(ty0, ty1));
            const float hi = fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1));
            const int m0 = max(mlo, (int)ceilf(lo));
            const int m1 = min(mhi, (int)floorf(hi));
            if (m0 > m1) continue;
            const float4 r = __ldg(rays + q);
            for (int m = m0; m <= m1; ++m) {
                const float mf = (float)m;
                if (cell_rel(mf, r.x, d.z) == cxr && cell_rel(mf, r.y, d.w) == cyr)
                    hit(j, m, q >= K ? q - K : q, cell_frac(mf, r.x, r.z, d.z, cxr),
                        cell_frac(mf, r.y, r.w, d.w, cyr));
            }
        }
    }
}

__device__ __forceinline__ void add_corners(float4& z, float a, float b, float w)
{
    const float wb = w * b, w1 = w - wb; // w b, w (1 - b)
    z.y = fmaf(a, w1, z.y);              // Z10 += w a (1 - b)
    z.x = fmaf(-a, w1, z.x + w1);        // Z00 += w (1 - a)(1 - b)
    z.w = fmaf(a, wb, z.w);              // Z11 += w a b
    z.z = fmaf(-a, wb, z.z + wb);        // Z01 += w (1 - a) b
}

__device__ __forceinline__ int take_item(int32_t* ctr, int lane)
{
    int item = 0;
    if (lane == 0) item = atomicAdd(ctr, 1);
    return __shfl_sync(0xffffffffu, item, 0);
}

// the last warp to run out of items re-arms the queue for the next launch
__device__ __forceinline__ void release_queue(int32_t* ctr, int lane)
{
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    if (lane == 0 && atomicAdd(ctr + 1, 1) == nwarps - 1) {
        ctr[0] = 0;
        ctr[1] = 0;
    }
}
} // namespace

// ---------------------------------------------------------------------------
// Compute mode: one warp per (8 x 4 cell patch, detector group); dynamic
// queue over items sorted by estimated cost.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 5) k_adj_cells(DevPlan dp)
{
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int G = dp.adj_groups;
    for (;;) {
        const int item = take_item(dp.work_counters, lane);
        if (item >= dp.n_cell_items) break;
        const CellItem it = dp.cell_items[item];
        const InstDev in = dp.inst[it.inst];
        const int n = in.n;
        const int cx = it.x0 + (lane & (kPatchW - 1)), cy = it.y0 + lane / kPatchW;
        if (cx > n - 1 || cy > n - 1) continue;
        const float cxf = (float)(cx - in.c0), cyf = (float)(cy - in.c0);
        const float* mb = dp.mbar + in.mbar_off;
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        enumerate_cell(dp, in, cxf, cyf, it.group, G, [&](int j, int m, int, float a, float b) {
            add_corners(z, a, b, __ldg(mb + (size_t)j * in.m_pitch + m));
        });
        dp.zbuf[in.z_off + (size_t)it.group * (n + 1) * (n + 1) + (size_t)(cy + 1) * (n + 1) + (cx + 1)] = z;
    }
    release_queue(dp.work_counters, lane);
}

// ---------------------------------------------------------------------------
// List building (plan creation), thread = cell, hits in enumeration order
// (j, q, m) over all detectors of instance `inst_idx` (layouts in
// pat_internal.h).
//
// Fraction lists: k_adj_build<0> counts every cell's samples, then
// k_adj_build<2> stores sample k of a cell (Mbar index j * m_pitch + m and
// the fractions a, b) in vector k / 4 of the part holding that vector,
// component k % 4, and null entries fill the cell's last vector.
//
// Code lists: k_adj_seg<PAIRS, false> takes, for every (patch, detector
// block), the longest entry count of the patch's cells (atomicMax into
// segmax); the host turns those into segment starts; k_adj_seg<PAIRS, true>
// then writes entry i of block b of a cell at position seg[b] + i of the
// patch's sequence, over a buffer that holds null codes everywhere else.
// PAIRS: two hits of one (j, q) at radii m, m + 1 make one entry, coded at m
// with bit 31 set.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) k_adj_build(DevPlan dp, int inst_idx, int32_t* __restrict__ counts,
                                                   const int64_t* __restrict__ pbase, uint32_t* __restrict__ out)
{
    const InstDev in = dp.inst[inst_idx];
    const int n = in.n, w = n + 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= w * w) return;
    const int cxa = idx % w, cya = idx / w;   // cell index + 1
    const float cxf = (float)(cxa - 1 - in.c0), cyf = (float)(cya - 1 - in.c0);
    const int mb = in.code_mbits;
    const int G = dp.adj_groups;
    int count = 0, nv = 0, lane = 0;
    const int64_t* pb = nullptr;
    if (MODE) {
        count = counts[idx];
        nv = (count + 3) >> 2;
        pb = pbase + ((int64_t)(cya / kPatchH) * in.patches_x + cxa / kPatchW) * G;
        lane = (cya % kPatchH) * kPatchW + cxa % kPatchW;
    }
    // part g holds vectors [g nv / G, (g + 1) nv / G): vector v is in part
    // ceil((v + 1) G / nv) - 1
    auto put = [&](int k, uint32_t widx, float a, float b) {
        const int v = k >> 2;
        const int g = (int)(((int64_t)(v + 1) * G + nv - 1) / nv) - 1;
        const int v0 = (int)((int64_t)g * nv / G);
        const int64_t slot = pb[g] + (int64_t)(v - v0) * 3 * kWarp + lane;
        const int c = k & 3;
        out[slot * 4 + c] = widx;
        out[(slot + kWarp) * 4 + c] = __float_as_uint(a);
        out[(slot + 2 * kWarp) * 4 + c] = __float_as_uint(b);
    };
    int k = 0;
    enumerate_cell(dp, in, cxf, cyf, 0, 1, [&](int j, int m, int, float a, float b) {
        // (the fill sees exactly the counted hits; never write past them)
        if (MODE && k < count) put(k, ((uint32_t)j << mb) | (uint32_t)m, a, b);
        ++k;
    });
    if (!MODE) {
        counts[idx] = k;
        return;
    }
    const uint32_t null_widx = (uint32_t)in.m_pitch - 1u;   // row 0, a column that is always zero
    for (int kk = count; kk < 4 * nv; ++kk) put(kk, null_widx, 0.f, 0.f);
}

// seg: per patch, the segment start of each detector block, then the
// patch's length in vectors (nblk + 1 entries per patch).
template <bool PAIRS, bool FILL>
__global__ void __launch_bounds__(256) k_adj_seg(DevPlan dp, int inst_idx, int jblock, int nblk,
                                                 int32_t* __restrict__ seg, const int64_t* __restrict__ pbase,
                                                 uint32_t* __restrict__ out)
{
    const InstDev in = dp.inst[inst_idx];
    const int n = in.n, w = n + 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= w * w) return;
    const int cxa = idx % w, cya = idx / w;   // cell index + 1
    const float cxf = (float)(cxa - 1 - in.c0), cyf = (float)(cya - 1 - in.c0);
    const int mb = in.code_mbits, jmb = in.code_jbits + in.code_mbits;
    const int G = dp.adj_groups;
    const int64_t patch = (int64_t)(cya / kPatchH) * in.patches_x + cxa / kPatchW;
    int32_t* sp = seg + patch * (nblk + 1);
    const int lane = (cya % kPatchH) * kPatchW + cxa % kPatchW;
    const int nv = FILL ? sp[nblk] : 0;
    const int64_t* pb = FILL ? pbase + patch * G : nullptr;
    int cur_b = -1, i = 0;   // current detector block, entries of this cell in it so far
    auto emit = [&](int j, int m, int q, uint32_t flag) {
        const int b = j / jblock;
        if (b != cur_b) {
            if (!FILL && cur_b >= 0) atomicMax(sp + cur_b, i);
            cur_b = b;
            i = 0;
        }
        if (FILL) {
            const int pos = sp[b] + i;
            const int v = pos >> 2;
            if (v < nv) {   // (always: the fill sees exactly the counted entries)
                const int g = (int)(((int64_t)(v + 1) * G + nv - 1) / nv) - 1;
                const int v0 = (int)((int64_t)g * nv / G);
                const int64_t slot = pb[g] + (int64_t)(v - v0) * kWarp + lane;
                out[slot * 4 + (pos & 3)] =
                    flag | ((uint32_t)q << jmb) | ((uint32_t)j << mb) | (uint32_t)m;
            }
        }
        ++i;
    };
    int pj = -1, pq = 0, pm = 0;   // pending hit that may start a run pair
    enumerate_cell(dp, in, cxf, cyf, 0, 1, [&](int j, int m, int q, float, float) {
        if constexpr (PAIRS) {
            if (pj == j && pq == q && pm + 1 == m) {
                emit(pj, pm, pq, 0x80000000u);
                pj = -1;
            } else {
                if (pj >= 0) emit(pj, pm, pq, 0u);
                pj = j;
                pq = q;
                pm = m;
            }
        } else {
            emit(j, m, q, 0u);
        }
    });
    if (PAIRS && pj >= 0) emit(pj, pm, pq, 0u);
    if (!FILL && cur_b >= 0) atomicMax(sp + cur_b, i);
}

__global__ void k_fill_u32(uint32_t* __restrict__ p, int64_t n, uint32_t v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ---------------------------------------------------------------------------
// List mode: lane = cell of an 8 x 4 patch, warp = (patch, part) item.  Each
// lane streams its cell's part as 16-byte vectors (a warp's load is 512
// contiguous bytes: the 32 cells' vectors are interleaved), four vectors in
// flight, and accumulates the moments sum w, sum w a, sum w b, sum w a b of
// its samples (w = Mbar[j][m]; a and b recomputed from the code exactly as
// the forward computes them, or stored); null entries have w = 0.  The
// cell's four corner sums
//     Z00 = sum w (1-a)(1-b), Z10 = sum w a (1-b), Z01 = sum w (1-a) b, Z11 = sum w a b
// go to plane `part` of Z, each written once (no atomics, deterministic).
// LM 0: code lists; LM 1: fraction lists; LM 2: run-pair code lists (a code
// with bit 31 set also stands for radius m + 1 on the same ray: one
// detector and one ray load serve both samples).  The code lists are
// aligned by detector blocks, so all lanes of an item have the same number
// of vectors and, at any step, read the tables of a few detectors only.
// Schedule: each warp first runs the items the plan assigned to it (LPT over
// item lengths), then takes items from a shared queue of the smallest ones,
// largest first (one atomic ticket per item, taken one item ahead; the last
// warp to finish re-arms the counter).  Which warp runs an item does not
// change any result: each (cell, part) is summed by one lane in list order.
// ---------------------------------------------------------------------------
namespace {
struct Moments {
    float s0 = 0.f, sa = 0.f, sb = 0.f, sab = 0.f;
    __device__ __forceinline__ void add(float w, float a, float b)
    {
        const float wa = w * a;
        s0 += w;
        sa += wa;
        sb = fmaf(w, b, sb);
        sab = fmaf(wa, b, sab);
    }
};
} // namespace

// prefetch of one 16-byte vector's line into L1
__device__ __forceinline__ void prefetch_l1(const void* p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

template <int LM>
__global__ void __launch_bounds__(256, 3) k_adj_list(DevPlan dp)
{
    pdl_wait();   // Mbar comes from the previous kernel
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int ib = dp.warp_items[warp], ie = dp.warp_items[warp + 1];
    constexpr int S = LM == 1 ? 3 : 1;   // 16-byte slots per vector
    const uint4* codes = reinterpret_cast<const uint4*>(dp.codes);
    const int G = dp.adj_groups;
    // one (patch, part) item; `first`: the warp's first item (the debug probe's entry)
    auto run_item = [&](const ListItem& it, bool first) {
        if (!dbg_ok(dp, it.inst >= 0 && it.inst < dp.n_inst && it.base >= 0 &&
                            (LM == 1 || it.base + (int64_t)it.nk * kWarp <= dp.n_code_vecs),
                    kSiteListItem))
            return;
        const InstDev in = dp.inst[it.inst];
        const int n = in.n, w = n + 1;
        const int cx = it.x0 + (lane & (kPatchW - 1)), cy = it.y0 + lane / kPatchW;
        if (cx > n - 1 || cy > n - 1) return;
        const int cell = (cy + 1) * w + (cx + 1);
        const uint4* L = codes + it.base + lane;
#ifdef PAT_DEBUG
        // test hook: lane 0 of warp 0 gives its first entry a detector index past the instance's
        // detectors (the tables it would address still lie inside the plan's allocations)
        bool plant = dp.bounds_probe != 0 && warp == 0 && lane == 0 && first;
        const uint32_t mb_size = (uint32_t)in.n_det * (uint32_t)in.m_pitch;
#endif
        const float* mb = dp.mbar + in.mbar_off;
        Moments acc;
        if constexpr (LM == 1) {
            const int nv = (dp.cell_cnt[in.list_off + cell] + 3) >> 2;
            const int nk = (int)((int64_t)(it.group + 1) * nv / G) - (int)((int64_t)it.group * nv / G);
            if (!dbg_ok(dp, it.base + (int64_t)nk * 3 * kWarp <= dp.n_code_vecs, kSiteListItem)) return;
#ifdef PAT_DEBUG
            auto wload = [&](uint32_t i) {
                if (plant) {
                    i += mb_size;
                    plant = false;
                }
                return dbg_ok(dp, i < mb_size, kSiteListEntry) ? __ldg(mb + i) : 0.f;
            };
#else
            auto wload = [&](uint32_t i) { return __ldg(mb + i); };
#endif
            // two vectors (8 entries) in flight per lane
            for (int kb = 0; kb < nk; kb += 2) {
                uint4 ci[2], ca[2], cb[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (kb + u < nk) {
                        const uint4* p = L + (size_t)(kb + u) * 3 * kWarp;
                        ci[u] = __ldcs(p);
                        ca[u] = __ldcs(p + kWarp);
                        cb[u] = __ldcs(p + 2 * kWarp);
                    } else {
                        ci[u] = ca[u] = cb[u] = make_uint4(0u, 0u, 0u, 0u);
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (kb + u >= nk) break;
                    acc.add(wload(ci[u].x), __uint_as_float(ca[u].x), __uint_as_float(cb[u].x));
                    acc.add(wload(ci[u].y), __uint_as_float(ca[u].y), __uint_as_float(cb[u].y));
                    acc.add(wload(ci[u].z), __uint_as_float(ca[u].z), __uint_as_float(cb[u].z));
                    acc.add(wload(ci[u].w), __uint_as_float(ca[u].w), __uint_as_float(cb[u].w));
                }
            }
        } else {
            // aligned lists: every lane of the item has the block's length
            const int nk = it.nk;
            const unsigned long long cxy = f2_pack((float)(cx - in.c0), (float)(cy - in.c0));
            const float4* det = dp.det + in.det_off;
            const float4* rays = dp.rays + in.ray_off;
            const int mbits = in.code_mbits, qshift = in.code_jbits + in.code_mbits;
            const uint32_t wmask = (1u << qshift) - 1u, mmask = (1u << mbits) - 1u;
            auto entry = [&](uint32_t c) {
#ifndef PAT_DEBUG
                const uint32_t widx = c & wmask;
#endif
                // (bit 31 is the pair flag in run-pair codes, the top bit of q in one-sample codes)
#ifdef PAT_DEBUG
                uint32_t widx = c & wmask;
                const int q = (int)((LM == 2 ? c & 0x7fffffffu : c) >> qshift);
                int j = (int)(widx >> mbits);
                if (plant) {
                    j += in.n_det;
                    widx += mb_size;
                    plant = false;
                }
                const uint32_t wlast = widx + ((LM == 2 && (int32_t)c < 0) ? 1u : 0u);   // the pair's second weight
                if (!dbg_ok(dp, j < in.n_det && q < 2 * in.K && wlast < mb_size, kSiteListEntry)) return;
#else
                const int q = (int)((LM == 2 ? c & 0x7fffffffu : c) >> qshift), j = (int)(widx >> mbits);
#endif
                const float mf = __uint_as_float((c & mmask) | kMagicBits) - kMagic;   // m < 2^22
                const float wv = __ldg(mb + widx);
                const float4 d = __ldg(det + j);
                const float4 r = __ldg(rays + q);
                // the sample lies in this cell: its relative cell is (cxf, cyf) - floor(U, V), so
                // -cell = floor(U, V) - (cxf, cyf) (exact), and (a, b) is cell_frac's sequence in
                // f32x2 pairs: fma(m, hi, -cell) + fma(m, lo, f0)
                const unsigned long long m2 = f2_pack(mf, mf);
                const unsigned long long hi = f2_pack(r.x, r.y), lo = f2_pack(r.z, r.w), f0 = f2_pack(d.z, d.w);
                const unsigned long long ncell = f2_sub(f2_pack(d.x, d.y), cxy);
                const float2 ab = f2_unpack(f2_add(f2_fma(m2, hi, ncell), f2_fma(m2, lo, f0)));
                acc.add(wv, ab.x, ab.y);
                if constexpr (LM == 2) {
                    // the pair's second sample, radius m + 1 (exact in FP32) on the same ray
                    const float w2 = (int32_t)c < 0 ? __ldg(mb + widx + 1) : 0.f;
                    const float mf2 = mf + 1.f;
                    const unsigned long long m2b = f2_pack(mf2, mf2);
                    const float2 ab2 = f2_unpack(f2_add(f2_fma(m2b, hi, ncell), f2_fma(m2b, lo, f0)));
                    acc.add(w2, ab2.x, ab2.y);
                }
            };
            // four vectors in flight per lane (the next four prefetched), then their 16 entries
            for (int kb = 0; kb < nk; kb += 4) {
                uint4 c[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    c[u] = (kb + u < nk) ? __ldcs(L + (size_t)(kb + u) * kWarp) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int u = 4; u < 8; ++u)
                    if (kb + u < nk) prefetch_l1(L + (size_t)(kb + u) * kWarp);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (kb + u >= nk) break;
                    entry(c[u].x);
                    entry(c[u].y);
                    entry(c[u].z);
                    entry(c[u].w);
                }
            }
        }
        const float z10 = acc.sa - acc.sab, z01 = acc.sb - acc.sab;
        dp.zbuf[in.z_off + (size_t)it.group * w * w + cell] = make_float4(acc.s0 - acc.sa - z01, z10, z01, acc.sab);
    };
    // this warp's static items, then the shared tail of small items (largest
    // first), whose next ticket is in flight while the current item runs
    int ii = ib, tk = 0;
    bool in_tail = false;
    for (;;) {
        int idx;
        if (ii < ie) {
            idx = ii++;
            if (ii < ie) {
                // the next item's first vectors, on their way while this item runs
                const ListItem nx = dp.list_items[ii];
                const uint4* Ln = codes + nx.base + lane;
                const int np = min(nx.nk, 4) * S;
                for (int u = 0; u < np; ++u) prefetch_l1(Ln + (size_t)u * kWarp);
            }
        } else {
            if (dp.n_tail_items == 0) break;
            if (!in_tail && lane == 0) tk = atomicAdd(dp.work_counters + kQueueStride, 1);
            in_tail = true;
            const int cur = __shfl_sync(0xffffffffu, tk, 0);
            if (cur >= dp.n_tail_items) break;
            if (lane == 0) tk = atomicAdd(dp.work_counters + kQueueStride, 1);
            idx = dp.list_tail0 + cur;
        }
        run_item(dp.list_items[idx], idx == ib && !in_tail);
    }
    if (dp.n_tail_items > 0) release_queue(dp.work_counters + kQueueStride, lane);
}

template <typename T>
__global__ void __launch_bounds__(256) k_adj_combine(DevPlan dp, T* __restrict__ fout)
{
    const ImgTile t = dp.img_tiles[blockIdx.x];
    pdl_wait();
    const InstDev in = dp.inst[t.inst];
    const int n = in.n;
    const int px = t.x0 + (threadIdx.x & 31), py = t.y0 + (threadIdx.x >> 5);
    if (px >= n || py >= n) return;
    const int w = n + 1;
    const float4* z = dp.zbuf + in.z_off;
    const int groups = dp.adj_groups;
    // cell (cx, cy) is stored at (cy + 1) * w + (cx + 1)
    const float s = corner_sum(z, (size_t)w * w, groups, (size_t)(py + 1) * w + px + 1, (size_t)(py + 1) * w + px,
                               (size_t)py * w + px + 1, (size_t)py * w + px);
    const float val = s * in.inv_K;
    if constexpr (sizeof(T) == 4) fout[in.f_off + (size_t)py * n + px] = val;
    else fout[in.f_off + (size_t)py * n + px] = __float2bfloat16(val);
}

int adj_cells_blocks_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adj_cells, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

namespace {
const void* adj_list_fn(int lm)
{
    if (lm == 1) return reinterpret_cast<const void*>(k_adj_list<1>);
    if (lm == 2) return reinterpret_cast<const void*>(k_adj_list<2>);
    return reinterpret_cast<const void*>(k_adj_list<0>);
}
} // namespace

int adj_list_blocks_per_sm(int lm)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, adj_list_fn(lm), 256, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_adj_frac_build(const DevPlan& dp, int inst_idx, int n, int32_t* counts, const int64_t* pbase,
                                  uint32_t* out, cudaStream_t st)
{
    const int cells = (n + 1) * (n + 1);
    const int blocks = (cells + 255) / 256;
    if (!out) k_adj_build<0><<<blocks, 256, 0, st>>>(dp, inst_idx, counts, pbase, out);
    else k_adj_build<2><<<blocks, 256, 0, st>>>(dp, inst_idx, counts, pbase, out);
    return cudaGetLastError();
}

cudaError_t launch_adj_seg(const DevPlan& dp, int inst_idx, int n, bool pairs, int jblock, int nblk, int32_t* seg,
                           const int64_t* pbase, uint32_t* out, cudaStream_t st)
{
    const int cells = (n + 1) * (n + 1);
    const int blocks = (cells + 255) / 256;
    if (!out) {
        if (pairs) k_adj_seg<true, false><<<blocks, 256, 0, st>>>(dp, inst_idx, jblock, nblk, seg, pbase, out);
        else k_adj_seg<false, false><<<blocks, 256, 0, st>>>(dp, inst_idx, jblock, nblk, seg, pbase, out);
    } else {
        if (pairs) k_adj_seg<true, true><<<blocks, 256, 0, st>>>(dp, inst_idx, jblock, nblk, seg, pbase, out);
        else k_adj_seg<false, true><<<blocks, 256, 0, st>>>(dp, inst_idx, jblock, nblk, seg, pbase, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_fill_u32(uint32_t* p, int64_t n, uint32_t v, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    k_fill_u32<<<(unsigned)blocks, 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_cells(const DevPlan& dp, cudaStream_t st)
{
    if (dp.adj_mode == 1 || dp.adj_mode == 3 || dp.adj_mode == 4) {
        if (dp.n_list_items == 0) return cudaSuccess;   // (cell_blocks x 8 warps run the items)
        if (dp.adj_mode == 3) return launch_pdl(k_adj_list<1>, dim3(dp.cell_blocks), dim3(256), 0, st, 1, dp);
        if (dp.adj_mode == 4) return launch_pdl(k_adj_list<2>, dim3(dp.cell_blocks), dim3(256), 0, st, 1, dp);
        return launch_pdl(k_adj_list<0>, dim3(dp.cell_blocks), dim3(256), 0, st, 1, dp);
    }
    if (dp.n_cell_items == 0) return cudaSuccess;
    return launch_pdl(k_adj_cells, dim3(dp.cell_blocks), dim3(256), 0, st, 1, dp);
}

cudaError_t launch_adjoint_gather(const DevPlan& dp, void* f, cudaStream_t st)
{
    cudaError_t e = launch_adjoint_cells(dp, st);
    if (e != cudaSuccess) return e;
    if (dp.bf16)
        return launch_pdl(k_adj_combine<__nv_bfloat16>, dim3(dp.n_img_tiles), dim3(256), 0, st, 1, dp,
                          static_cast<__nv_bfloat16*>(f));
    return launch_pdl(k_adj_combine<float>, dim3(dp.n_img_tiles), dim3(256), 0, st, 1, dp, static_cast<float*>(f));
}

} // namespace patgpu
