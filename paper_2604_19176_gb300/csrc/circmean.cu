// circmean.cu — forward circular means M = C f (the first stage of A).
//
// M[j][m] = sum_q f~(y_j + r_m (cos phi_q, sin phi_q)) (the 1/K of the
// trapezoid rule is applied by the Abel stage), f~ the bilinear interpolant
// of f with zero outside the grid: the circular mean of the 2D Poisson
// formula for the wave problem Eq. (1)-(2), discretised as in include/pat.h.
//
// Tiles.  Every image is partitioned into tiles of pixels.  A bilinear sample
// is linear in the four pixels of its cell, so it is the sum over tiles of the
// sample taken from a copy of the image in which only that tile's pixels are
// kept (the rest zero).  A CTA working on a tile stages, for every cell
// [c, c+1] x [r, r+1] that touches the tile, the coefficients of that partial
// interpolant,
//     f~(c + a, r + b) = c00 + a cx + b (cy + a cxy),
//     c00 = f00, cx = f10 - f00, cy = f01 - f00, cxy = f11 - f10 - f01 + f00,
// as one float4 (pixels outside the tile read as zero), so a sample costs one
// 16-byte shared-memory load and three FMAs.  A sample's cell is clamped to
// the staged block, whose outer ring of cells is all zero, so samples that
// miss the tile add exactly zero and no per-sample test is needed.
//
// Work.  A unit is (detector j, ML consecutive radii, a range of angles) of
// one tile; lane l handles radius m0 + l % ML and angles q0 + l / ML +
// i * (32 / ML), walking along rays so that its cell reads are spatially
// coherent.  CTA c works on tile tasks cta_seg[c] .. cta_seg[c+1]-1; for
// each it stages the tile's cells (computed from f through L2) and the
// instance's K ray directions (one TMA bulk copy on an mbarrier with a
// bounded wait), and each of its warps processes the list of units the plan
// assigned to it (balanced by their sample counts at plan time: a sample costs
// the same everywhere, so no run-time queue is needed).  Each unit writes its
// own partial-sum slot; k_msum then adds every (detector, radius block)'s
// slots in slot order, so the result does not depend on scheduling and no
// atomics or fences are needed.
//
// Sample position.  Split form (pat_internal.h): the cell index along u is
// floor(fma(m, hi, Uf)) relative to the detector's integer part and the
// fraction a = fma(m, hi, -cell) + fma(m, lo, Uf), bit-identical to the
// adjoint's cell_rel / cell_frac.  The floor is taken by floor_biased, whose
// result's bit pattern is the biased integer cell: it is clamped and turned
// into a shared-memory byte offset with integer arithmetic only.
#include "device_common.cuh"
#include "kernels.h"

namespace patgpu {

namespace {

// Stages the coefficient cells of tile task sg (see the file comment) from
// image fi (N x N, row-major) into cells (pitch sg.pitch).  A thread takes a
// column of kStageRows cells: it issues the kStageRows + 1 rows' loads of its
// two pixel columns at once (one round trip through L2), then forms the cells.
constexpr int kStageRows = 8;
template <typename T>
__device__ __forceinline__ void stage_cells(float4* __restrict__ cells, const T* __restrict__ fi, int n,
                                            const Segment& sg)
{
    const int SW = sg.x1 - sg.x0 + 3, SH = sg.y1 - sg.y0 + 3;
    const int segs = SW * ((SH + kStageRows - 1) / kStageRows);
    for (int idx = threadIdx.x; idx < segs; idx += blockDim.x) {
        const int sgi = idx / SW, cc = idx - sgi * SW;
        const int rb = sgi * kStageRows;
        const int px = sg.x0 - 2 + cc;   // the cell's left pixel column
        const bool okx0 = px >= sg.x0 && px < sg.x1, okx1 = px + 1 >= sg.x0 && px + 1 < sg.x1;
        float v0[kStageRows + 1], v1[kStageRows + 1];
#pragma unroll
        for (int i = 0; i <= kStageRows; ++i) {
            const int py = sg.y0 - 2 + rb + i;   // pixel row i of this column of cells
            const bool oky = py >= sg.y0 && py < sg.y1;
            const T* p = fi + (size_t)(oky ? py : sg.y0) * n;
            v0[i] = (oky && okx0) ? ld_img(p + px) : 0.f;
            v1[i] = (oky && okx1) ? ld_img(p + px + 1) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < kStageRows; ++i) {
            if (rb + i >= SH) break;
            const float cx = v1[i] - v0[i];
            cells[(rb + i) * sg.pitch + cc] = make_float4(v0[i], cx, v0[i + 1] - v0[i], (v1[i + 1] - v0[i + 1]) - cx);
        }
    }
}

// Per-unit constants of the sample evaluation: clamp bounds of the biased
// cell bits (floor_biased results) and the offset that turns the clamped
// bits into a byte offset of the staged cell.
struct UnitFrame {
    uint32_t ulo, uhi, vlo, vhi, row_bytes, koff;
    uint32_t lim;   // debug builds: largest valid byte offset of a staged cell
};

__device__ __forceinline__ UnitFrame unit_frame(const Segment& sg, const InstDev& in, float4 d)
{
    UnitFrame u;
    const int Ui = __float2int_rz(d.x), Vi = __float2int_rz(d.y);
    // staged column index = floor + Ui + c0 - (x0 - 2); bits = kMagicBits + floor
    u.ulo = kMagicBits + (uint32_t)(sg.x0 - 2 - Ui - in.c0);
    u.vlo = kMagicBits + (uint32_t)(sg.y0 - 2 - Vi - in.c0);
    u.uhi = u.ulo + (uint32_t)(sg.x1 - sg.x0 + 2);
    u.vhi = u.vlo + (uint32_t)(sg.y1 - sg.y0 + 2);
    u.row_bytes = (uint32_t)sg.pitch * 16u;
    u.koff = 0u - (u.vlo * u.row_bytes + u.ulo * 16u);   // modulo 2^32
    return u;
}

// One sample (radius mf, ray r = (hi_u, hi_v, lo_u, lo_v)) of the staged tile.
// The u and v halves of the split form run as f32x2 pairs (m2 = (mf, mf),
// f0 = (Uf, Vf)), in the order of cell_rel and cell_frac: t = floor_biased of
// fma(m, hi, f0); -cell = kMagic - t (exact); a = fma(m, hi, -cell) +
// fma(m, lo, f0).
__device__ __forceinline__ float sample(const unsigned char* __restrict__ smem, const UnitFrame& u,
                                        unsigned long long m2, float4 r, unsigned long long f0
#ifdef PAT_DEBUG
                                        , const DevPlan* dbg_plan
#endif
)
{
    const unsigned long long hi = f2_pack(r.x, r.y), lo = f2_pack(r.z, r.w);
    const unsigned long long magic2 = f2_pack(kMagic, kMagic);
    const unsigned long long t = f2_add_rd(f2_fma(m2, hi, f0), magic2);   // biased floors (tu, tv)
    const unsigned long long ncell = f2_sub(magic2, t);                   // (-cell_u, -cell_v)
    const float2 ab = f2_unpack(f2_add(f2_fma(m2, hi, ncell), f2_fma(m2, lo, f0)));
    const float2 tt = f2_unpack(t);
    const float a = ab.x, b = ab.y;
    const uint32_t iu = min(max(__float_as_uint(tt.x), u.ulo), u.uhi);
    const uint32_t iv = min(max(__float_as_uint(tt.y), u.vlo), u.vhi);
    const uint32_t off = iv * u.row_bytes + iu * 16u + u.koff;
#ifdef PAT_DEBUG
    if (!dbg_ok(*dbg_plan, off <= u.lim, kSiteCircCell)) return 0.f;
#endif
    const float4 c = *reinterpret_cast<const float4*>(smem + off);
    return fmaf(b, fmaf(a, c.w, c.z), fmaf(a, c.y, c.x));
}

} // namespace

#ifdef PAT_DEBUG
#define PAT_DBG_ARG , &dp
#else
#define PAT_DBG_ARG
#endif

template <int ML, typename T>
__global__ void __launch_bounds__(kCircThreads, 2) k_circmean(DevPlan dp, const T* __restrict__ f)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    float4* cells = reinterpret_cast<float4*>(smem_raw);
    float4* rays_s = reinterpret_cast<float4*>(smem_raw + dp.fwd_rays_off);
    constexpr int QL = kWarp / ML;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ml = lane % ML, ql = lane / ML;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);   // the wait probe's barrier: nothing ever arrives on it
        fence_mbar_init();
    }
    __syncthreads();

    uint32_t parity = 0;
    const int task_begin = dp.cta_seg[blockIdx.x], task_end = dp.cta_seg[blockIdx.x + 1];
    for (int tidx = task_begin; tidx < task_end; ++tidx) {
        const Segment sg = dp.segs[tidx];
        const InstDev in = dp.inst[sg.inst];
        __syncthreads(); // every warp is done with the previous tile

        // the staged rays must fit behind the largest tile (uniform over the CTA)
        if (!dbg_ok(dp, (int64_t)in.K * (int64_t)sizeof(float4) <= (int64_t)dp.fwd_smem_bytes - dp.fwd_rays_off,
                    kSiteCircRays))
            return;

        // ---- the instance's rays (TMA bulk copy; a plan table, so before the
        // dependency wait) and the tile's cells (from f, after it) -----------
        if (threadIdx.x == 0) {
            const uint32_t ray_bytes = (uint32_t)in.K * (uint32_t)sizeof(float4);
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[0], ray_bytes);
            bulk_g2s(rays_s, dp.rays + in.ray_off, ray_bytes, &bar[0]);
        }
        if (tidx == task_begin) pdl_wait();   // f belongs to earlier work in the stream
        stage_cells(cells, f + in.f_off, in.n, sg);
        __syncthreads();
        if (!mbar_wait_bounded(&bar[0], parity, dp.status, 1)) {
            mbar_wait_bounded(&bar[0], parity, dp.status, 1); // let copies in flight land before exiting
            return;
        }
        parity ^= 1u;
        if (dp.wait_probe > 0 && blockIdx.x == 0 && tidx == task_begin) {
            // test hook: a wait that runs out (no copy is in flight here)
            if (!mbar_wait_bounded(&bar[1], 0, dp.status, 2, dp.wait_probe)) return;
        }

        // ---- this warp's units (static schedule) ------------------------------
        const float4* det = dp.det + in.det_off;
        const size_t plane = (size_t)in.n_det * in.n_r;
        float* mpart = dp.mpart + in.mpart_off;
        const int ub = dp.warp_units[sg.warp_off + warp], ue = dp.warp_units[sg.warp_off + warp + 1];
        Unit un{};
        if (ub < ue) un = dp.units[ub];
        for (int ui = ub; ui < ue; ++ui) {
            Unit un2{};
            if (ui + 1 < ue) un2 = dp.units[ui + 1];   // the next unit's record, in flight meanwhile
            if (!dbg_ok(dp, un.j >= 0 && un.j < in.n_det && un.q0 >= 0 && un.nq >= 0 && un.q0 + un.nq <= in.K &&
                                un.slot >= 0 && un.slot < in.n_slots && un.m0 >= 0,
                        kSiteCircUnit)) {
                un = un2;
                continue;
            }
            const int m = un.m0 + ml;
            const float mf = (float)m;
            const float4 d = __ldg(det + un.j);
            UnitFrame fr = unit_frame(sg, in, d);
            fr.lim = (uint32_t)((sg.y1 - sg.y0 + 3) * sg.pitch - 1) * 16u;
            const float4* tq = rays_s + un.q0 + ql;   // units never wrap past K
            const unsigned long long m2 = f2_pack(mf, mf), f0 = f2_pack(d.z, d.w);
            float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
            int i = ql;
            for (; i + 3 * QL < un.nq; i += 4 * QL, tq += 4 * QL) {
                const float4 c0 = tq[0], c1 = tq[QL], c2 = tq[2 * QL], c3 = tq[3 * QL];
                acc0 += sample(smem_raw, fr, m2, c0, f0 PAT_DBG_ARG);
                acc1 += sample(smem_raw, fr, m2, c1, f0 PAT_DBG_ARG);
                acc2 += sample(smem_raw, fr, m2, c2, f0 PAT_DBG_ARG);
                acc3 += sample(smem_raw, fr, m2, c3, f0 PAT_DBG_ARG);
            }
            for (; i < un.nq; i += QL, tq += QL) acc0 += sample(smem_raw, fr, m2, *tq, f0 PAT_DBG_ARG);
            float acc = (acc0 + acc1) + (acc2 + acc3);
#pragma unroll
            for (int o = ML; o < kWarp; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (ql == 0 && m < in.n_r) mpart[(size_t)un.slot * plane + (size_t)un.j * in.n_r + m] = acc;
            un = un2;
        }
    }
}

// M[j][m] = sum over the slots of (j, m / ML) in slot order.  Grid (rows of
// M, radius chunks of 128); a row is an (instance, detector) pair.
// A thread keeps eight slots' loads in flight and adds them in slot order.
__global__ void __launch_bounds__(128) k_msum(DevPlan dp)
{
    const int2 row = dp.msum_rows[blockIdx.x];
    const InstDev in = dp.inst[row.x];
    const int j = row.y;
    const int m = blockIdx.y * blockDim.x + threadIdx.x;
    if (m >= in.n_r) return;
    const int cnt = __ldg(reinterpret_cast<const int32_t*>(dp.slotcnt + in.slotcnt_off) + (size_t)j * in.nmb +
                          m / dp.m_lanes);
    const size_t plane = (size_t)in.n_det * in.n_r;
    const float* src = dp.mpart + in.mpart_off + (size_t)j * in.n_r + m;
    pdl_wait();   // the partial slots come from the circular-mean kernel
    float s = 0.f;
    for (int sl = 0; sl < cnt; sl += 8) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = sl + k < cnt ? __ldcg(src + (size_t)(sl + k) * plane) : 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (sl + k < cnt) s += v[k];
    }
    dp.msum[in.mbar_off + (size_t)j * in.m_pitch + m] = s;
}

// Samples whose cell touches the grid, counted with the kernels' FP32 arithmetic.
__global__ void k_count_samples(DevPlan dp, int inst_idx, unsigned long long* __restrict__ out)
{
    const InstDev in = dp.inst[inst_idx];
    const int j = blockIdx.x;
    const float4 d = dp.det[in.det_off + j];
    const float Ui = d.x, Vi = d.y;
    const float4* rays = dp.rays + in.ray_off;
    const float lo = (float)(-1 - in.c0), hi = (float)(in.n - 1 - in.c0);
    unsigned long long c = 0;
    for (int m = threadIdx.x; m < in.n_r; m += blockDim.x) {
        const float mf = (float)m;
        for (int q = 0; q < in.K; ++q) {
            const float4 r = rays[q];
            const float fu = Ui + cell_rel(mf, r.x, d.z), fv = Vi + cell_rel(mf, r.y, d.w);
            c += (fu >= lo && fu <= hi && fv >= lo && fv <= hi) ? 1ull : 0ull;
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

// ---------------------------------------------------------------------------
namespace {
template <int ML, typename T>
const void* circ_fn()
{
    return reinterpret_cast<const void*>(k_circmean<ML, T>);
}
const void* circ_select(int ml, bool bf16)
{
    if (bf16) return ml == 16 ? circ_fn<16, __nv_bfloat16>() : ml == 8 ? circ_fn<8, __nv_bfloat16>()
                                                                           : circ_fn<32, __nv_bfloat16>();
    return ml == 16 ? circ_fn<16, float>() : ml == 8 ? circ_fn<8, float>() : circ_fn<32, float>();
}
} // namespace

cudaError_t launch_circmean(const DevPlan& dp, const void* f, cudaStream_t st, bool msum)
{
    if (dp.n_fwd_ctas == 0) return cudaSuccess;
    const void* fn = circ_select(dp.m_lanes, dp.bf16 != 0);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dp.fwd_smem_bytes);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(dp.n_fwd_ctas);
    cfg.blockDim = dim3(kCircThreads);
    cfg.dynamicSmemBytes = (size_t)dp.fwd_smem_bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DevPlan copy = dp;
    const void* fptr = f;
    void* args[] = {&copy, &fptr};
    e = cudaLaunchKernelExC(&cfg, fn, args);
    if (e != cudaSuccess || !msum) return e;
    return launch_pdl(k_msum, dim3((unsigned)dp.n_msum_rows, (unsigned)((dp.n_r_max + 127) / 128)), dim3(128), 0, st,
                      1, dp);
}

int circmean_blocks_per_sm(int m_lanes, bool bf16, int smem_bytes)
{
    const void* fn = circ_select(m_lanes, bf16);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kCircThreads, smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_count_samples(const DevPlan& dp, int inst_idx, int n_det, unsigned long long* out, cudaStream_t st)
{
    k_count_samples<<<n_det, 128, 0, st>>>(dp, inst_idx, out);
    return cudaGetLastError();
}

} // namespace patgpu
