// circmean.cu — forward circular means M = C f (the first stage of A).
//
// M[j][m] = sum_q f~(y_j + r_m (cos phi_q, sin phi_q)) (the 1/K of the
// trapezoid rule is applied by the Abel stage), f~ the bilinear interpolant
// of f with zero outside the grid: the circular mean of the 2D Poisson
// formula for the wave problem Eq. (1)-(2), discretised as in include/pat.h.
//
// Persistent CTAs.  The work is split into band tasks (an image band of one
// instance and the units whose samples can fall in it).  CTA c works on band
// tasks cta_seg[c] .. cta_seg[c+1]-1; for each it stages the band and the
// instance's K ray directions in shared memory (TMA bulk copies, one per
// image row and one for the rays, completing on an mbarrier) and
// its warps take units, largest first, from the task's global queue, which
// all CTAs assigned to the task share (the last one to finish re-arms it).
// Lane l of a warp handles radius m0 + l % ML and angles
// q0 + l / ML + i * (32 / ML); lanes walk along rays, so their 2 x 2 texel
// reads are spatially coherent.  Each unit writes its own partial-sum slot,
// so the result does not depend on scheduling.
#include "device_common.cuh"
#include "kernels.h"

namespace patgpu {

namespace {

// One bilinear sample of the staged band, branch free: a sample whose cell
// lies outside the band (it belongs to another band or to no pixel) reads the
// zero 2 x 2 block at offset 1 of the band's left padding instead.  Cells are
// relative to the detector's integer part (Ui, Vi); `base` is the offset of
// cell (Ui, Vi) in the band, and the relative cell (iu, iv) is inside the band
// iff iu - ul <= uw and iv - vl <= vw (unsigned).
template <typename T>
__device__ __forceinline__ float sample(const T* __restrict__ s, int W, int base, float mf, float4 r, float Uf,
                                        float Vf, int ul, unsigned uw, int vl, unsigned vw)
{
    const float fu = cell_rel(mf, r.x, Uf), fv = cell_rel(mf, r.y, Vf);
    const int iu = __float2int_rz(fu), iv = __float2int_rz(fv);
    const bool ok = ((unsigned)(iu - ul) <= uw) & ((unsigned)(iv - vl) <= vw);
    const T* p = s + (ok ? iv * W + iu + base : 1);
    const float a = cell_frac(mf, r.x, r.z, Uf, fu), b = cell_frac(mf, r.y, r.w, Vf, fv);
    const float f00 = ld_img(p), f10 = ld_img(p + 1), f01 = ld_img(p + W), f11 = ld_img(p + W + 1);
    const float top = fmaf(a, f10 - f00, f00);
    const float bot = fmaf(a, f11 - f01, f01);
    return fmaf(b, bot - top, top);
}

} // namespace

template <int ML, typename T>
__global__ void __launch_bounds__(kCircThreads) k_circmean(DevPlan dp, const T* __restrict__ f)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    T* s = reinterpret_cast<T*>(smem_raw);
    float4* rays_s = reinterpret_cast<float4*>(smem_raw + dp.fwd_rays_off);
    constexpr int QL = kWarp / ML;
    constexpr int CO = ImgTraits<T>::col_off;
    const int lane = threadIdx.x & 31;
    const int ml = lane % ML, ql = lane / ML;

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();   // f and the work queues belong to earlier work in the stream

    uint32_t parity = 0;
    const int task_begin = dp.cta_seg[blockIdx.x], task_end = dp.cta_seg[blockIdx.x + 1];
    for (int tidx = task_begin; tidx < task_end; ++tidx) {
        const Segment sg = dp.segs[tidx];
        const InstDev in = dp.inst[sg.inst];
        const int n = in.n;
        const int W = ImgTraits<T>::pitch(n);
        const int rows = sg.band_hi - sg.band_lo + 1;
        const int nu = sg.unit_end - sg.unit_begin;
        __syncthreads(); // every warp is done with the previous band

        // ---- stage the band's image rows (TMA bulk copies) -----------------
        if (threadIdx.x < 32) {
            const int r0 = max(sg.band_lo, 0), r1 = min(sg.band_hi, n - 1);
            const uint32_t row_bytes = (uint32_t)n * sizeof(T);
            const uint32_t ray_bytes = (uint32_t)in.K * (uint32_t)sizeof(float4);
            if (lane == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bar, (r1 >= r0 ? (uint32_t)(r1 - r0 + 1) * row_bytes : 0u) + ray_bytes);
                bulk_g2s(rays_s, dp.rays + in.ray_off, ray_bytes, &bar);
            }
            __syncwarp();
            for (int r = r0 + lane; r <= r1; r += 32)
                bulk_g2s(s + (r - sg.band_lo) * W + CO, f + in.f_off + (size_t)r * n, row_bytes, &bar);
        }
        // ---- zero borders: columns 0 .. CO-1 and N+CO .. W-1 (padding), rows
        // outside the image; columns 1, 2 of rows 0, 1 are the zero block
        const T zero = T(0.f);
        const int pad = W - (CO + n);
        for (int i = threadIdx.x; i < rows * (pad + CO); i += blockDim.x) {
            const int ri = i / (pad + CO), c = i - ri * (pad + CO);
            s[ri * W + (c < CO ? c : n + c)] = zero;
        }
        // only the first band row (-1) and the last (n) can lie outside the image
        if (sg.band_lo < 0)
            for (int c = threadIdx.x; c < n; c += blockDim.x) s[CO + c] = zero;
        if (sg.band_hi >= n)
            for (int c = threadIdx.x; c < n; c += blockDim.x) s[(n - sg.band_lo) * W + CO + c] = zero;
        __syncthreads();
        if (!mbar_wait_bounded(&bar, parity, dp.status, 1)) {
            mbar_wait_bounded(&bar, parity, dp.status, 1); // let copies in flight land before exiting
            return;
        }
        parity ^= 1u;

        // ---- units: shared queue of every CTA working on this band task ----
        // centred cell (i0c, j0c) lives at s[(j0c + c0 - band_lo) * W + i0c + c0 + CO]
        const int ulo = -1 - in.c0, vlo = sg.band_lo - in.c0;
        const unsigned uw = (unsigned)n, vw = (unsigned)(sg.band_hi - 1 - sg.band_lo);
        const float4* det = dp.det + in.det_off;
        const Unit* units = dp.units + sg.unit_begin;
        int32_t* queue = dp.work_counters + (2 + sg.queue) * kQueueStride;

        const size_t plane = (size_t)in.n_det * in.n_r;
        const int32_t* slotcnt = reinterpret_cast<const int32_t*>(dp.slotcnt + in.slotcnt_off);
        // The last unit of (j, radius block) to arrive sums the block's slots in
        // slot order (deterministic) into M and re-arms the counter.
        // blocks are j * nmb + m0 / ML; this lane's radius in a block is m0 + ml
        int p_blk = -1;                  // slot written, arrival not yet counted
        int q_blk = -1, q_total = 0;     // arrival counted, result pending (lane 0)
        int q_ret = 0;
        auto resolve = [&]() {
            const int last = __shfl_sync(0xffffffffu, q_ret == q_total - 1 ? 1 : 0, 0);
            if (last) {
                __threadfence();
                const int q_j = q_blk / in.nmb, q_m = (q_blk - q_j * in.nmb) * ML + ml;
                if (ql == 0 && q_m < in.n_r) {
                    const float* sl0 = dp.mpart + in.mpart_off + (size_t)q_j * in.n_r + q_m;
                    // four slots' loads in flight at a time, added in slot order
                    float sum = 0.f;
                    int sl = 0;
                    for (; sl + 4 <= q_total; sl += 4) {
                        const float a0 = __ldcg(sl0 + (size_t)sl * plane), a1 = __ldcg(sl0 + (size_t)(sl + 1) * plane);
                        const float a2 = __ldcg(sl0 + (size_t)(sl + 2) * plane), a3 = __ldcg(sl0 + (size_t)(sl + 3) * plane);
                        sum += a0;
                        sum += a1;
                        sum += a2;
                        sum += a3;
                    }
                    for (; sl < q_total; ++sl) sum += __ldcg(sl0 + (size_t)sl * plane);
                    dp.msum[in.mbar_off + (size_t)q_j * in.n_rp + q_m] = sum;
                }
                if (lane == 0) dp.slot_arrivals[in.arrive_off + q_blk] = 0;
            }
            q_blk = -1;
        };

        int u = 0;
        if (lane == 0) u = atomicAdd(queue, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        Unit un{};
        if (u < nu) un = units[u];
        while (u < nu) {
            // take and fetch the next unit while this one is processed
            int u2 = 0;
            if (lane == 0) u2 = atomicAdd(queue, 1);
            u2 = __shfl_sync(0xffffffffu, u2, 0);
            Unit un2{};
            if (u2 < nu) un2 = units[u2];

            const int m = un.m0 + ml;
            const float mf = (float)m;
            const float4 d = __ldg(det + un.j);
            const int Ui = __float2int_rz(d.x), Vi = __float2int_rz(d.y);
            const int base = (Vi + in.c0 - sg.band_lo) * W + Ui + in.c0 + CO;
            const int ul = ulo - Ui, vl = vlo - Vi;
            const float4* tq = rays_s + un.q0 + ql;   // units never wrap past K
            float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
            int i = ql;
            for (; i + 3 * QL < un.nq; i += 4 * QL, tq += 4 * QL) {
                const float4 c0 = tq[0], c1 = tq[QL], c2 = tq[2 * QL], c3 = tq[3 * QL];
                acc0 += sample(s, W, base, mf, c0, d.z, d.w, ul, uw, vl, vw);
                acc1 += sample(s, W, base, mf, c1, d.z, d.w, ul, uw, vl, vw);
                acc2 += sample(s, W, base, mf, c2, d.z, d.w, ul, uw, vl, vw);
                acc3 += sample(s, W, base, mf, c3, d.z, d.w, ul, uw, vl, vw);
            }
            for (; i < un.nq; i += QL, tq += QL) acc0 += sample(s, W, base, mf, *tq, d.z, d.w, ul, uw, vl, vw);
            float acc = (acc0 + acc1) + (acc2 + acc3);
#pragma unroll
            for (int o = ML; o < kWarp; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            // Pipelined arrival: the arrival counted for the unit before last
            // is resolved now (its atomic returned while this unit was sampled),
            // the previous unit's arrival is issued now (its slot write has
            // drained, so the fence is cheap), and this unit's slot is written.
            if (q_blk >= 0) resolve();
            if (p_blk >= 0) {
                __threadfence();
                q_blk = p_blk;
                q_total = slotcnt[p_blk];
                if (lane == 0) q_ret = atomicAdd(dp.slot_arrivals + in.arrive_off + p_blk, 1);
            }
            if (ql == 0 && m < in.n_r) dp.mpart[in.mpart_off + (size_t)un.slot * plane + (size_t)un.j * in.n_r + m] = acc;
            p_blk = un.j * in.nmb + un.m0 / ML;
            u = u2;
            un = un2;
        }
        if (q_blk >= 0) resolve();
        if (p_blk >= 0) {
            __threadfence();
            q_blk = p_blk;
            q_total = slotcnt[p_blk];
            if (lane == 0) q_ret = atomicAdd(dp.slot_arrivals + in.arrive_off + p_blk, 1);
            resolve();
        }
        // this CTA is done with the band task; its last participant re-arms the queue
        __syncthreads();
        if (threadIdx.x == 0 && atomicAdd(queue + 1, 1) == sg.parts - 1) {
            queue[0] = 0;
            queue[1] = 0;
        }
    }
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

cudaError_t launch_circmean(const DevPlan& dp, const void* f, cudaStream_t st)
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
    return cudaLaunchKernelExC(&cfg, fn, args);
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
