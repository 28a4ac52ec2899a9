// kernels.cu — device kernels of the photoacoustic operator library (sm_103a).
//
//   k_circmean        circular means: M = C f            (gather over samples)
//   k_abel_fwd        Abel + time derivative: g = P M / K (lower-triangular)
//   k_abel_adj        its transpose: Mbar = P^T g         (upper-triangular)
//   k_adjoint_gather  C^T Mbar as a gather over pixels    (no atomics)
//   k_tv              smoothed isotropic TV value + gradient
//   k_residual, k_descent, k_tile_sums   small elementwise helpers
//
// The operator is the direct discretisation of the 2D Poisson solution of
// the wave problem Eq. (1)-(3) described in include/pat.h; the coordinate
// conventions and the shared sample expression are in pat_internal.h.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "pat_internal.h"
#include "kernels.h"

namespace patgpu {

namespace {

__device__ __forceinline__ float ld_img(const float* p) { return *p; }
__device__ __forceinline__ float ld_img(const __nv_bfloat16* p) { return __bfloat162float(*p); }

__device__ __forceinline__ int pitch_f32(int n)
{
    int w = n + kColOff + 1;
    return w + ((12 - (w & 31)) & 31);
}
__device__ __forceinline__ int pitch_bf16(int n)
{
    int w = n + kColOffBF16 + 1;
    return w + ((24 - (w & 63)) & 63);
}

// ---------------------------------------------------------------------------
// Stage rows [lo, hi] (absolute, inclusive; rows outside 0..N-1 are zero) of
// an N-wide image into shared memory with row pitch W and column 0 at offset
// col_off; columns -1 and N are zero.
// ---------------------------------------------------------------------------
__device__ void stage_band(float* s, const float* __restrict__ img, int n, int lo, int hi, int W)
{
    const int rows = hi - lo + 1;
    const int nv = n >> 2;
    const int total = rows * nv;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int ri = i / nv, c4 = i - ri * nv;
        const int r = lo + ri;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r >= 0 && r < n) v = __ldg(reinterpret_cast<const float4*>(img + (size_t)r * n) + c4);
        *reinterpret_cast<float4*>(s + ri * W + kColOff + 4 * c4) = v;
    }
    for (int ri = threadIdx.x; ri < rows; ri += blockDim.x) {
        s[ri * W + kColOff - 1] = 0.f;
        s[ri * W + kColOff + n] = 0.f;
    }
}

__device__ void stage_band(__nv_bfloat16* s, const __nv_bfloat16* __restrict__ img, int n, int lo, int hi, int W)
{
    const int rows = hi - lo + 1;
    const int nv = n >> 3;
    const int total = rows * nv;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int ri = i / nv, c8 = i - ri * nv;
        const int r = lo + ri;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r >= 0 && r < n) v = __ldg(reinterpret_cast<const uint4*>(img + (size_t)r * n) + c8);
        *reinterpret_cast<uint4*>(s + ri * W + kColOffBF16 + 8 * c8) = v;
    }
    const __nv_bfloat16 z = __float2bfloat16(0.f);
    for (int ri = threadIdx.x; ri < rows; ri += blockDim.x) {
        s[ri * W + kColOffBF16 - 1] = z;
        s[ri * W + kColOffBF16 + n] = z;
    }
}

template <typename T> struct ImgTraits;
template <> struct ImgTraits<float> {
    static __device__ __forceinline__ int pitch(int n) { return pitch_f32(n); }
    static constexpr int col_off = kColOff;
};
template <> struct ImgTraits<__nv_bfloat16> {
    static __device__ __forceinline__ int pitch(int n) { return pitch_bf16(n); }
    static constexpr int col_off = kColOffBF16;
};

// One bilinear sample of the staged band.  Returns 0 for samples whose cell
// lies outside the band (they belong to another band or to no pixel).
template <typename T>
__device__ __forceinline__ float sample(const T* __restrict__ s, int W, float rho, float2 cs, float U,
                                        float V, float ulo, float uhi, float vlo, float vhi)
{
    const float u = __fmaf_rn(rho, cs.x, U);
    const float v = __fmaf_rn(rho, cs.y, V);
    const float fu = floorf(u), fv = floorf(v);
    const bool ok = (fu >= ulo) & (fu <= uhi) & (fv >= vlo) & (fv <= vhi);
    float r = 0.f;
    if (ok) {
        const float a = __fsub_rn(u, fu), b = __fsub_rn(v, fv);
        const T* p = s + (__float2int_rz(fv) * W + __float2int_rz(fu));
        const float f00 = ld_img(p), f10 = ld_img(p + 1);
        const float f01 = ld_img(p + W), f11 = ld_img(p + W + 1);
        const float top = fmaf(a, f10 - f00, f00);
        const float bot = fmaf(a, f11 - f01, f01);
        r = fmaf(b, bot - top, top);
    }
    return r;
}

} // namespace

// ---------------------------------------------------------------------------
// Circular means.  Persistent CTAs; CTA c owns segments cta_seg[c]..; for each
// it stages the segment's image band in shared memory, then its warps take
// the segment's units in order (largest first) from a shared counter.  Lane
// l of a warp handles radius m0 + l % ML and angles q0 + l / ML + i * (32/ML);
// the partial sum of a unit is written to its own slot, so the result does
// not depend on scheduling.
// ---------------------------------------------------------------------------
template <int ML, typename T>
__global__ void __launch_bounds__(kCircThreads) k_circmean(DevPlan dp, const T* __restrict__ f)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s = reinterpret_cast<T*>(smem_raw);
    __shared__ int s_next;
    constexpr int QL = kWarp / ML;
    const int lane = threadIdx.x & 31;
    const int ml = lane % ML, ql = lane / ML;

    const int seg_begin = dp.cta_seg[blockIdx.x], seg_end = dp.cta_seg[blockIdx.x + 1];
    for (int sidx = seg_begin; sidx < seg_end; ++sidx) {
        const Segment sg = dp.segs[sidx];
        const InstDev in = dp.inst[sg.inst];
        const int W = ImgTraits<T>::pitch(in.n);
        __syncthreads(); // previous segment finished with the shared band
        stage_band(s, f + in.f_off, in.n, sg.band_lo, sg.band_hi, W);
        if (threadIdx.x == 0) s_next = 0;
        __syncthreads();

        // cell (i0c, j0c) in centred units lives at s[j0c * W + i0c + base]
        const T* sb = s + ((in.c0 - sg.band_lo) * W + in.c0 + ImgTraits<T>::col_off);
        const float ulo = (float)(-1 - in.c0), uhi = (float)(in.n - 1 - in.c0);
        const float vlo = (float)(sg.band_lo - in.c0), vhi = (float)(sg.band_hi - 1 - in.c0);
        const float* detU = dp.detU + in.det_off;
        const float* detV = dp.detV + in.det_off;
        const float2* trig = dp.trig + in.trig_off;
        const int nunits = sg.unit_end - sg.unit_begin;

        for (;;) {
            int u = 0;
            if (lane == 0) u = atomicAdd(&s_next, 1);
            u = __shfl_sync(0xffffffffu, u, 0);
            if (u >= nunits) break;
            const Unit un = dp.units[sg.unit_begin + u];
            const int m = un.m0 + ml;
            const float rho = (float)m * in.delta;
            const float U = __ldg(detU + un.j), V = __ldg(detV + un.j);
            const float2* tq = trig + un.q0 + ql;
            float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
            int i = ql;
            for (; i + 3 * QL < un.nq; i += 4 * QL, tq += 4 * QL) {
                const float2 c0 = __ldg(tq), c1 = __ldg(tq + QL), c2 = __ldg(tq + 2 * QL), c3 = __ldg(tq + 3 * QL);
                acc0 += sample(sb, W, rho, c0, U, V, ulo, uhi, vlo, vhi);
                acc1 += sample(sb, W, rho, c1, U, V, ulo, uhi, vlo, vhi);
                acc2 += sample(sb, W, rho, c2, U, V, ulo, uhi, vlo, vhi);
                acc3 += sample(sb, W, rho, c3, U, V, ulo, uhi, vlo, vhi);
            }
            for (; i < un.nq; i += QL, tq += QL) acc0 += sample(sb, W, rho, __ldg(tq), U, V, ulo, uhi, vlo, vhi);
            float acc = (acc0 + acc1) + (acc2 + acc3);
#pragma unroll
            for (int o = ML; o < kWarp; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (ql == 0 && m < in.n_r)
                dp.mpart[in.mpart_off + ((size_t)un.slot * in.n_det + un.j) * in.n_r + m] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Abel stage, forward:  g[j][kk] = (1/K) sum_{m <= kk+2} P[kk][m] M[j][m],
// M[j][m] = sum over the unit slots of (j, m / ML).  Tile 16 detectors x 64
// times, m in chunks of 32; the triangle above m = kk + 2 is skipped.
// ---------------------------------------------------------------------------
constexpr int kTJ = 16, kTX = 64, kTC = 32;

__global__ void __launch_bounds__(256) k_abel_fwd(DevPlan dp, float* __restrict__ g)
{
    __shared__ float sA[kTJ][kTC + 1];
    __shared__ float sB[kTX][kTC + 1];
    const TimeTile t = dp.fwd_tiles[blockIdx.x];
    const InstDev in = dp.inst[t.inst];
    const int tid = threadIdx.x;
    const int tj = tid >> 4, tk = tid & 15;
    const int n_r = in.n_r;
    const int m_end = min(n_r, t.x0 + kTX + 2);
    const float* P = dp.P + in.p_off;
    const float* mp = dp.mpart + in.mpart_off;
    const int32_t* cnt = reinterpret_cast<const int32_t*>(dp.slotcnt + in.slotcnt_off);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int m0 = 0; m0 < m_end; m0 += kTC) {
        for (int e = tid; e < kTJ * kTC; e += 256) {
            const int r = e / kTC, c = e % kTC;
            const int j = t.j0 + r, m = m0 + c;
            float v = 0.f;
            if (j < in.n_det && m < n_r) {
                const int ns = cnt[j * in.nmb + m / dp.m_lanes];
                for (int sl = 0; sl < ns; ++sl) v += mp[((size_t)sl * in.n_det + j) * n_r + m];
            }
            sA[r][c] = v;
        }
        for (int e = tid; e < kTX * kTC; e += 256) {
            const int r = e / kTC, c = e % kTC;
            const int kk = t.x0 + r, m = m0 + c;
            sB[r][c] = (kk < in.n_t && m < n_r) ? __ldg(P + (size_t)kk * n_r + m) : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < kTC; ++c) {
            const float a = sA[tj][c];
            acc[0] = fmaf(sB[tk][c], a, acc[0]);
            acc[1] = fmaf(sB[tk + 16][c], a, acc[1]);
            acc[2] = fmaf(sB[tk + 32][c], a, acc[2]);
            acc[3] = fmaf(sB[tk + 48][c], a, acc[3]);
        }
        __syncthreads();
    }
    const int j = t.j0 + tj;
    if (j < in.n_det) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int kk = t.x0 + tk + 16 * i;
            if (kk < in.n_t) g[in.g_off + (size_t)j * in.n_t + kk] = acc[i] * in.inv_K;
        }
    }
}

// ---------------------------------------------------------------------------
// Abel stage, adjoint:  Mbar[j][m] = sum_{kk >= m-2} P[kk][m] g[j][kk].
// Tile 16 detectors x 64 radii, kk in chunks of 32 starting at max(0, m0-2).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_abel_adj(DevPlan dp, const float* __restrict__ g)
{
    __shared__ float sA[kTJ][kTC + 1];
    __shared__ float sB[kTC][kTX + 1];
    const TimeTile t = dp.adj_tiles[blockIdx.x];
    const InstDev in = dp.inst[t.inst];
    const int tid = threadIdx.x;
    const int tj = tid >> 4, tm = tid & 15;
    const int n_r = in.n_r, n_t = in.n_t;
    const float* P = dp.P + in.p_off;
    const float* gi = g + in.g_off;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = max(0, t.x0 - 2); k0 < n_t; k0 += kTC) {
        for (int e = tid; e < kTJ * kTC; e += 256) {
            const int r = e / kTC, c = e % kTC;
            const int j = t.j0 + r, kk = k0 + c;
            sA[r][c] = (j < in.n_det && kk < n_t) ? __ldg(gi + (size_t)j * n_t + kk) : 0.f;
        }
        for (int e = tid; e < kTC * kTX; e += 256) {
            const int r = e / kTX, c = e % kTX;
            const int kk = k0 + r, m = t.x0 + c;
            sB[r][c] = (kk < n_t && m < n_r) ? __ldg(P + (size_t)kk * n_r + m) : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < kTC; ++c) {
            const float a = sA[tj][c];
            acc[0] = fmaf(sB[c][tm], a, acc[0]);
            acc[1] = fmaf(sB[c][tm + 16], a, acc[1]);
            acc[2] = fmaf(sB[c][tm + 32], a, acc[2]);
            acc[3] = fmaf(sB[c][tm + 48], a, acc[3]);
        }
        __syncthreads();
    }
    const int j = t.j0 + tj;
    if (j < in.n_det) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = t.x0 + tm + 16 * i;
            if (m < n_r) dp.mbar[in.mbar_off + (size_t)j * n_r + m] = acc[i];
        }
    }
}

// ---------------------------------------------------------------------------
// Adjoint circular means as a gather.  Thread = cell (i0, j0) of a 16 x 16
// tile; for every detector it enumerates the (m, q) samples that can land in
// its cell — radii with |r_m - rho_c| <= R and, per radius, the angles of the
// arc within R of the cell centre (R = half the cell diagonal plus a margin
// that covers the FP32 rounding of the sample positions) — re-evaluates each
// candidate with exactly the forward's expression, and accumulates the four
// corner weights of the samples that do land in the cell.  Pixels then sum
// the corner sums of their four cells.  Each output is summed by one thread in
// a fixed order: deterministic, no atomics.
// ---------------------------------------------------------------------------
namespace {

constexpr float kR = 0.70710678f + 0.004f;
constexpr float kR2 = kR * kR;
constexpr float kPi = 3.14159265358979f;
constexpr float kAtanErr = 1.0e-5f;  // > 5x the bound on |atan2_approx - atan2| (radians)

// atan(x) on [0, 1]: odd polynomial x * p(x^2), coefficients fitted by
// iteratively reweighted least squares on 4000 Chebyshev nodes; evaluated in
// FP32 its max abs error is 1.7e-6 rad.  Only the adjoint's candidate window
// uses it, widened by kAtanErr, and every candidate is re-checked exactly.
__device__ __forceinline__ float atan_01(float x)
{
    const float x2 = x * x;
    float p = -0.01171913f;
    p = fmaf(p, x2, 0.05264734f);
    p = fmaf(p, x2, -0.11642648f);
    p = fmaf(p, x2, 0.19354038f);
    p = fmaf(p, x2, -0.33262283f);
    p = fmaf(p, x2, 0.99997722f);
    return x * p;
}

__device__ __forceinline__ float atan2_approx(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = mx > 0.f ? __fdividef(mn, mx) : 0.f;
    float r = atan_01(t);
    if (ay > ax) r = 0.5f * kPi - r;
    if (x < 0.f) r = kPi - r;
    return copysignf(r, y);
}

// Upper bound of asin(s) for s in [0, 1].
__device__ __forceinline__ float asin_upper(float s)
{
    return s <= 0.7f ? s * fmaf(0.25f, s * s, 1.0f) : asinf(fminf(s, 1.0f)) + 1e-6f;
}

} // namespace

template <int G, typename T>
__global__ void __launch_bounds__(256 * G) k_adjoint_gather(DevPlan dp, T* __restrict__ fout)
{
    __shared__ float4 sz[G][256];
    const AdjTile t = dp.gather_tiles[blockIdx.x];
    const InstDev in = dp.inst[t.inst];
    const int cell = threadIdx.x & 255, grp = threadIdx.x >> 8;
    const int tx = cell & 15, ty = cell >> 4;
    const int cx = t.x0 - 1 + tx, cy = t.y0 - 1 + ty;
    const float cxc = (float)(cx - in.c0), cyc = (float)(cy - in.c0);
    float z00 = 0.f, z10 = 0.f, z01 = 0.f, z11 = 0.f;
    if (cx <= in.n - 1 && cy <= in.n - 1) {
        const float ccx = cxc + 0.5f, ccy = cyc + 0.5f;
        const float* detU = dp.detU + in.det_off;
        const float* detV = dp.detV + in.det_off;
        const float2* trig = dp.trig + in.trig_off;
        const float* mb = dp.mbar + in.mbar_off;
        const int K = in.K;
        for (int j = grp; j < in.n_det; j += G) {
            const float U = __ldg(detU + j), V = __ldg(detV + j);
            const float du = ccx - U, dv = ccy - V;
            const float rc = sqrtf(fmaf(du, du, dv * dv));
            const int mlo = max(0, (int)ceilf((rc - kR) * in.inv_delta));
            const int mhi = min(in.n_r - 1, (int)floorf((rc + kR) * in.inv_delta));
            if (mlo > mhi) continue;
            const float phic = atan2_approx(dv, du);
            const float* mbj = mb + (size_t)j * in.n_r;
            for (int m = mlo; m <= mhi; ++m) {
                const float rho = (float)m * in.delta;
                const float d = rho - rc;
                const float num = kR2 - d * d;           // R^2 - (rho - rc)^2
                if (num < 0.f) continue;                 // circle misses the disc about the centre
                const float den = 4.f * rho * rc;
                int qlo = 0, qn = K;
                if (den > num) {                         // otherwise the whole circle is within R
                    // half-angle of the arc within R of the cell centre:
                    // sin^2(alpha/2) = (R^2 - (rho - rc)^2) / (4 rho rc)
                    const float alpha = 2.f * asin_upper(sqrtf(__fdividef(num, den))) + kAtanErr;
                    const float lo = (phic - alpha) * in.inv_dphi;
                    const float hi = (phic + alpha) * in.inv_dphi;
                    qlo = (int)ceilf(lo);
                    qn = min((int)floorf(hi) - qlo + 1, K);
                    if (qn <= 0) continue;
                    if (qlo < 0) qlo += K;
                }
                float s1 = 0.f, sa = 0.f, sb = 0.f, sab = 0.f;
                const float2* tq = trig + qlo;
                for (int i = 0; i < qn; ++i) {
                    const float2 cs = __ldg(tq + i);
                    const float u = __fmaf_rn(rho, cs.x, U);
                    const float v = __fmaf_rn(rho, cs.y, V);
                    const float fu = floorf(u), fv = floorf(v);
                    if (fu == cxc && fv == cyc) {
                        const float a = __fsub_rn(u, fu), b = __fsub_rn(v, fv);
                        s1 += 1.f;
                        sa += a;
                        sb += b;
                        sab = fmaf(a, b, sab);
                    }
                }
                if (s1 > 0.f) {
                    const float w = __ldg(mbj + m);
                    z00 = fmaf((s1 - sa) - (sb - sab), w, z00);
                    z10 = fmaf(sa - sab, w, z10);
                    z01 = fmaf(sb - sab, w, z01);
                    z11 = fmaf(sab, w, z11);
                }
            }
        }
    }
    sz[grp][cell] = make_float4(z00, z10, z01, z11);
    __syncthreads();
    if (grp == 0) {
        float4 z = sz[0][cell];
#pragma unroll
        for (int gi = 1; gi < G; ++gi) {
            const float4 w = sz[gi][cell];
            z.x += w.x; z.y += w.y; z.z += w.z; z.w += w.w;
        }
        sz[0][cell] = z;
    }
    __syncthreads();
    if (grp == 0 && tx < kAdjOut && ty < kAdjOut) {
        const int px = t.x0 + tx, py = t.y0 + ty;
        if (px < in.n && py < in.n) {
            // pixel (px, py) = Z00(px,py) + Z10(px-1,py) + Z01(px,py-1) + Z11(px-1,py-1)
            const float v = sz[0][(ty + 1) * 16 + tx + 1].x + sz[0][(ty + 1) * 16 + tx].y +
                            sz[0][ty * 16 + tx + 1].z + sz[0][ty * 16 + tx].w;
            const float val = v * in.inv_K;
            if constexpr (sizeof(T) == 4) fout[in.f_off + (size_t)py * in.n + px] = val;
            else fout[in.f_off + (size_t)py * in.n + px] = __float2bfloat16(val);
        }
    }
}

// ---------------------------------------------------------------------------
// Smoothed isotropic TV: value partial sums per 32 x 8 tile and gradient.
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ float tv_term(const float* f, int n, int i, int j, float eps2, float& dx, float& dy)
{
    const float c = f[(size_t)i * n + j];
    dx = (j + 1 < n) ? f[(size_t)i * n + j + 1] - c : 0.f;
    dy = (i + 1 < n) ? f[(size_t)(i + 1) * n + j] - c : 0.f;
    return sqrtf(fmaf(dx, dx, fmaf(dy, dy, eps2)));
}

template <int NT>
__device__ __forceinline__ float block_sum(float v, float* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}
} // namespace

__global__ void __launch_bounds__(256) k_tv(DevPlan dp, const float* __restrict__ f, float eps, float* __restrict__ grad)
{
    __shared__ float red[8];
    const ImgTile t = dp.img_tiles[blockIdx.x];
    const InstDev in = dp.inst[t.inst];
    const int n = in.n;
    const float* fi = f + in.f_off;
    const int j = t.x0 + (threadIdx.x & 31), i = t.y0 + (threadIdx.x >> 5);
    const float eps2 = eps * eps;
    float val = 0.f;
    if (i < n && j < n) {
        float dx, dy;
        const float s = tv_term(fi, n, i, j, eps2, dx, dy);
        val = s;
        if (grad) {
            float gsum = -(dx + dy) / s;
            if (j > 0) {
                float dxl, dyl;
                const float sl = tv_term(fi, n, i, j - 1, eps2, dxl, dyl);
                gsum += dxl / sl;
            }
            if (i > 0) {
                float dxu, dyu;
                const float su = tv_term(fi, n, i - 1, j, eps2, dxu, dyu);
                gsum += dyu / su;
            }
            grad[in.f_off + (size_t)i * n + j] = gsum;
        }
    }
    const float s = block_sum<256>(val, red);
    if (threadIdx.x == 0) dp.tv_partial[blockIdx.x] = s;
}

// Per-instance sums of per-tile partials (fixed order): out[i*stride + c].
__global__ void k_tile_sums(DevPlan dp, const float* __restrict__ part, int ncomp, float* __restrict__ out)
{
    const int inst = blockIdx.x;
    if (threadIdx.x >= ncomp) return;
    float s = 0.f;
    for (int b = 0; b < dp.n_img_tiles; ++b)
        if (dp.img_tiles[b].inst == inst) s += part[(size_t)b * ncomp + threadIdx.x];
    out[(size_t)inst * ncomp + threadIdx.x] = s;
}

__global__ void k_residual(const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ r, float scale,
                           int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = scale * (a[i] - b[i]);
}

__global__ void __launch_bounds__(256) k_descent(DevPlan dp, float* __restrict__ f, const float* __restrict__ adj,
                                                 const float* __restrict__ tvg, float tau, float lam, int nonneg,
                                                 float* __restrict__ part)
{
    __shared__ float red[8];
    const ImgTile t = dp.img_tiles[blockIdx.x];
    const InstDev in = dp.inst[t.inst];
    const int n = in.n;
    const int j = t.x0 + (threadIdx.x & 31), i = t.y0 + (threadIdx.x >> 5);
    float d2 = 0.f, n2 = 0.f;
    if (i < n && j < n) {
        const size_t idx = in.f_off + (size_t)i * n + j;
        const float old = f[idx];
        float gr = adj[idx];
        if (tvg) gr = fmaf(lam, tvg[idx], gr);
        float nv = fmaf(-tau, gr, old);
        if (nonneg) nv = fmaxf(nv, 0.f);
        f[idx] = nv;
        d2 = (nv - old) * (nv - old);
        n2 = nv * nv;
    }
    if (part) {
        const float s0 = block_sum<256>(d2, red);
        const float s1 = block_sum<256>(n2, red);
        if (threadIdx.x == 0) {
            part[2 * blockIdx.x] = s0;
            part[2 * blockIdx.x + 1] = s1;
        }
    }
}

// Samples whose cell touches the grid, per (instance, detector, radius block).
__global__ void k_count_samples(DevPlan dp, int inst_idx, unsigned long long* __restrict__ out)
{
    const InstDev in = dp.inst[inst_idx];
    const int j = blockIdx.x;
    const float U = dp.detU[in.det_off + j], V = dp.detV[in.det_off + j];
    const float2* trig = dp.trig + in.trig_off;
    const float lo = (float)(-1 - in.c0), hi = (float)(in.n - 1 - in.c0);
    unsigned long long c = 0;
    for (int m = threadIdx.x; m < in.n_r; m += blockDim.x) {
        const float rho = (float)m * in.delta;
        for (int q = 0; q < in.K; ++q) {
            const float2 cs = trig[q];
            const float fu = floorf(__fmaf_rn(rho, cs.x, U)), fv = floorf(__fmaf_rn(rho, cs.y, V));
            c += (fu >= lo && fu <= hi && fv >= lo && fv <= hi) ? 1ull : 0ull;
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <int ML, typename T>
static cudaError_t launch_circ_t(const DevPlan& dp, const void* f, cudaStream_t st)
{
    auto kern = k_circmean<ML, T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dp.fwd_smem_bytes);
    if (e != cudaSuccess) return e;
    kern<<<dp.n_fwd_ctas, kCircThreads, dp.fwd_smem_bytes, st>>>(dp, static_cast<const T*>(f));
    return cudaGetLastError();
}

cudaError_t launch_circmean(const DevPlan& dp, const void* f, cudaStream_t st)
{
    if (dp.n_fwd_ctas == 0) return cudaSuccess;
    if (dp.bf16) {
        switch (dp.m_lanes) {
        case 16: return launch_circ_t<16, __nv_bfloat16>(dp, f, st);
        case 8: return launch_circ_t<8, __nv_bfloat16>(dp, f, st);
        default: return launch_circ_t<32, __nv_bfloat16>(dp, f, st);
        }
    }
    switch (dp.m_lanes) {
    case 16: return launch_circ_t<16, float>(dp, f, st);
    case 8: return launch_circ_t<8, float>(dp, f, st);
    default: return launch_circ_t<32, float>(dp, f, st);
    }
}

cudaError_t launch_abel_fwd(const DevPlan& dp, float* g, cudaStream_t st)
{
    if (dp.n_fwd_tiles == 0) return cudaSuccess;
    k_abel_fwd<<<dp.n_fwd_tiles, 256, 0, st>>>(dp, g);
    return cudaGetLastError();
}

cudaError_t launch_abel_adj(const DevPlan& dp, const float* g, cudaStream_t st)
{
    if (dp.n_adj_tiles == 0) return cudaSuccess;
    k_abel_adj<<<dp.n_adj_tiles, 256, 0, st>>>(dp, g);
    return cudaGetLastError();
}

template <int G>
static cudaError_t launch_gather_g(const DevPlan& dp, void* f, cudaStream_t st)
{
    if (dp.bf16) k_adjoint_gather<G, __nv_bfloat16><<<dp.n_gather_tiles, 256 * G, 0, st>>>(dp, static_cast<__nv_bfloat16*>(f));
    else k_adjoint_gather<G, float><<<dp.n_gather_tiles, 256 * G, 0, st>>>(dp, static_cast<float*>(f));
    return cudaGetLastError();
}

cudaError_t launch_adjoint_gather(const DevPlan& dp, void* f, cudaStream_t st)
{
    if (dp.n_gather_tiles == 0) return cudaSuccess;
    switch (dp.adj_groups) {
    case 1: return launch_gather_g<1>(dp, f, st);
    case 2: return launch_gather_g<2>(dp, f, st);
    default: return launch_gather_g<4>(dp, f, st);
    }
}

cudaError_t launch_tv(const DevPlan& dp, const float* f, float eps, float* grad, float* value, cudaStream_t st)
{
    if (dp.n_img_tiles == 0) return cudaSuccess;
    k_tv<<<dp.n_img_tiles, 256, 0, st>>>(dp, f, eps, grad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !value) return e;
    k_tile_sums<<<dp.n_inst, 32, 0, st>>>(dp, dp.tv_partial, 1, value);
    return cudaGetLastError();
}

cudaError_t launch_residual(const float* a, const float* b, float* r, float scale, int64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    k_residual<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(a, b, r, scale, n);
    return cudaGetLastError();
}

cudaError_t launch_descent(const DevPlan& dp, float* f, const float* adj, const float* tvg, float tau, float lam,
                           int nonneg, float* delta, cudaStream_t st)
{
    if (dp.n_img_tiles == 0) return cudaSuccess;
    k_descent<<<dp.n_img_tiles, 256, 0, st>>>(dp, f, adj, tvg, tau, lam, nonneg, delta ? dp.tv_partial : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !delta) return e;
    k_tile_sums<<<dp.n_inst, 32, 0, st>>>(dp, dp.tv_partial, 2, delta);
    return cudaGetLastError();
}

cudaError_t launch_count_samples(const DevPlan& dp, int inst_idx, int n_det, unsigned long long* out, cudaStream_t st)
{
    k_count_samples<<<n_det, 128, 0, st>>>(dp, inst_idx, out);
    return cudaGetLastError();
}

} // namespace patgpu

namespace patgpu {

int circmean_blocks_per_sm(int m_lanes, bool bf16, int smem_bytes)
{
    const void* fn = nullptr;
    if (bf16) {
        fn = m_lanes == 16 ? (const void*)k_circmean<16, __nv_bfloat16>
           : m_lanes == 8  ? (const void*)k_circmean<8, __nv_bfloat16>
                           : (const void*)k_circmean<32, __nv_bfloat16>;
    } else {
        fn = m_lanes == 16 ? (const void*)k_circmean<16, float>
           : m_lanes == 8  ? (const void*)k_circmean<8, float>
                           : (const void*)k_circmean<32, float>;
    }
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

} // namespace patgpu
