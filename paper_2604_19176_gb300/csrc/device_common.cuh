// device_common.cuh — small device helpers shared by the kernels of this
// library (split-form sample coordinates, TMA bulk copies with mbarriers,
// bounded waits, reductions, the polynomial atan2 of the adjoint window).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pat_internal.h"

namespace patgpu {

__device__ __forceinline__ float ld_img(const float* p) { return *p; }
__device__ __forceinline__ float ld_img(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// ---------------------------------------------------------------------------
// Sample coordinates in split form (the coordinate conventions of
// pat_internal.h).  cell_rel: cell of radius index mf along direction
// component hi, relative to the detector's integer part, from the detector's
// fraction f0.  cell_frac: the sample's fraction inside that cell.  Both
// the forward and the adjoint gathers call exactly these.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float cell_rel(float mf, float hi, float f0)
{
    return floorf(__fmaf_rn(mf, hi, f0));
}
__device__ __forceinline__ float cell_frac(float mf, float hi, float lo, float f0, float cell)
{
    return __fadd_rn(__fmaf_rn(mf, hi, -cell), __fmaf_rn(mf, lo, f0));
}

// Floor of x (|x| < 2^22) by one directed-rounding add: x + 1.5 * 2^23
// rounded toward -inf is floor(x) + 1.5 * 2^23 exactly (the sum's ulp is 1),
// so the returned float's bit pattern is kMagicBits + floor(x) and
// floor(x) = result - kMagic.  The ordinary FP32 pipe does this; floorf and
// float->int conversions go through the slower conversion unit.
constexpr float kMagic = 12582912.0f;       // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;
__device__ __forceinline__ float floor_biased(float x) { return __fadd_rd(x, kMagic); }

// ---------------------------------------------------------------------------
// Paired FP32 arithmetic (Blackwell f32x2): two independent FP32 operations in
// one instruction on a 64-bit register pair; each half is rounded exactly as
// the scalar operation with the same rounding mode, so a paired evaluation of
// the u and v halves of the split form gives the bits of cell_rel/cell_frac.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_add_rd(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---------------------------------------------------------------------------
// Debug builds (-DPAT_DEBUG): device-side bounds checks.  dbg_ok(dp, ok, site)
// returns ok; when ok is false it records kBoundsFlag | site in the plan's
// status word (the first recorded error stays) and the caller skips the
// access, so a bad index is reported by pat_plan_sync_status as
// PAT_ERR_BOUNDS instead of trapping or faulting.  In release builds it is
// the constant true and costs nothing.
// ---------------------------------------------------------------------------
enum BoundsSite : int32_t {
    kSiteCircUnit = 1,     // circular-mean unit record (detector, angles, slot)
    kSiteCircCell = 2,     // circular-mean staged-cell offset of a sample
    kSiteCircRays = 3,     // circular-mean ray staging (shared-memory capacity)
    kSiteListItem = 4,     // adjoint list item (instance, code vectors)
    kSiteListEntry = 5,    // adjoint list entry (detector, ray, Mbar index)
    kSiteTimeRows = 6,     // fused time stage rows and slots
};
__device__ __forceinline__ bool dbg_ok(const DevPlan& dp, bool ok, int32_t site)
{
#ifdef PAT_DEBUG
    if (!ok && dp.status) atomicCAS(dp.status, 0, kBoundsFlag | site);
    return ok;
#else
    (void)dp;
    (void)site;
    return true;
#endif
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Kernels of the operator chain are launched
// with programmatic stream serialization, so the next kernel is launched as
// soon as this one's CTAs exit (its launch overlaps the end of this one);
// each kernel reads only the plan's immutable tables until pdl_wait, which
// returns once the previous kernel in the stream has completed and its
// memory is visible.  (Releasing dependents from the start of a kernel was
// measured slower: their waiting CTAs crowd the running kernel.)  A no-op
// without the launch attribute.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Adjoint value of one pixel before the 1/K: over the cell-sum parts, Z00 of
// its own cell, Z10 of the cell to its left, Z01 of the cell below and Z11 of
// the diagonal one (float4 offsets within a part plane of `plane` cells).
// The loads of four parts are in flight together; the additions keep part
// order (the result does not depend on the batching).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float corner_sum(const float4* __restrict__ z, size_t plane, int parts, size_t c_self,
                                            size_t c_left, size_t c_down, size_t c_diag)
{
    float s = 0.f;
    int g = 0;
    for (; g + 4 <= parts; g += 4) {
        float v[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4* zg = z + (size_t)(g + u) * plane;
            v[u][0] = __ldg(&zg[c_self].x);
            v[u][1] = __ldg(&zg[c_left].y);
            v[u][2] = __ldg(&zg[c_down].z);
            v[u][3] = __ldg(&zg[c_diag].w);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) s += v[u][0] + v[u][1] + v[u][2] + v[u][3];
    }
    for (; g < parts; ++g) {
        const float4* zg = z + (size_t)g * plane;
        s += __ldg(&zg[c_self].x) + __ldg(&zg[c_left].y) + __ldg(&zg[c_down].z) + __ldg(&zg[c_diag].w);
    }
    return s;
}

// ---------------------------------------------------------------------------
// TMA (bulk async copy) and mbarrier wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the barrier, giving up after ~limit_cycles SM
// clocks; on give-up records `code` in the device status word and returns
// false (the caller must then not use the data the barrier guards).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int32_t* status, int32_t code,
                                                  long long limit_cycles = 2000000000LL)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit_cycles) {
            if (status) atomicExch(status, code);
            return false;
        }
    }
    return true;
}

// Bulk prefetch of [src, src + bytes) into L2 (src 16-byte aligned, bytes a
// multiple of 16); no completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// 16-byte asynchronous global -> shared copy (L2 only), and its completion.
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// 4-byte asynchronous copy that writes zero when !valid (nothing is read then).
__device__ __forceinline__ void cp_async4_zfill(void* dst, const void* src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Angular window of the adjoint gather
// ---------------------------------------------------------------------------
constexpr float kPi = 3.14159265358979f;

// atan(x) on [0, 1]: odd polynomial x * p(x^2), coefficients fitted by
// iteratively reweighted least squares on 4000 Chebyshev nodes; evaluated in
// FP32 its max abs error is 1.7e-6 rad.  Only the adjoint's candidate window
// uses it (widened by a margin) and every candidate is re-checked exactly.
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

// Upper bound of asin(s), s in [0, 1]: s (1 + s^2/4) >= asin(s) for s <= 0.7.
__device__ __forceinline__ float asin_upper(float s)
{
    return s <= 0.7f ? s * fmaf(0.25f, s * s, 1.0f) : asinf(fminf(s, 1.0f)) + 1e-6f;
}

// ---------------------------------------------------------------------------
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

} // namespace patgpu
