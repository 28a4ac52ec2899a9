// noalloc.cu — smoothed TV value and gradient for callers that cannot allocate.
//
// pat_tv_grad works through a plan, and creating a plan allocates device
// memory (tables and workspace).  Some callers cannot do that: code running
// under another framework's allocator that already owns the device memory,
// a real-time loop that must not call cudaMalloc after start-up, or a host
// callback / embedding where allocation is not permitted at all.  For them,
// pat_tv_grad_noalloc computes the same TV value and gradient with no plan
// and no allocation.  Its only scratch (one partial sum of the TV value per
// 32 x 8 tile) lives in the fixed-size static device array below, which every
// GPU that loads this library holds until the process exits.
//
// The device address of that array is looked up once per device, with that
// device current, on the first call made on the device; make that first call
// before any stream capture.  All calls share the array: calls whose work
// overlaps on the GPU (different streams, no ordering) race on it.  Every call
// writes each scratch entry it later reads, so nothing has to start at zero.
#include <climits>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "device_common.cuh"
#include "pat.h"

namespace patgpu {

namespace {

static __device__ __align__(256) float g_tv_scratch[PAT_TV_NOALLOC_MAX_TILES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
float* g_scratch_ptr[kMaxDevices] = {};

__device__ __forceinline__ float tv_term_na(const float* f, int n, int i, int j, float eps2, float& dx, float& dy)
{
    const float c = f[(size_t)i * n + j];
    dx = (j + 1 < n) ? f[(size_t)i * n + j + 1] - c : 0.f;
    dy = (i + 1 < n) ? f[(size_t)(i + 1) * n + j] - c : 0.f;
    return sqrtf(fmaf(dx, dx, fmaf(dy, dy, eps2)));
}

// One CTA per 32 x 8 tile of one image; tiles numbered image by image, row by row.
__global__ void __launch_bounds__(256) k_tv_noalloc(const float* __restrict__ f, int n, int tiles_x, int tiles_img,
                                                    float eps, float* __restrict__ grad, float* __restrict__ partial)
{
    __shared__ float red[8];
    const int img = blockIdx.x / tiles_img, t = blockIdx.x - img * tiles_img;
    const int x0 = (t % tiles_x) * 32, y0 = (t / tiles_x) * 8;
    const float* fi = f + (size_t)img * n * n;
    const int j = x0 + (threadIdx.x & 31), i = y0 + (threadIdx.x >> 5);
    const float eps2 = eps * eps;
    float val = 0.f;
    if (i < n && j < n) {
        float dx, dy;
        const float s = tv_term_na(fi, n, i, j, eps2, dx, dy);
        val = s;
        if (grad) {
            float gsum = -(dx + dy) / s;
            if (j > 0) {
                float dxl, dyl;
                const float sl = tv_term_na(fi, n, i, j - 1, eps2, dxl, dyl);
                gsum += dxl / sl;
            }
            if (i > 0) {
                float dxu, dyu;
                const float su = tv_term_na(fi, n, i - 1, j, eps2, dxu, dyu);
                gsum += dyu / su;
            }
            grad[(size_t)img * n * n + (size_t)i * n + j] = gsum;
        }
    }
    if (partial) {
        const float s = block_sum<256>(val, red);
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
    }
}

// value[img] = sum of the image's tile partials.  One warp per image: lane l
// adds tiles l, l + 32, l + 64, ... in order, then the 32 lane sums are added
// by a fixed shuffle tree, so the result is the same on every call.
__global__ void k_tv_noalloc_sum(const float* __restrict__ partial, int tiles_img, float* __restrict__ value)
{
    const float* p = partial + (size_t)blockIdx.x * tiles_img;
    float s = 0.f;
    for (int t = threadIdx.x; t < tiles_img; t += 32) s += p[t];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) value[blockIdx.x] = s;
}

// true when the byte ranges [a, a + na) and [b, b + nb) overlap
bool overlaps(const void* a, size_t na, const void* b, size_t nb)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

// Device address of g_tv_scratch on the current device, looked up once per device.
pat_status_t scratch_address(float** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return PAT_ERR_CUDA;
    if (dev >= kMaxDevices) return PAT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_tv_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PAT_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return PAT_OK;
}

} // namespace

} // namespace patgpu

extern "C" pat_status_t pat_tv_grad_noalloc(const float* d_f, int32_t n, int32_t batch, float eps, float* d_grad,
                                            float* d_value, void* stream)
{
    using namespace patgpu;
    if (!d_f || n < 1 || n > 16384 || batch < 1 || !(eps > 0.f) || !std::isfinite(eps)) return PAT_ERR_INVALID_ARG;
    if (!d_grad && !d_value) return PAT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_f) & 3u) || (reinterpret_cast<uintptr_t>(d_grad) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_value) & 3u))
        return PAT_ERR_INVALID_ARG;
    const int tiles_x = (n + 31) / 32, tiles_y = (n + 7) / 8;
    const int64_t tiles_img = (int64_t)tiles_x * tiles_y;
    const int64_t tiles = tiles_img * batch;
    if (tiles > INT32_MAX) return PAT_ERR_INVALID_ARG;
    // The stencil reads neighbours that other CTAs may already have written:
    // the gradient must not overlap the images, nor the values either of them.
    const size_t img_bytes = sizeof(float) * (size_t)n * (size_t)n * (size_t)batch;
    if (d_grad && overlaps(d_f, img_bytes, d_grad, img_bytes)) return PAT_ERR_INVALID_ARG;
    if (d_value) {
        const size_t vb = sizeof(float) * (size_t)batch;
        if (overlaps(d_f, img_bytes, d_value, vb) || (d_grad && overlaps(d_grad, img_bytes, d_value, vb)))
            return PAT_ERR_INVALID_ARG;
        if (tiles > PAT_TV_NOALLOC_MAX_TILES) return PAT_ERR_INVALID_ARG; // beyond the fixed scratch
    }
    float* scratch = nullptr;
    if (d_value) {
        const pat_status_t s = scratch_address(&scratch);
        if (s != PAT_OK) return s;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_tv_noalloc<<<(unsigned)tiles, 256, 0, st>>>(d_f, n, tiles_x, (int)tiles_img, eps, d_grad, scratch);
    if (cudaGetLastError() != cudaSuccess) return PAT_ERR_CUDA;
    if (d_value) {
        k_tv_noalloc_sum<<<batch, 32, 0, st>>>(scratch, (int)tiles_img, d_value);
        if (cudaGetLastError() != cudaSuccess) return PAT_ERR_CUDA;
    }
    return PAT_OK;
}
