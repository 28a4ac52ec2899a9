// misc.cu — TV value/gradient, data residual and projected descent step.
//
// TV(f) = sum_{i,j} sqrt(dx^2 + dy^2 + eps^2) with forward differences
// (zero on the last column / row): the regulariser of Eq. (4) and Eq. (5).
// The descent step applies the projection onto f >= 0 of Eq. (4).
#include "device_common.cuh"
#include "kernels.h"

namespace patgpu {

namespace {
__device__ __forceinline__ float tv_term(const float* f, int n, int i, int j, float eps2, float& dx, float& dy)
{
    const float c = f[(size_t)i * n + j];
    dx = (j + 1 < n) ? f[(size_t)i * n + j + 1] - c : 0.f;
    dy = (i + 1 < n) ? f[(size_t)(i + 1) * n + j] - c : 0.f;
    return sqrtf(fmaf(dx, dx, fmaf(dy, dy, eps2)));
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

// Per-instance sums of per-tile partials (fixed order): out[i*ncomp + c].
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

// Fused last stage of one projected-gradient TV iteration (Eq. (4)): the
// adjoint value of each pixel from its four cells' corner sums (as
// k_adj_combine), the TV gradient (as k_tv) and the projected update, written
// to a second buffer because the stencil reads the neighbours' old values.
__global__ void __launch_bounds__(256) k_tv_update(DevPlan dp, const float* __restrict__ f, float* __restrict__ fout,
                                                   float tau, float lam, float eps, int nonneg,
                                                   float* __restrict__ part)
{
    __shared__ float red[8];
    const ImgTile t = dp.img_tiles[blockIdx.x];
    const InstDev in = dp.inst[t.inst];
    pdl_wait();   // the cell sums come from the previous kernel
    const int n = in.n;
    const float* fi = f + in.f_off;
    const int j = t.x0 + (threadIdx.x & 31), i = t.y0 + (threadIdx.x >> 5);
    float d2 = 0.f, n2 = 0.f;
    if (i < n && j < n) {
        // A^T r at pixel (j, i): corner sums of cells (j,i), (j-1,i), (j,i-1), (j-1,i-1)
        const int w = n + 1;
        const float4* z = dp.zbuf + in.z_off;
        const float s = corner_sum(z, (size_t)w * w, dp.adj_groups, (size_t)(i + 1) * w + j + 1,
                                   (size_t)(i + 1) * w + j, (size_t)i * w + j + 1, (size_t)i * w + j);
        const float adj = s * in.inv_K;
        const float eps2 = eps * eps;
        float dx, dy;
        const float st = tv_term(fi, n, i, j, eps2, dx, dy);
        float gtv = -(dx + dy) / st;
        if (j > 0) {
            float dxl, dyl;
            const float sl = tv_term(fi, n, i, j - 1, eps2, dxl, dyl);
            gtv += dxl / sl;
        }
        if (i > 0) {
            float dxu, dyu;
            const float su = tv_term(fi, n, i - 1, j, eps2, dxu, dyu);
            gtv += dyu / su;
        }
        const float old = fi[(size_t)i * n + j];
        float nv = fmaf(-tau, fmaf(lam, gtv, adj), old);
        if (nonneg) nv = fmaxf(nv, 0.f);
        fout[in.f_off + (size_t)i * n + j] = nv;
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

// Primal-dual (Chambolle-Pock) TV iteration for Eq. (4), written as
// min_f F(K f) + G(f) with K f = (A f, grad f), F(z, q) = 1/2 ||z - g||^2 +
// alpha sum_i |q_i| and G the indicator of f >= 0.  The dual variable of the
// TV term is p = (px, py), one 2-vector per pixel, stored as two image-shaped
// planes.  grad is the forward difference of k_tv (zero on the last column /
// row) and grad^T its exact transpose.
//
// Dual step of the TV term: p <- projection onto |p_i| <= alpha of
// p + sigma grad fbar, pixel by pixel, in place.
__global__ void __launch_bounds__(256) k_pdhg_dual_tv(DevPlan dp, const float* __restrict__ fbar,
                                                      float* __restrict__ px, float* __restrict__ py, float sigma,
                                                      float alpha)
{
    const ImgTile t = dp.img_tiles[blockIdx.x];
    const InstDev in = dp.inst[t.inst];
    pdl_wait();   // fbar and p come from the previous iteration
    const int n = in.n;
    const int j = t.x0 + (threadIdx.x & 31), i = t.y0 + (threadIdx.x >> 5);
    if (i >= n || j >= n) return;
    const float* fi = fbar + in.f_off;
    const size_t idx = in.f_off + (size_t)i * n + j;
    const float c = fi[(size_t)i * n + j];
    const float dx = (j + 1 < n) ? fi[(size_t)i * n + j + 1] - c : 0.f;
    const float dy = (i + 1 < n) ? fi[(size_t)(i + 1) * n + j] - c : 0.f;
    const float qx = fmaf(sigma, dx, px[idx]);
    const float qy = fmaf(sigma, dy, py[idx]);
    const float mag = sqrtf(fmaf(qx, qx, qy * qy));
    const float s = mag > alpha ? alpha / mag : 1.f;
    px[idx] = qx * s;
    py[idx] = qy * s;
}

// Primal step and extrapolation, in place:
//   f_new = max(0, f - tau (A^T y + grad^T p + grad h(f))),  fbar = 2 f_new - f,  f = f_new
// with A^T y from the four cells' corner sums (as k_adj_combine), and the
// per-tile sums of |f_new - f|^2, |f_new|^2 and f_new for the relative-change
// rule and the instance mean.  h(f) = beta/2 (mean(f) - c)^2 is the optional
// mean-intensity penalty (beta != 0; fmean then holds the mean of f per
// instance), an explicit gradient term beta (mean(f) - c) / P on every pixel.
__global__ void __launch_bounds__(256) k_pdhg_primal(DevPlan dp, float* __restrict__ f, float* __restrict__ fbar,
                                                     const float* __restrict__ px, const float* __restrict__ py,
                                                     float tau, int nonneg, const float* __restrict__ fmean,
                                                     float beta, float mean_target, float* __restrict__ part)
{
    __shared__ float red[8];
    const ImgTile t = dp.img_tiles[blockIdx.x];
    const InstDev in = dp.inst[t.inst];
    pdl_wait();   // the cell sums come from the previous kernel
    const int n = in.n;
    const int j = t.x0 + (threadIdx.x & 31), i = t.y0 + (threadIdx.x >> 5);
    float d2 = 0.f, n2 = 0.f, s1 = 0.f;
    if (i < n && j < n) {
        const int w = n + 1;
        const float4* z = dp.zbuf + in.z_off;
        const float s = corner_sum(z, (size_t)w * w, dp.adj_groups, (size_t)(i + 1) * w + j + 1,
                                   (size_t)(i + 1) * w + j, (size_t)i * w + j + 1, (size_t)i * w + j);
        const size_t idx = in.f_off + (size_t)i * n + j;
        // grad^T p: the differences that pixel (j, i) enters with +1 (from the
        // left / upper neighbour) and -1 (its own, unless on the last column / row)
        float div = 0.f;
        if (j > 0) div += px[idx - 1];
        if (j + 1 < n) div -= px[idx];
        if (i > 0) div += py[idx - n];
        if (i + 1 < n) div -= py[idx];
        if (beta != 0.f) div += beta * (fmean[t.inst] - mean_target) / ((float)n * (float)n);
        const float old = f[idx];
        float nv = fmaf(-tau, fmaf(s, in.inv_K, div), old);
        if (nonneg) nv = fmaxf(nv, 0.f);
        f[idx] = nv;
        fbar[idx] = fmaf(2.f, nv, -old);
        d2 = (nv - old) * (nv - old);
        n2 = nv * nv;
        s1 = nv;
    }
    if (part) {
        const float a = block_sum<256>(d2, red);
        const float b = block_sum<256>(n2, red);
        const float c = block_sum<256>(s1, red);
        if (threadIdx.x == 0) {
            part[3 * blockIdx.x] = a;
            part[3 * blockIdx.x + 1] = b;
            part[3 * blockIdx.x + 2] = c;
        }
    }
}

// Per-instance sums of k_pdhg_primal's partials (fixed order): delta[2i],
// delta[2i+1] = |f_new - f|^2, |f_new|^2 and fmean[i] = mean of f_new (each nullable).
__global__ void k_pdhg_sums(DevPlan dp, const float* __restrict__ part, float* __restrict__ delta,
                            float* __restrict__ fmean)
{
    const int inst = blockIdx.x, c = threadIdx.x;
    if (c >= 3) return;
    float s = 0.f;
    for (int b = 0; b < dp.n_img_tiles; ++b)
        if (dp.img_tiles[b].inst == inst) s += part[(size_t)b * 3 + c];
    if (c < 2) {
        if (delta) delta[2 * inst + c] = s;
    } else if (fmean) {
        const int n = dp.inst[inst].n;
        fmean[inst] = s / ((float)n * (float)n);
    }
}

cudaError_t launch_pdhg_dual_tv(const DevPlan& dp, const float* fbar, float* px, float* py, float sigma, float alpha,
                                cudaStream_t st)
{
    if (dp.n_img_tiles == 0) return cudaSuccess;
    return launch_pdl(k_pdhg_dual_tv, dim3(dp.n_img_tiles), dim3(256), 0, st, 1, dp, fbar, px, py, sigma, alpha);
}

cudaError_t launch_pdhg_primal(const DevPlan& dp, float* f, float* fbar, const float* px, const float* py, float tau,
                               int nonneg, float* fmean, float beta, float mean_target, float* delta, cudaStream_t st)
{
    if (dp.n_img_tiles == 0) return cudaSuccess;
    const bool sums = delta || fmean;
    cudaError_t e = launch_pdl(k_pdhg_primal, dim3(dp.n_img_tiles), dim3(256), 0, st, 1, dp, f, fbar, px, py, tau,
                               nonneg, (const float*)fmean, beta, mean_target, sums ? dp.tv_partial : nullptr);
    if (e != cudaSuccess || !sums) return e;
    k_pdhg_sums<<<dp.n_inst, 32, 0, st>>>(dp, dp.tv_partial, delta, fmean);
    return cudaGetLastError();
}

cudaError_t launch_tv_update(const DevPlan& dp, const float* f_in, float* f_out, float tau, float lam, float eps,
                             int nonneg, float* delta, cudaStream_t st)
{
    if (dp.n_img_tiles == 0) return cudaSuccess;
    cudaError_t e = launch_pdl(k_tv_update, dim3(dp.n_img_tiles), dim3(256), 0, st, 1, dp, f_in, f_out, tau, lam,
                               eps, nonneg, delta ? dp.tv_partial : nullptr);
    if (e != cudaSuccess || !delta) return e;
    k_tile_sums<<<dp.n_inst, 32, 0, st>>>(dp, dp.tv_partial, 2, delta);
    return cudaGetLastError();
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

} // namespace patgpu
