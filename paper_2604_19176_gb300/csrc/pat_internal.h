// pat_internal.h — internal descriptors shared by the host plan builder and
// the device kernels of the photoacoustic operator library.
//
// Coordinates.  All kernels work in "centred pixel units": for an N x N image
// with h = 2/N and c0 = N/2, the world point (x, y) has coordinates
//     ubar = x / h - 1/2,   vbar = y / h - 1/2,
// so pixel (iy, ix) sits at (ix - c0, iy - c0) and cell (i0, j0) (the unit
// square whose lower-left corner is pixel (i0, j0)) is
// [i0 - c0, i0 - c0 + 1) x [j0 - c0, j0 - c0 + 1).  Centring halves the
// magnitude of the coordinates and so halves their FP32 rounding error.
//
// A sample of the circular mean about detector j at radius index m and angle
// index q is
//     ubar = fma(rho_m, cos_q, U_j),   vbar = fma(rho_m, sin_q, V_j),
// with rho_m = float(m) * delta, (cos_q, sin_q) and (U_j, V_j) read from the
// plan's FP32 tables.  The forward gather and the adjoint gather evaluate
// exactly this expression (explicit __fmaf_rn, no contraction freedom), so
// both kernels see every sample in the same cell with the same bilinear
// weights: the adjoint is the transpose of the forward matrix.
#pragma once

#include <cstddef>
#include <cstdint>

namespace patgpu {

constexpr int kWarp = 32;
constexpr int kColOff = 4;        // FP32 shared image: column 0 at word offset 4 (16 B aligned)
constexpr int kColOffBF16 = 8;    // BF16 shared image: column 0 at element offset 8 (16 B aligned)
constexpr int kAdjTile = 16;      // adjoint CTA: 16 x 16 cells -> 15 x 15 output pixels
constexpr int kAdjOut = kAdjTile - 1;

// Per-instance descriptor (device resident, read by every kernel).
struct InstDev {
    int32_t n, n_det, n_t, n_r;
    int32_t K, c0, det_off, trig_off;
    float delta, inv_delta, dphi, inv_dphi;
    float inv_K, pad0;
    int32_t n_slots, nmb;          // forward partial slots; radius blocks per detector
    int64_t f_off, g_off;          // element offsets of the instance's image / data
    int64_t mpart_off;             // float offset of forward partial slots (n_slots x n_det x n_r)
    int64_t mbar_off;              // float offset of the adjoint's Mbar (n_det x n_r)
    int64_t p_off;                 // float offset of the Abel matrix (n_t x n_r)
    int64_t slotcnt_off;           // byte offset of the slot counts (n_det x nmb)
};

// Circular-mean work unit: radii [m0, m0 + m_lanes) of detector j, angles
// q0 .. q0 + nq - 1 (mod K), restricted to one image band; its partial sums
// go to forward slot `slot`.
struct Unit {
    int32_t j, m0, q0, nq, slot, pad;
};

// A contiguous range of units of one (instance, band), processed by one CTA
// after it has staged that band of the image in shared memory.
struct Segment {
    int32_t inst;
    int32_t band_lo;   // first cell row of the band (absolute, may be -1)
    int32_t band_hi;   // one past the last cell row (absolute, <= N)
    int32_t unit_begin, unit_end;
    int32_t pad[3];
};

// Output tile of the two Abel (time) stages.
struct TimeTile {
    int32_t inst, j0, x0, pad;     // x0: first time index (forward) or radius index (adjoint)
};

// Output tile of the adjoint gather: 16 x 16 cells whose lower-left cell is
// (x0 - 1, y0 - 1); produces pixels [x0, x0 + 15) x [y0, y0 + 15).
struct AdjTile {
    int32_t inst, x0, y0, pad;
};

// Tile of the elementwise / stencil kernels (TV).
struct ImgTile {
    int32_t inst, x0, y0, pad;
};

// Everything a kernel launch needs, by value (fits the 4 KB parameter space).
struct DevPlan {
    const InstDev* inst;
    const float* detU;             // U_j (centred pixel units), concatenated per instance
    const float* detV;
    const float2* trig;            // (cos, sin)(2 pi q / K), concatenated per distinct K
    const float* P;                // Abel matrices, concatenated per distinct n_t
    const uint8_t* slotcnt;        // forward slots per (detector, radius block)
    const Unit* units;
    const Segment* segs;
    const int32_t* cta_seg;        // CTA c processes segments [cta_seg[c], cta_seg[c+1])
    const TimeTile* fwd_tiles;
    const TimeTile* adj_tiles;
    const AdjTile* gather_tiles;
    const ImgTile* img_tiles;
    float* mpart;                  // forward partial slots
    float* mbar;                   // adjoint Mbar
    float* tv_partial;             // per image tile TV partial sums
    int32_t* status;               // device status word (bounded waits)
    int32_t n_inst;
    int32_t n_fwd_ctas, n_fwd_tiles, n_adj_tiles, n_gather_tiles, n_img_tiles;
    int32_t m_lanes, adj_groups;
    int32_t smem_pitch_max;        // unused by kernels; for diagnostics
    int32_t fwd_smem_bytes;        // dynamic shared memory of the circular-mean kernel
    int32_t bf16;                  // image storage is BF16
    int32_t tv_tiles_per_inst_max;
};

// Shared-memory row pitch (elements) of a band of an N-wide image.  The
// pitch leaves a zero column on each side, keeps rows 16-byte aligned, and is
// congruent to 12 (FP32 words) mod 32 so that the 2 x 2 texel reads of 32
// lanes walking along a ray spread over the 32 banks.
inline int band_pitch_f32(int n)
{
    int w = n + kColOff + 1;
    while (w % 32 != 12) ++w;
    return w;
}
inline int band_pitch_bf16(int n)
{
    int w = n + kColOffBF16 + 1;   // elements; words = w / 2
    while (w % 64 != 24) ++w;
    return w;
}

} // namespace patgpu
