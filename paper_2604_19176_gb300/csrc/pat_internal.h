// pat_internal.h — internal descriptors shared by the host plan builder and
// the device kernels of the photoacoustic operator library.
//
// Coordinates.  All kernels work in "centred pixel units": for an N x N image
// with h = 2/N and c0 = N/2, the world point (x, y) has coordinates
//     ubar = x / h - 1/2,   vbar = y / h - 1/2,
// so pixel (iy, ix) sits at (ix - c0, iy - c0) and cell (i0, j0) (the unit
// square whose lower-left corner is pixel (i0, j0)) is
// [i0 - c0, i0 - c0 + 1) x [j0 - c0, j0 - c0 + 1).  Centring halves the
// magnitude of the coordinates.
//
// A sample of the circular mean about detector j at radius index m and angle
// index q sits at (U_j + m dcos_q, V_j + m dsin_q), dcos_q = delta cos(2 pi q/K).
// FP32 cannot hold that point to better than half an ulp of |ubar| (up to
// N/2), which at N >= 384 alone costs ~1e-5 of relative error in A and A^T.
// The kernels therefore work in split form:
//   * detector: U = float(U_j), Ui = floor(U), Uf = float(U_j - Ui);
//   * direction: dcos_q = hi + lo (two FP32 numbers, from FP64);
//   * cell (relative to Ui):  cu = floor(fma(m, hi, Uf));
//   * fraction in the cell:   a  = fma(m, hi, -cu) + fma(m, lo, Uf),
// and the same for v.  m * hi is exact inside the FMA and the rounded
// results are below 2 in magnitude, so a is within ~3 * 2^-25 of the exact
// fraction at any N (the cell decision itself may differ from the exact one
// only for samples within ~N * 2^-24 of a grid line, where both cells give
// the same interpolated value to that order).  The forward gather and the
// adjoint gather evaluate exactly these expressions (explicit __fmaf_rn /
// __fadd_rn, no contraction freedom), so both kernels see every sample in
// the same cell with the same bilinear weights: the adjoint is the transpose
// of the forward matrix.
#pragma once

#include <cstddef>
#include <cstdint>

namespace patgpu {

constexpr int kWarp = 32;
constexpr int kPatchW = 8;        // adjoint: one warp owns an 8 x 4 patch of cells
constexpr int kPatchH = 4;
// Work queues live kQueueStride ints apart (one 128-byte line each, so that
// queues taken by different CTAs do not serialise on one L2 line): queue 0 is
// the adjoint cell kernel's (the list kernel's schedule is static).  Each
// queue is two ints: the next item and the count of finished participants.
constexpr int kQueueStride = 32;

// Per-instance descriptor (device resident, read by every kernel).
struct InstDev {
    int32_t n, n_det, n_t, n_r;
    int32_t K, c0, det_off, pad1;
    float delta, inv_delta, dphi, inv_dphi;
    float inv_K, pad0;
    int32_t n_slots, nmb;          // forward partial slots; radius blocks per detector
    int64_t f_off, g_off;          // element offsets of the instance's image / data
    int64_t mpart_off;             // float offset of forward partial slots (n_slots x n_det x n_r)
    int64_t mbar_off;              // float offset of M and of Mbar (n_det rows of pitch m_pitch)
    int64_t p_off;                 // float offset of P (n_t rows, pitch n_rp), then P^T (n_r rows, pitch n_tp),
                                   //   then both in 32 x 32 blocks (the fused time stage)
    int64_t slotcnt_off;           // byte offset of the slot counts (n_det x nmb int32)
    int64_t z_off;                 // float4 offset of the adjoint cell sums (groups x (n+1)^2)
    int64_t ray_off;               // entry offset of the instance's 2K rays and reciprocal rays
    int64_t list_off;              // adjoint lists: offset of the instance's (n+1)^2 cell counts
    int64_t pbase_off;             // adjoint lists: offset of the instance's (patch, part) block bases
    int32_t code_jbits, code_mbits; // adjoint list mode: code = q << (jb+mb) | j << mb | m
    int32_t n_rp;                  // row pitch (multiple of 32) of P
    int32_t n_tp;                  // row pitch (multiple of 32) of P^T
    int32_t m_pitch;               // row pitch of M and Mbar: a power of two > n_r (the columns from
                                   //   n_r on stay zero), so a list code's low bits are j * m_pitch + m
    int32_t patches_x;             // adjoint lists: 8 x 4 cell patches per row of cells
};

// Circular-mean work unit: radii [m0, m0 + m_lanes) of detector j, angles
// q0 .. q0 + nq - 1 (never past K), restricted to one tile; its partial sums
// go to forward slot `slot` (the slots of a (detector, radius block) are
// added in slot order by k_msum).  32 bytes.
struct Unit {
    int32_t j, m0, q0, nq, slot, pad[3];
};

// Tile task of the circular means: the pixels [x0, x1) x [y0, y1) of one
// instance (tiles partition every image), processed by one CTA.  The staged
// cells are [x0 - 2, x1] x [y0 - 2, y1] (cell (c, r) spans pixels c..c+1,
// r..r+1; pixels outside the tile count as zero), `pitch` cells per row.
// Warp w of the CTA processes units[warp_units[warp_off + w] ..
// warp_units[warp_off + w + 1]) (a static schedule, balanced at plan time).
struct Segment {
    int32_t inst;
    int32_t x0, x1;    // owned pixel columns
    int32_t y0, y1;    // owned pixel rows
    int32_t pitch;     // staged cells per row (>= x1 - x0 + 3)
    int32_t warp_off;  // index of this task's first per-warp offset
    int32_t pad[5];
};

// Output tile of the two Abel (time) stages: detectors [j0, j0 + kAbelJ),
// outputs [x0, x0 + kAbelX) (times for the forward, radii for the adjoint).
struct TimeTile {
    int32_t inst, j0, x0, pad;
};

// Group of the fused time stage (k_time_pair): detectors [j0, j0 + jn) of
// instance inst, jn <= kTimeJ, processed by one cluster of kTimeCS CTAs.
struct TimeGroup {
    int32_t inst, j0, jn, pad;
};
constexpr int kTimeJ = 4;          // detectors per fused time group
constexpr int kTimeCS = 8;         // CTAs per cluster of the fused time stage
constexpr int kTimeWarps = 8;      // warps per fused time CTA

// Adjoint cell item of instance inst: the 8 x 4 patch of cells with
// lower-left cell (x0, y0) (absolute indices, >= -1); in enumeration mode for
// detectors j = group (mod G), in list mode part `group` of the cells' lists.
struct CellItem {
    int32_t inst, x0, y0, group;
};

// Adjoint lists.  Cells are numbered (cy + 1) * (n + 1) + cx + 1; one warp
// item is (8 x 4 patch of cells, part), lane = cell, and every list is kept
// in 16-byte vectors of four entries, the 32 cells' vectors interleaved:
// vector k of the cell in lane l at slot base + k * 32 + l (code lists), or
// base + (3 k + s) * 32 + l for fraction lists (s = 0: Mbar indices, 1: a,
// 2: b).  list_base gives the first slot of each (patch, part) block, and one
// more entry after the last block (the kernel reads bases and lengths from
// its ListItem records).
//   Code lists (adj_mode 1, 4): a patch's entries are aligned by detector
// blocks of jblock detectors: the entries of block b (in the order (j, q, m))
// of every cell of the patch start at the same position, the block's
// segment as long as the patch's longest, shorter cells padded with null
// entries (weight index of the always-zero column m_pitch - 1 of row 0), so
// that the 32 lanes of a warp read the detector, ray and Mbar entries of at
// most jblock detectors at a time.  The patch's sequence (padded to whole
// vectors) is split into G parts of consecutive vectors, the same for every
// lane: a block holds (its length in vectors) x 32 slots.  An entry is
// q << (jb + mb) | j << mb | m (one sample) or, in run-pair lists (adj_mode
// 4), the same with bit 31 set for two samples of one ray at radii m, m + 1.
//   Fraction lists (adj_mode 3): cell c has count[c] samples in the order
// (j, q, m), in vectors padded at the end with null entries, each cell's
// vectors split into G parts (part g holds vectors [g nv / G, (g + 1) nv / G)
// of a cell with nv vectors); a block is as long as the patch's longest part.

// Item of the list gather: part `group` of the 8 x 4 patch with lower-left
// cell (x0, y0) of instance inst, whose block starts at 16-byte slot `base`
// and holds nk vectors per lane (code lists; the longest lane's for
// fraction lists).  Items are assigned to warps at plan time (LPT by nk);
// warp w runs warp_items[w] .. warp_items[w + 1] - 1.  32 bytes.
struct ListItem {
    int64_t base;
    int32_t nk, inst, group, x0, y0, pad;
};

// Tile of the elementwise / stencil kernels: 32 x 8 pixels.
struct ImgTile {
    int32_t inst, x0, y0, pad;
};

// Device status word values: small positive codes are bounded waits that
// gave up; kBoundsFlag | site is a failed bounds check of a debug build.
constexpr int32_t kBoundsFlag = 0x100;

// Everything a kernel launch needs, by value (fits the 4 KB parameter space).
struct DevPlan {
    const InstDev* inst;
    const float4* det;             // (Ui, Vi, Uf, Vf) of each detector (split form), per instance
    const float4* rays;            // (dcos hi, dsin hi, dcos lo, dsin lo) per q, 2K entries per instance
    const float2* rtrig;           // (1/dcos hi, 1/dsin hi), 2K entries per instance
    const float* P;                // Abel matrices P then P^T, per distinct n_t
    const uint8_t* slotcnt;        // forward slots per (detector, radius block), int32
    const Unit* units;             // circular-mean units, grouped by (tile task, warp)
    const int32_t* warp_units;     // per (tile task, warp): first unit (see Segment)
    const Segment* segs;
    const int32_t* cta_seg;        // CTA c processes segments [cta_seg[c], cta_seg[c+1])
    const int2* msum_rows;         // (instance, detector) of every row of M, for k_msum
    const TimeTile* fwd_tiles;
    const TimeTile* adj_tiles;
    const CellItem* cell_items;
    const ImgTile* img_tiles;
    const TimeGroup* time_groups;  // fused time stage groups, most work first
    const int64_t* list_base;      // adjoint lists: first 16-byte slot of each (patch, part) block
    const int32_t* cell_cnt;       // adjoint fraction lists: samples of each cell
    const uint32_t* codes;         // adjoint lists: the blocks (codes, or indices and fractions)
    const ListItem* list_items;    // adjoint list mode: (patch, part) items, grouped by warp
    const int32_t* warp_items;     // adjoint list mode: first item of each warp (+ end)
    float* mpart;                  // forward partial slots
    float* msum;                   // forward circular-mean sums M (same layout as Mbar)
    int32_t* work_counters;        // dynamic work queues, kQueueStride ints apart (see kQueueStride)
    float* mbar;                   // adjoint Mbar
    float4* zbuf;                  // adjoint per-group cell sums
    float* tv_partial;             // per image tile partial sums
    int32_t* status;               // device status word (bounded waits)
    int32_t n_inst;
    int32_t n_fwd_ctas, n_fwd_tiles, n_adj_tiles, n_cell_items, n_img_tiles, n_list_items;
    int32_t n_msum_rows;           // rows of M over all instances
    int32_t n_r_max;               // largest n_r of any instance
    int32_t m_lanes, adj_groups;
    int32_t adj_mode;              // 4 = run-pair code lists, 3 = fraction lists, 1 = code lists,
                                   //   0 = compute mode
    int32_t adj_jblock;            // code lists: detectors per aligned block
    int32_t cell_blocks;           // CTAs of the adjoint cell kernel (8 warps each)
    int32_t fwd_smem_bytes;        // dynamic shared memory of the circular-mean kernel
    int32_t fwd_rays_off;          // byte offset of the staged rays (after the largest tile)
    int32_t wait_probe;            // test hook: CTA 0 of the next circular-mean launch waits on a
                                   //   barrier nothing completes (bounded by wait_probe clocks)
    int32_t bounds_probe;          // test hook (debug builds): the next list gather plants one
                                   //   out-of-range detector index for its bounds check to report
    int64_t n_code_vecs;           // adjoint lists: 16-byte vectors in the codes buffer
    int32_t list_tail0;            // adjoint lists: list_items[list_tail0 ..] is the shared tail queue
    int32_t n_tail_items;          //   of small items (largest first), after the per-warp items
    int32_t abel_cluster_fwd;      // CTAs per cluster splitting each forward time contraction
    int32_t abel_cluster_adj;      // the same for the adjoint time contraction
    int32_t bf16;                  // image storage is BF16
    int32_t n_time_groups;
    int32_t time_chunks;           // fused time stage: most output chunks of a CTA in one phase; 0 = not used
    int32_t time_rows_r;           // largest n_rp: rows of M staged per fused time CTA
    int32_t time_rows_t;           // largest n_tp: rows of the residual staged per fused time CTA
    int32_t time_smem_bytes;       // dynamic shared memory of the fused time stage
};

constexpr int kAbelJ = 32;         // detectors per Abel tile (4 per warp)
constexpr int kAbelX = 32;         // outputs per Abel tile (one per lane)
constexpr int kAbelWarps = 8;      // warps per Abel CTA
constexpr int kAbelKC = 32;        // contraction rows staged per pipeline stage

// Staged cells per row of a circular-mean tile `w` pixels wide: w + 3 cells,
// padded to 5 mod 8.  A cell is 16 bytes (4 banks); eight lanes reading the
// cells along a 4-pixel stretch of a ray then fall into distinct bank groups
// except for offsets (+-3, -+1)-like pairs (v * pitch + u = 0 mod 8).
inline int cell_pitch(int w)
{
    int p = w + 3;
    while (p % 8 != 5) ++p;
    return p;
}

} // namespace patgpu
