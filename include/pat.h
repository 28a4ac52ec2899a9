/*
 * pat.h — C ABI of the GB300 (sm_103a) photoacoustic operator library.
 *
 * The library evaluates the discrete forward operator A of 2D photoacoustic
 * tomography in a circular (possibly limited-view) detection geometry and its
 * exact discrete adjoint A^T, plus the smoothed total-variation term used by
 * the variational and deep-image-prior reconstructions.
 *
 *   Model.  Eq. (1) (Sec. 2.1) is the wave initial-value problem with initial
 *   pressure f and zero initial velocity, observed on the detection curve by
 *   Eq. (2); Eq. (3) writes the measurement as g = A f + delta.  With c = 1
 *   the 2D Poisson formula gives
 *       p(y, t) = d/dt  int_0^t  r (M f)(y, r) / sqrt(t^2 - r^2)  dr,
 *   (M f)(y, r) the mean of f over the circle of radius r about detector y.
 *   Limited view (Sec. 2.1): only detectors on an arc are present.
 *
 *   Discretisation (the paper defers it to its fast operators; this library
 *   uses the following direct one):
 *     - image N x N on [-1,1]^2, h = 2/N, pixel (iy, ix) centred at
 *       (-1 + (ix+1/2) h, -1 + (iy+1/2) h), stored row-major f[iy*N + ix];
 *     - detector j at angle theta0 + (j + 1/2) Phi / n_det on the unit circle
 *       (cell-centred, matching the 256-on-270-degree array of Sec. 2.4.2);
 *     - Delta = T / n_t, times t_k = k Delta (k = 1..n_t), radii r_m = m Delta
 *       (m = 0..n_t+1);
 *     - circular mean by the K-node periodic trapezoid rule over bilinear
 *       samples of f (zero outside the grid);
 *     - Abel integral by exact product integration of the piecewise-linear
 *       mean, time derivative by the midpoint difference over +-Delta/2; the
 *       weights are built once per plan in FP64 and stored in FP32.
 *   Everything else runs in FP32 (optionally BF16 image storage, FP32 math).
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA device addresses on the device that was current
 *     when the plan was created, 16-byte aligned, owned by the caller.
 *   - Host pointers are ordinary host addresses owned by the caller.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued asynchronously on it; no call synchronises the host
 *     unless stated.
 *   - Arguments are validated before anything is enqueued; an invalid call
 *     returns an error status and enqueues nothing.  Errors reported by the
 *     CUDA runtime while enqueueing map to PAT_ERR_CUDA.  Nothing throws.
 *   - A plan holds one workspace: calls using the same plan must be ordered
 *     (same stream or explicit events).  Different plans are independent.
 *
 * Layout of a plan with n_instances instances (see pat_plan_layout):
 *   f (images):  instance i occupies N_i*N_i elements at f_offsets[i];
 *   g (data):    instance i occupies n_det_i*n_t_i FP32 at g_offsets[i],
 *                row j = detector, time fastest (g[j*n_t + (k-1)] = g(y_j, t_k)).
 *   With identical geometries the offsets are i*N*N and i*n_det*n_t.
 */
#ifndef PAT_H
#define PAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pat_plan* pat_plan_t;

typedef enum {
    PAT_OK = 0,
    PAT_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or geometry        */
    PAT_ERR_CUDA = 2,        /* CUDA runtime error while enqueueing / creating  */
    PAT_ERR_OOM = 3,         /* device or host allocation failed                */
    PAT_ERR_UNSUPPORTED = 4, /* valid request the library does not implement    */
    PAT_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up              */
    PAT_ERR_BAD_PLAN = 6,    /* NULL, destroyed or foreign plan handle          */
    PAT_ERR_BOUNDS = 7       /* a device-side bounds check failed (debug build) */
} pat_status_t;

typedef enum { PAT_F32 = 0, PAT_BF16 = 1 } pat_dtype_t;

/* Schedules for pat_forward / pat_adjoint.  Only PAT_SCHED_STAGED is built:
 * every stage is already one persistent (or tile-indexed) launch over all
 * instances of a plan, and a whole operator call can be captured in one CUDA
 * graph by the caller.  PAT_SCHED_PERSISTENT (a single fused launch per
 * operator) is reserved and returns PAT_ERR_UNSUPPORTED. */
typedef enum {
    PAT_SCHED_STAGED = 0,     /* one launch per stage (circular means, time, gather) */
    PAT_SCHED_PERSISTENT = 1  /* reserved                                            */
} pat_schedule_t;

/* One acquisition geometry (one instance). */
typedef struct {
    int32_t n;         /* image side N (N x N pixels); multiple of 4 (8 for BF16), 8..4096 */
    int32_t n_det;     /* detectors on the arc, 1..16384                                   */
    double arc_start;  /* theta0 in radians                                                */
    double arc_span;   /* Phi in radians, 0 < Phi <= 2 pi                                  */
    int32_t n_t;       /* time samples on (0, t_max], 1..16384                             */
    double t_max;      /* T > 0 (unit sound speed, unit detector radius)                   */
    int32_t n_angles;  /* K angular quadrature nodes per circular mean, 3..65536           */
} pat_geometry_t;

/* Plan options; zero-initialised options select the defaults. */
typedef struct {
    int32_t image_dtype; /* pat_dtype_t: storage of f in pat_forward / pat_adjoint           */
    int32_t schedule;    /* pat_schedule_t                                                   */
    int32_t tune;        /* 0 = tile fields below (0 = built-in), 1 = time candidate tile     */
                         /*     shapes at creation on these geometries (temporary device      */
                         /*     buffers, synchronises the stream; cached per process), 2 = 0  */
    int32_t m_lanes;     /* radii per warp in the circular-mean kernel (32, 16 or 8); 0=auto */
    int32_t q_piece;     /* max angular nodes per work unit (multiple of 4); 0 = auto        */
    int32_t band_rows;   /* max pixel rows of a circular-mean tile; 0 = auto                 */
    int32_t adj_groups;  /* detector groups of the adjoint gather, 1..16; 0 = auto           */
    int32_t adj_mode;    /* adjoint gather: 0 = auto (4 if it fits the list budget, else 1,   */
                         /*   else 3, else 2); 1 = per-cell sample code lists built at        */
                         /*   creation (device memory ~4 B per sample); 2 = enumerate on      */
                         /*   every call (no list memory); 3 = per-cell fraction lists built  */
                         /*   at creation (~12 B per sample: Mbar index and the FP32 bilinear */
                         /*   fractions); 4 = per-cell run-pair code lists (one 4 B code per  */
                         /*   pair of samples at consecutive radii of one ray, or per lone    */
                         /*   sample; needs one code bit more than 1)                         */
    int32_t abel_split;  /* CTAs (a thread-block cluster) sharing each time-stage tile: 1, 2, */
                         /*   4 or 8; 0 = auto (more when there are fewer tiles than SMs)     */
    int32_t tile_cols;   /* max pixel columns of a circular-mean tile; 0 = auto               */
    int32_t time_pair;   /* time stages of pat_tv_step / pat_pdhg_step: 0 = auto (one fused   */
                         /*   launch per step where its shared memory fits: n_t up to ~4400), */
                         /*   1 = separate launches (radius sums, forward, adjoint)          */
    int32_t adj_jblock;  /* code lists (adj_mode 1, 4): detectors per aligned block, 1..16384; */
                         /*   the 32 cells of a patch enter each block together (shorter      */
                         /*   lists wait on null entries) so that a warp's table loads share  */
                         /*   cache lines; 0 = auto                                           */
    int32_t reserved[4];
} pat_options_t;

/* Plan statistics (pat_plan_info). */
typedef struct {
    int32_t n_instances;
    int32_t device;          /* CUDA ordinal the plan is bound to                         */
    int64_t f_elems;         /* total image elements over all instances                   */
    int64_t g_elems;         /* total data elements over all instances                    */
    int64_t samples;         /* sum over instances of (j,m,q) samples touching the grid   */
    int64_t sample_slots;    /* samples the circular-mean kernel evaluates (incl. waste)  */
    int64_t time_macs;       /* multiply-adds of the two Abel stages per operator call    */
    int64_t work_units;      /* circular-mean work units                                  */
    int64_t device_bytes;    /* device memory held by the plan                            */
    int32_t m_lanes, q_piece, band_rows, adj_groups; /* tile shape in use              */
    int32_t bands_max;       /* largest number of circular-mean tiles of any instance     */
    int32_t adj_mode;        /* adjoint gather in use: 1 = code lists, 2 = enumeration,   */
                             /*   3 = fraction lists, 4 = run-pair code lists             */
    int64_t list_bytes;      /* device memory of the adjoint sample lists                 */
    int32_t abel_split_fwd;  /* CTAs per forward / adjoint time-stage tile in use         */
    int32_t abel_split_adj;
    int32_t tile_cols;       /* widest circular-mean tile (pixels); band_rows the tallest */
    int32_t time_pair;       /* 1 = the steps run the fused time stage, 0 = separate      */
    int32_t adj_jblock;      /* detectors per aligned block of the code lists (0: none)   */
    int32_t reserved;
} pat_plan_info_t;

/*
 * pat_plan_create — build the tables, weights and work lists for
 * n_instances geometries (Eq. (1)-(3), Sec. 2.1) on the current device.
 *   geoms:   host array of n_instances geometries (read only during the call).
 *   opt:     host pointer or NULL for defaults.
 *   stream:  used for the uploads (and autotuning); the call returns after
 *            the uploads completed.
 *   out:     receives the plan handle; unchanged on error.
 * The Abel weights are computed once per distinct n_t in FP64 and rounded to
 * FP32.  Errors: PAT_ERR_INVALID_ARG (geometry out of range, NULL out),
 * PAT_ERR_OOM, PAT_ERR_CUDA.
 */
pat_status_t pat_plan_create(const pat_geometry_t* geoms, int32_t n_instances,
                             const pat_options_t* opt, void* stream, pat_plan_t* out);

/* pat_plan_destroy — free a plan (after the work using it has completed).
 * NULL returns PAT_ERR_BAD_PLAN; a destroyed handle must not be reused. */
pat_status_t pat_plan_destroy(pat_plan_t plan);

/*
 * pat_plan_layout — element offsets of each instance in the packed f and g
 * buffers.  f_offsets and g_offsets are host arrays of n_instances + 1
 * entries (the last entry is the total); either may be NULL.
 */
pat_status_t pat_plan_layout(pat_plan_t plan, int64_t* f_offsets, int64_t* g_offsets);

/* pat_plan_info — statistics and the tile shape chosen (host struct). */
pat_status_t pat_plan_info(pat_plan_t plan, pat_plan_info_t* info);

/*
 * pat_forward — g = A f for every instance (Eq. (3) without noise).
 *   d_f: device, packed images in the plan's image dtype (FP32 or BF16).
 *   d_g: device, packed FP32 data, overwritten.
 * Errors: PAT_ERR_BAD_PLAN, PAT_ERR_INVALID_ARG (NULL / misaligned), PAT_ERR_CUDA.
 */
pat_status_t pat_forward(pat_plan_t plan, const void* d_f, float* d_g, void* stream);

/*
 * pat_adjoint — f = A^T g for every instance: the exact transpose of the
 * discrete A above, the operator whose application gives the data-term
 * gradient of Eq. (4) and Eq. (5) (Sec. 2.2).  Evaluated as a gather over
 * pixels (each output element is summed by one thread in a fixed order; no
 * atomics), so results are deterministic.
 *   d_g: device, packed FP32 data (read only).
 *   d_f: device, packed images in the plan's image dtype, overwritten.
 */
pat_status_t pat_adjoint(pat_plan_t plan, const float* d_g, void* d_f, void* stream);

/*
 * pat_tv_grad — value and gradient of the smoothed isotropic total variation
 *   TV(f) = sum_{i,j} sqrt(dx^2 + dy^2 + eps^2),
 *   dx = f[i][j+1]-f[i][j], dy = f[i+1][j]-f[i][j] (zero on the last
 *   column / row), the regulariser of Eq. (4) and Eq. (5).
 *   d_f:     device FP32 images (packed like pat_forward's input).
 *   eps:     smoothing, > 0.
 *   d_grad:  device FP32, overwritten with dTV/df (may be NULL); must not
 *            overlap d_f (the stencil reads neighbours other threads may
 *            already have written), else PAT_ERR_INVALID_ARG.
 *   d_value: device FP32 array of n_instances values (may be NULL; not both
 *            NULL); must not overlap d_f or d_grad.
 * FP32 plans only (PAT_ERR_UNSUPPORTED for BF16 plans).
 */
pat_status_t pat_tv_grad(pat_plan_t plan, const float* d_f, float eps, float* d_grad,
                         float* d_value, void* stream);

/*
 * pat_residual — d_r = scale * (d_Af - d_g) over all packed data elements
 * (the data-fit residual of Eq. (4); scale 2 gives the gradient factor of
 * the un-halved data term of Eq. (5)).  In-place use (d_r == d_Af) is allowed.
 */
pat_status_t pat_residual(pat_plan_t plan, const float* d_Af, const float* d_g, float* d_r,
                          float scale, void* stream);

/*
 * pat_descent_step — f <- f - tau * (d_adj + lam * d_tvgrad), then f <- max(f, 0)
 * when nonneg != 0 (the constraint f >= 0 of Eq. (4)); FP32 images.
 * d_tvgrad may be NULL (no TV term).  d_delta (nullable, device FP32, two
 * values per instance) receives ||f_new - f_old||^2 and ||f_new||^2 for the
 * relative-change stopping rule of Sec. 2.3.
 */
pat_status_t pat_descent_step(pat_plan_t plan, float* d_f, const float* d_adj,
                              const float* d_tvgrad, float tau, float lam, int32_t nonneg,
                              float* d_delta, void* stream);

/*
 * pat_tv_step — one projected-gradient iteration of the TV reconstruction of
 * Eq. (4), min_{f >= 0} 1/2 ||A f - g||^2 + lam TV_eps(f):
 *     r = A f_in - g;   f_out = max(0, f_in - tau (A^T r + lam grad TV_eps(f_in)))
 * (the max only when nonneg != 0).  Same arithmetic as pat_forward,
 * pat_residual, pat_adjoint, pat_tv_grad and pat_descent_step in sequence, in
 * fewer kernels: the adjoint's final pixel sums, the TV gradient and the
 * update share one kernel, and the time stages of A and A^T with the residual
 * between them are one launch (pat_options_t.time_pair = 0, where it fits;
 * it adds the contractions of the time stages in another order, so the result
 * matches the separate calls to FP32 rounding; with time_pair = 1 it is the
 * same bit for bit).  FP32 plans.
 *   d_f_in:  device FP32 images (read only).   d_f_out: device FP32 images,
 *            overwritten; must not alias d_f_in (the TV stencil reads the old
 *            neighbours).   d_g: device FP32 measured data (read only).
 *   d_delta: nullable, two values per instance as in pat_descent_step.
 */
pat_status_t pat_tv_step(pat_plan_t plan, const float* d_f_in, float* d_f_out, const float* d_g, float tau,
                         float lam, float eps, int32_t nonneg, float* d_delta, void* stream);

/*
 * pat_pdhg_step — one iteration of the primal-dual hybrid gradient method
 * (Chambolle-Pock) for the TV problem of Eq. (4),
 *     min_{f >= 0} 1/2 ||A f - g||^2 + alpha TV(f),
 * the paper's TV baseline solver (Sec. 2.1).  TV is the unsmoothed isotropic
 * total variation sum_i |grad f_i| with the forward differences of
 * pat_tv_grad.  With K f = (A f, grad f), dual variables y (data shaped) and
 * p = (px, py) (image shaped), one call performs, in this order:
 *     px, py <- each (px_i, py_i) + sigma grad fbar_i projected onto the disk of radius alpha
 *     y      <- (y + sigma (A fbar - g)) / (1 + sigma)
 *     f_new  <- f - tau (A^T y + grad^T p + beta (mean(f) - c) / P),
 *               then max(f_new, 0) when nonneg != 0
 *     fbar   <- 2 f_new - f;   f <- f_new
 * Convergence needs sigma tau ||K||^2 < 1 with ||K||^2 <= ||A||^2 + 8.
 * Start from f = fbar = y = px = py = 0 (or any warm start with fbar = f).
 * The beta term is the mouse-data variant of Sec. 2.1: with nonneg = 0 and
 * beta > 0 the objective gains the quadratic mean-intensity penalty
 * beta/2 (mean(f) - c)^2 (P pixels per instance), taken as an explicit
 * gradient step (primal-dual method with a smooth term; it also needs
 * 1/tau - sigma ||K||^2 >= beta / (2 P)).
 * FP32 plans only (PAT_ERR_UNSUPPORTED for BF16 plans).
 *   d_f, d_fbar, d_px, d_py: device FP32 images (packed like pat_forward's
 *            input), read and overwritten.
 *   d_y:     device FP32 data-shaped dual variable, read and overwritten.
 *   d_g:     device FP32 measured data (read only).
 *   All six buffers 16-byte aligned, owned by the caller and pairwise
 *   disjoint (PAT_ERR_INVALID_ARG otherwise).
 *   sigma, tau: dual and primal steps, > 0.   alpha: TV weight, >= 0.
 *   beta:    mean-penalty weight, >= 0 (0: no penalty).   mean_target: c.
 *   d_fmean: device FP32, one value per instance, disjoint from the others;
 *            read as the mean of f on entry, overwritten with the mean of
 *            f_new.  Required when beta > 0 (initialise it with the mean of
 *            the starting f), else nullable.
 *   d_delta: nullable, two values per instance as in pat_descent_step
 *            (||f_new - f||^2, ||f_new||^2), for the relative-change rule of
 *            Sec. 2.3.
 */
pat_status_t pat_pdhg_step(pat_plan_t plan, float* d_f, float* d_fbar, float* d_y, float* d_px, float* d_py,
                           const float* d_g, float sigma, float tau, float alpha, int32_t nonneg, float beta,
                           float mean_target, float* d_fmean, float* d_delta, void* stream);

/*
 * pat_plan_sync_status — synchronise the stream and report a device-side
 * error recorded by a bounded wait in a persistent launch (PAT_ERR_TIMEOUT)
 * or, in debug builds, by a failed bounds check (PAT_ERR_BOUNDS, see below),
 * clearing it.  Returns PAT_OK when none was recorded.
 * A launch whose wait gave up returns early: the results of that call are
 * undefined (some of its partial sums are missing), later calls are not
 * affected (the circular-mean kernel keeps no state across calls; its work is
 * scheduled statically).  The status word stays set until this call reports
 * and clears it (it also re-arms the adjoint kernels' work queues, which no
 * bounded wait can leave armed).
 */
pat_status_t pat_plan_sync_status(pat_plan_t plan, void* stream);

/*
 * pat_plan_set_wait_probe — test hook for the failure path above.  With
 * clocks > 0, the next circular-mean launch of this plan (pat_forward,
 * pat_tv_step, pat_pdhg_step) has its first CTA wait, bounded by `clocks`
 * SM clock cycles, on an mbarrier that nothing completes; the wait runs out,
 * records PAT_ERR_TIMEOUT in the device status word and that CTA returns
 * (no copy is in flight at that point, nothing faults).  The probe disarms
 * itself after that one launch.  clocks = 0 disarms it; negative clocks
 * return PAT_ERR_INVALID_ARG.  Synchronous with respect to the host only.
 */
pat_status_t pat_plan_set_wait_probe(pat_plan_t plan, int32_t clocks);

/*
 * Debug builds.  Compiling the library with -DPAT_DEBUG (build.py:
 * build(debug=True) makes libpatgpu_debug.so beside libpatgpu.so) adds
 * device-side bounds checks to the hot kernels: the circular means check each
 * work unit's detector, angle range and slot and each sample's staged-cell
 * offset, the ray staging checks its shared-memory capacity, the fused time
 * stage its staged rows and slot counts, and the list gather each item's code
 * range and each entry's detector, ray and Mbar index.  A failed check skips
 * the access, records the site in the plan's device status word (the first
 * error is kept) and the kernel carries on; it never traps.  The results of
 * that call are then undefined and pat_plan_sync_status reports
 * PAT_ERR_BOUNDS once, clearing the word.  Release builds compile the checks
 * out.  The checks serve where no device memory checker can be run.
 *
 * pat_debug_build — 1 when the library was compiled with -DPAT_DEBUG, else 0.
 *
 * pat_plan_set_bounds_probe — test hook for the checks above.  With enable
 * != 0, the next adjoint gather of this plan (pat_adjoint, pat_tv_step,
 * pat_pdhg_step) in code- or fraction-list form gives the first entry of its
 * first warp's first item a detector index (and Mbar index) past the
 * instance's detectors; everything that index would address still lies inside
 * the plan's allocations, so nothing faults even where a check were missing.
 * The entry check reports it and the entry is skipped.  The probe disarms
 * itself after that one launch.  Returns PAT_ERR_UNSUPPORTED in release
 * builds.  Synchronous with respect to the host only.
 */
int32_t pat_debug_build(void);
pat_status_t pat_plan_set_bounds_probe(pat_plan_t plan, int32_t enable);

/*
 * pat_debug_fail_alloc — test hook for the allocation-failure path of
 * pat_plan_create (any build).  After pat_debug_fail_alloc(n), the n-th next
 * device allocation made by plan creation or by the autotuner (n = 0: the
 * next one) fails as if the device were out of memory, once; the call that
 * made it then returns PAT_ERR_OOM (an autotuner candidate that fails is
 * skipped instead) after freeing every allocation it had made.  n < 0
 * disarms the hook.  Process-wide, for all devices; always returns PAT_OK.
 */
pat_status_t pat_debug_fail_alloc(int32_t n);

/*
 * Per-kernel timing (tracing).  When enabled, every kernel the plan enqueues
 * is bracketed by a pair of CUDA events recorded on the launch stream.
 * pat_plan_kernel_times synchronises those events, adds their elapsed times
 * per kernel kind into total_ms[kind] and launch counts into launches[kind]
 * (host arrays of n_kinds entries, either may be NULL) and forgets them.
 * Kinds (pat_kernel_kind_t order): circular means, Abel forward, Abel
 * adjoint, adjoint gather, TV, residual, descent step, fused TV update,
 * primal-dual TV dual step, primal-dual primal step, fused time stage of
 * the steps (radius sums + Abel forward + residual + Abel adjoint).
 */
typedef enum {
    PAT_K_CIRCMEAN = 0, PAT_K_ABEL_FWD = 1, PAT_K_ABEL_ADJ = 2, PAT_K_ADJ_GATHER = 3,
    PAT_K_TV = 4, PAT_K_RESIDUAL = 5, PAT_K_DESCENT = 6, PAT_K_TV_UPDATE = 7, PAT_K_PDHG_DUAL = 8,
    PAT_K_PDHG_PRIMAL = 9, PAT_K_TIME_PAIR = 10, PAT_K_COUNT = 11
} pat_kernel_kind_t;
pat_status_t pat_plan_set_timing(pat_plan_t plan, int32_t enable);
pat_status_t pat_plan_kernel_times(pat_plan_t plan, double* total_ms, int64_t* launches, int32_t n_kinds);

/*
 * pat_tv_grad_noalloc — the TV value and gradient of pat_tv_grad for a batch
 * of same-sized FP32 images, for callers that cannot allocate device memory.
 * It needs no plan (creating a plan allocates) and allocates nothing.  The
 * paper has no counterpart: this is a deployment variant of pat_tv_grad for
 * code that runs under another framework's allocator, inside a real-time loop
 * that must not call cudaMalloc after start-up, or anywhere allocation is not
 * permitted.
 *   d_f:     device FP32, batch images of n x n, row-major, packed (read only).
 *   n:       image side, 1..16384.        batch: number of images, >= 1.
 *   eps:     smoothing, > 0.
 *   d_grad:  device FP32, same layout as d_f, overwritten with dTV/df (may be
 *            NULL); must not overlap d_f (the stencil reads neighbours other
 *            threads may already have written), else PAT_ERR_INVALID_ARG.
 *   d_value: device FP32, batch values (may be NULL; not both NULL); must not
 *            overlap d_f or d_grad.
 *   Pointers 4-byte aligned, owned by the caller.
 * Scratch: the value (and only the value) needs one partial sum per 32 x 8
 * tile, kept in a fixed static device array of PAT_TV_NOALLOC_MAX_TILES
 * floats (256 KB).  With d_value set, batch * ceil(n/32) * ceil(n/8) must not
 * exceed PAT_TV_NOALLOC_MAX_TILES, else PAT_ERR_INVALID_ARG and nothing is
 * enqueued: n = 256 allows batch <= 256, n = 1024 batch <= 16, n = 4096 batch 1,
 * and no batch for n > 4096.  Gradient-only calls (d_value NULL) use no
 * scratch and take every n and batch.
 * The first call with d_value set on a device looks up the array's device
 * address (with that device current); make it before any stream capture.
 * All calls share the array, so calls that overlap on the GPU race; order them
 * on one stream.
 */
#define PAT_TV_NOALLOC_MAX_TILES 65536
pat_status_t pat_tv_grad_noalloc(const float* d_f, int32_t n, int32_t batch, float eps, float* d_grad,
                                 float* d_value, void* stream);

/* Human-readable name of a status code (static string). */
const char* pat_status_string(pat_status_t status);

#ifdef __cplusplus
}
#endif
#endif /* PAT_H */
