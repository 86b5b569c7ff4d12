/*
 * kct.h -- C ABI of the cutting voxel projector (CVP) for NVIDIA B300 (sm_103a).
 *
 * Method: Kulvait & Rose, "Cutting Voxel Projector: a New Approach to Construct 3D Cone
 * Beam CT Operator", arXiv 2110.09841. The library computes the cone-beam CT operator
 * b = A x (Eq. fundament) and its exact adjoint x = A^T y for a float32 voxel volume and a
 * stack of flat-panel projections, one 3x4 projection matrix per view (Sec. III-C).
 *
 *   b[view, v, u] = F(u, v) * S(u, v),   S = sum_vox mu_vox * W(vox, pixel)   (Eq. cvpsu)
 *   x[vox]        = sum_view sum_pixel W(vox, pixel) * F(u, v) * y[view, v, u]
 *
 * W is the pair weight of the chosen variant:
 *   KCT_CVP_EXACT    W = |V_cut| / r^2, V_cut the intersection of the voxel with the pyramid
 *                    of all rays from the source to the pixel, r the distance from the source
 *                    to the centre of mass of V_cut (Eq. vox, Sec. II-E, centre-of-mass r);
 *   KCT_CVP_RELAXED  W = A_n * d / r_vox^2, A_n the area of the column cut of the voxel base,
 *                    d the x_3 length through the centre of mass of that cut projecting into
 *                    the pixel row, r_vox the distance to the voxel centre (Sec. III-A, Eq.
 *                    cutvolume, Eq. vox with voxel-centre r).
 * F is the pixel factor (Sec. III-C "second phase"):
 *   KCT_SCALE_COS    F = f^2 / (a cos^3 theta) at the pixel centre (Eq. cvp);
 *   KCT_SCALE_EXACT  F = 1 / abar, abar the solid angle of the pixel (Eq. cvpus).
 *
 * Conventions (Sec. II-A, II-B, III-A):
 *   - the volume box is centred at the origin; voxel (i, j, k) has its centre at
 *     ((i - (nx-1)/2) ax, (j - (ny-1)/2) ay, (k - (nz-1)/2) az) in mm;
 *   - pixel (u, v) is the unit square around detector index coordinates (u, v);
 *     the projection matrix maps homogeneous world points (mm) to (u, v, 1) up to scale;
 *   - geometry must follow the paper's arrangement: the detector column index u does not
 *     depend on x_3 (P[0][2] = P[2][2] = 0), the detector rows run along x_3 (pixels are
 *     rectangles: the horizontal part of P row 1 is parallel to that of P row 2), and the
 *     whole volume lies in front of the source.
 *
 * Memory layouts (all C-contiguous float32, device memory owned by the caller):
 *   volume       [nz][ny][nx]          (x_1 fastest)
 *   projections  [nviews][nv][nu]      (u fastest)
 *
 * Errors: every function returns a kct_status and never aborts the process. Invalid
 * arguments are rejected before any launch. Kernel launch failures return
 * KCT_ERR_CUDA; kct_last_error_message() gives a human-readable detail of the last
 * failure on the calling thread.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 * kct_project and kct_backproject enqueue work only: they allocate nothing, do not
 * synchronise and may be captured in a CUDA graph.
 *
 * Devices: a plan belongs to the device that was current when it was created. Every call
 * that takes a plan makes that device current while it runs and gives the calling thread
 * its previous current device back before returning; `stream` must belong to the plan's
 * device.
 */
#ifndef KCT_H
#define KCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KCT_VERSION 101

typedef enum kct_status {
    KCT_OK = 0,
    KCT_ERR_INVALID_ARG = 1,   /* null pointer, non-positive size, unknown enum value */
    KCT_ERR_GEOMETRY = 2,      /* projection matrices violate the required arrangement */
    KCT_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
    KCT_ERR_OOM = 4,           /* device or host allocation failed in kct_plan_create */
    KCT_ERR_DEVICE_CHECK = 5,  /* a kernel reported an inconsistent footprint */
    KCT_ERR_UNSUPPORTED = 6    /* request outside what the library supports */
} kct_status;

typedef enum kct_variant {
    KCT_CVP_EXACT = 0,         /* cut volume and centre of mass of each voxel-pixel pair */
    KCT_CVP_RELAXED = 1        /* column area times x_3 segment at the column centre of mass */
} kct_variant;

typedef enum kct_scaling {
    KCT_SCALE_COS = 0,         /* f^2 / (a cos^3 theta), Eq. cvp */
    KCT_SCALE_EXACT = 1        /* 1 / solid angle of the pixel, Eq. cvpus */
} kct_scaling;

typedef struct kct_volume_desc {
    int32_t nx, ny, nz;        /* voxels per edge (Sec. II-A: N_1, N_2, N_3) */
    double ax, ay, az;         /* voxel size in mm (a_1, a_2, a_3) */
} kct_volume_desc;

typedef struct kct_detector_desc {
    int32_t nu, nv;            /* pixels per row (u) and per column (v) */
    double pu, pv;             /* pixel pitch in mm (b_1, b_2); informational */
} kct_detector_desc;

typedef struct kct_plan kct_plan;

/*
 * Create a plan for one geometry on the current CUDA device.
 *   pmats   host pointer, float64 [nviews][3][4] row-major projection matrices mapping
 *           (x_1, x_2, x_3, 1) in mm to homogeneous detector index coordinates; copied.
 *   nviews  number of views, >= 1.
 * Validates the arrangement above (KCT_ERR_GEOMETRY otherwise), converts each view to the
 * kernel's FP32 parameters (source, principal direction, detector scales) and uploads them.
 * The plan owns that device memory (a few hundred bytes per view) until kct_plan_destroy.
 * Allocation failure returns KCT_ERR_OOM. On error *out is set to NULL. A plan may be used
 * from several streams at once: calls share only read-only state and the error word.
 */
kct_status kct_plan_create(kct_plan **out, const kct_volume_desc *vol, const kct_detector_desc *det,
                           const double *pmats, int32_t nviews, kct_variant variant,
                           kct_scaling scaling);

/* Release the plan and its device memory. Waits for nothing: the caller must make sure no
 * work that uses the plan is still pending. NULL is accepted. No counterpart in the paper
 * (resource management of this library). */
kct_status kct_plan_destroy(kct_plan *plan);

/*
 * Forward projection b = A x (Eq. cvpsu then the pixel factor).
 *   d_vol   device float32 [nz][ny][nx], read only.
 *   d_proj  device float32 [nviews][nv][nu]; overwritten (accumulate = 0) or added to
 *           (accumulate != 0). Must not overlap d_vol.
 * Enqueued on `stream`; returns after enqueueing. Accumulation order between voxels is
 * not fixed (float atomics), so results can differ in the last bits between runs.
 */
kct_status kct_project(const kct_plan *plan, const float *d_vol, float *d_proj, int32_t accumulate,
                       void *stream);

/*
 * Adjoint (backprojection) x = A^T y, with the same pair weights and pixel factors as
 * kct_project, so that <A x, y> = <x, A^T y> up to float32 rounding (Sec. III-D).
 *   d_proj  device float32 [nviews][nv][nu], read only.
 *   d_vol   device float32 [nz][ny][nx]; overwritten (accumulate = 0) or added to.
 * Each voxel is written by exactly one thread: the result is deterministic.
 */
kct_status kct_backproject(const kct_plan *plan, const float *d_proj, float *d_vol, int32_t accumulate,
                           void *stream);

/*
 * Batched forward projection: nbatch volumes, contiguous [nbatch][nz][ny][nx], through the
 * plan's views into nbatch projection stacks [nbatch][nviews][nv][nu], in one launch.
 * Same semantics as kct_project per batch member; ceil(nviews / chunk) * nbatch must not
 * exceed 65535, chunk being the plan's views per forward block (KCT_ERR_UNSUPPORTED
 * otherwise).
 */
kct_status kct_project_batch(const kct_plan *plan, const float *d_vol, int32_t nbatch, float *d_proj,
                             int32_t accumulate, void *stream);

/*
 * Batched adjoint: nbatch projection stacks [nbatch][nviews][nv][nu] into nbatch volumes
 * [nbatch][nz][ny][nx], in one launch; 1 <= nbatch <= 65535. Same semantics as
 * kct_backproject per batch member.
 */
kct_status kct_backproject_batch(const kct_plan *plan, const float *d_proj, int32_t nbatch, float *d_vol,
                                 int32_t accumulate, void *stream);

/*
 * Forward-kernel tuning. Each forward block takes one brick of voxels (8 x 8 columns x 64
 * voxels) through `chunk` consecutive views; more views per block re-read the brick from
 * HBM less often, fewer give more blocks to small problems. Default 16.
 *
 * kct_plan_autotune times one forward projection of d_vol with each candidate chunk
 * (1, 2, 4, 8, 16, 32, 64; a warm-up launch, then a timed one, CUDA events on `stream`) over
 * the plan's first min(nviews, 64) views, and keeps the fastest in the plan.
 *   d_vol   device float32 [nz][ny][nx], read only (the volume the timing uses).
 *   d_proj  device float32 [nviews][nv][nu]; its first min(nviews, 64) views are
 *           overwritten with scratch.
 *   chunk   optional: receives the chosen chunk.   ms: optional: its forward time (ms).
 * Synchronises `stream`; not for stream capture. Tune before capturing graphs that use
 * the plan: a captured launch keeps the chunk it was captured with.
 * kct_plan_set_view_chunk sets the chunk directly (1..64, KCT_ERR_INVALID_ARG otherwise);
 * kct_plan_get_view_chunk reads it. Work already enqueued keeps its chunk.
 */
kct_status kct_plan_autotune(kct_plan *plan, const float *d_vol, float *d_proj, int32_t *chunk, float *ms,
                             void *stream);
kct_status kct_plan_set_view_chunk(kct_plan *plan, int32_t chunk);
kct_status kct_plan_get_view_chunk(const kct_plan *plan, int32_t *chunk);

/*
 * Ray-driven comparator (not the CVP operator): for every pixel of every view, the average
 * over K x K rays through the sub-pixel points (u - 1/2 + (a + 1/2)/K, v - 1/2 + (b + 1/2)/K)
 * of the line integral of the volume, with exact path lengths through the voxel grid
 * (Siddon's method; the paper's multi-ray comparison projectors, Sec. IV). weighting 0
 * averages with equal weights (pixel-area average), 1 with the rays' solid-angle weights.
 *   d_vol   device float32 [nz][ny][nx];  d_proj  device float32 [nviews][nv][nu], overwritten.
 *   K in [1, 64]. Enqueued on `stream`. Used by the accuracy study of the two variants.
 */
kct_status kct_siddon_project(const kct_plan *plan, const float *d_vol, float *d_proj, int32_t K, int32_t weighting,
                              void *stream);

/*
 * Pixel factors F(u, v) of every view of the plan (its scaling mode) into
 * d_out, device float32 [nviews][nv][nu]. Enqueued on `stream`.
 */
kct_status kct_pixel_factors(const kct_plan *plan, float *d_out, void *stream);

/*
 * Number of nonzero voxel-pixel pairs A has, counted on the device for the plan's variant
 * (a pair counts when its weight is > 0). Synchronises `stream`.
 */
kct_status kct_count_pairs(const kct_plan *plan, uint64_t *count, void *stream);

/* Read and clear the plan's device error word (0 = no error). Synchronises `stream` (an
 * argument beyond the minimal boundary: the word is read on the caller's stream, after the
 * work it checks). Nonzero codes: 1 = a voxel footprint larger than the kernel's bound was
 * skipped. No counterpart in the paper (its kernels have no error reporting). */
kct_status kct_last_device_error(const kct_plan *plan, int32_t *code, void *stream);

/*
 * Forward projection for callers that must not allocate device memory (for example code
 * running inside another framework's memory pool, or a runtime with no allocator, where a
 * cudaMalloc would break the host application's memory accounting). The paper has no
 * counterpart: this is the same operator as kct_project with the plan's geometry passed
 * directly, and no plan.
 *   vol, det, pmats, nviews, variant, scaling  as for kct_plan_create (pmats on the host);
 *   d_vol, d_proj, accumulate, stream           as for kct_project.
 * Its scratch (per-view parameters, the unscaled sums, an error word) is a fixed array of
 * about 32.5 MiB compiled into the library, which every GPU that loads the library keeps
 * until the process exits. Limits: nviews <= 4096 and nu * nv * nviews <= 8388608 pixels;
 * larger requests return KCT_ERR_UNSUPPORTED before any work is enqueued.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and must therefore come before any stream capture on that device. All calls share the
 * one array and it keeps the last call's contents (cleared where needed at each call):
 * calls that overlap on the GPU, on any streams, race and give wrong results.
 * Every view is validated before anything is enqueued; the per-view parameters then reach
 * the array as the by-value arguments of small kernels, 32 views per launch, so no host
 * buffer has to outlive the call.
 * A voxel whose footprint is larger than the kernel's bound is skipped and recorded in the
 * array's error word, which kct_project_static_device_error reads.
 */
kct_status kct_project_static(const kct_volume_desc *vol, const kct_detector_desc *det, const double *pmats,
                              int32_t nviews, kct_variant variant, kct_scaling scaling, const float *d_vol,
                              float *d_proj, int32_t accumulate, void *stream);

/*
 * Read and clear the error word of the last kct_project_static call on the current device
 * (0 = no error; 1 = a voxel footprint larger than the kernel's bound was skipped, so the
 * projection misses that voxel). Companion of kct_project_static, which has no plan whose
 * error word kct_last_device_error could read; like it, this call allocates nothing. It
 * synchronises `stream`, which should be the stream of the call it checks. No counterpart
 * in the paper.
 */
kct_status kct_project_static_device_error(int32_t *code, void *stream);

/*
 * CGLS reconstruction with the plan's operator: conjugate gradients on the normal equations
 * A^T A x = A^T b, applying A and A^T once per step (the reconstruction that drives the
 * projector timings of Sec. IV-A; Krylov methods of Sec. V "Software"; textbook CGLS,
 * Bjorck 1996, Sec. 7.4). Per step: one kct_project, one kct_backproject and four vector
 * kernels (squared norms, x += alpha p with r -= alpha q, p = s + beta p); alpha and beta
 * stay on the device.
 *
 * Stopping rule: the normal-equation residual |A^T (b - A x_k)| / |A^T b| <= tol, checked
 * after every step (and once before the first, so a start that already meets it takes no
 * step), or max_iter steps.
 *
 *   d_b        device float32 [nviews][nv][nu], read only.
 *   d_x        device float32 [nz][ny][nx]: on entry the start x0 if warm_start != 0
 *              (ignored otherwise: the start is 0); on return the solution.
 *   d_atb      optional device float32 [nz][ny][nx], read only: A^T b of this plan if the
 *              caller already has it (a learned warm start computes it for its network input);
 *              the solve then does one backprojection fewer. NULL: computed here.
 *   max_iter   >= 0.   tol >= 0 (0 runs max_iter steps).
 *   d_work     device scratch of at least kct_cgls_workspace_bytes(plan) bytes, 256-byte
 *              aligned; owned by the caller, contents on entry ignored.
 *   h_normal, h_data   optional host arrays of max_iter + 1 doubles (NULL to skip): entry k
 *              gets the normal residual and |b - A x_k| / |b| after k steps.
 *   report     optional: steps taken, whether tol was met, and the final residuals.
 * d_b, d_x and d_atb must be 16-byte aligned and must not overlap d_work.
 * Synchronous: it reads the residuals from the device after every step (one 16-byte copy and
 * a stream synchronisation) and returns when the solve is done. Not for stream capture.
 */
typedef struct kct_cgls_report {
    int32_t iterations;        /* steps taken */
    int32_t converged;         /* 1 if the normal residual reached tol */
    double normal_residual;    /* |A^T (b - A x)| / |A^T b| at return */
    double data_residual;      /* |b - A x| / |b| at return */
} kct_cgls_report;

size_t kct_cgls_workspace_bytes(const kct_plan *plan);

kct_status kct_cgls(const kct_plan *plan, const float *d_b, float *d_x, const float *d_atb, int32_t warm_start,
                    int32_t max_iter, double tol, void *d_work, size_t work_bytes, double *h_normal, double *h_data,
                    kct_cgls_report *report, void *stream);

/* Static description of a status code. No counterpart in the paper (error reporting of
 * this library). */
const char *kct_status_string(kct_status status);

/* Detail of the last failure on the calling thread ("" if none). No counterpart in the
 * paper. */
const char *kct_last_error_message(void);

/* KCT_VERSION of the library. No counterpart in the paper. */
int32_t kct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KCT_H */
