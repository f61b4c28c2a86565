/*
 * usvol -- GB300 (sm_103a) free-hand ultrasound volume reconstruction.
 *
 * C ABI of the data-parallel path of "Real-time volumetric free-hand
 * ultrasound imaging for large-sized organs" (arXiv 2412.00058):
 *
 *   pose-tracked B-mode frames --insert--> voxel accumulators
 *        --fill (normalise + 3x3x3 hole fill)--> voxel values + has-data mask
 *        --project (depth band)--> coronal spine view
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Axes: x lateral, y along the spine (sweep), z depth.  Volumes are stored
 *    C-order [nz][ny][nx] (x fastest).  Voxel (i,j,k) has its centre at
 *    origin + (i,j,k)*spacing (mm).
 *  - Linear-probe frame pixel (u, v) = (column, row) sits at the image-frame
 *    point (u*sx, 0, v*sy) mm, the upper-left pixel at the origin (the
 *    paper's Alg. 1 steps 2-3 locate frames by their upper-left pixel).
 *    Convex frames hold pre-scan-conversion samples: row i is the radius
 *    r = r0 + i*dr, column j the beam angle theta_j = -sector/2 +
 *    j*sector/(W-1); the sample sits at (r sin theta, 0, r cos theta - r0).
 *  - image_to_probe (calibration) and poses (probe->world, the paper's
 *    T_T^W, Alg. 1) are 4x4 row-major float64 matrices; the world point of
 *    a pixel is p = pose * image_to_probe * (x_img, 0, z_img, 1)^T.
 *  - Every call is asynchronous on the caller's CUDA stream (`stream` is a
 *    cudaStream_t; NULL = legacy default stream).  Device-side conditions
 *    (skipped frames, saturated voxels) are reported by usv_status().
 *  - Pointers named *_dev are device pointers owned by the caller; they must
 *    stay valid until the stream has passed the call.  Pointers named *_host
 *    are host memory read during the call only.  The library never
 *    allocates device memory: the volume lives in caller-provided storage
 *    (each volume handle owns 2 MB of pinned host memory for staging poses).
 *  - Return value: USV_OK (0) or a negative USV_ERR_* code.  Argument errors
 *    are detected on the host before anything is launched.
 *  - A usv_volume is not thread-safe; use it from one host thread / stream.
 */
#ifndef USVOL_H
#define USVOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define USVOL_ABI_VERSION 2

/* ---- return codes ---- */
#define USV_OK 0
#define USV_ERR_ARG (-1)     /* bad argument (null pointer, bad size, bad matrix) */
#define USV_ERR_RANGE (-2)   /* argument outside the supported range            */
#define USV_ERR_CUDA (-3)    /* a CUDA runtime call failed                      */
#define USV_ERR_TIMEOUT (-4) /* a bounded device wait ran out                   */
#define USV_ERR_NOMEM (-5)   /* caller storage smaller than usv_volume_bytes()  */
#define USV_ERR_UNSUPPORTED (-6) /* mode / geometry / dtype combination not built */

/* ---- device status bits returned by usv_status() ---- */
#define USV_STATUS_BAD_POSE 0x1u   /* >= 1 frame skipped: non-affine pose, NaN/Inf or out of range */
#define USV_STATUS_SATURATED 0x2u  /* >= 1 voxel count reached 2^24 (its sum may have wrapped)     */
#define USV_STATUS_TIMEOUT 0x4u    /* a bounded device wait gave up                                 */
#define USV_STATUS_OOB 0x8u        /* checked build only: a kernel write outside its buffer was
                                      caught and skipped (a library bug; never set otherwise)     */

typedef struct usv_volume usv_volume; /* opaque, host-side handle */

typedef enum {
    USV_PNN = 0,      /* pixel nearest neighbour, exact integer sum + count (Sec. II.C) */
    USV_TRILINEAR = 1 /* trilinear splat, FP32 weighted sum + weight                    */
} usv_mode;

/* Flag OR-ed into the mode of usv_volume_bytes() / usv_volume_create(): the
 * storage also holds a spare set of accumulators, which lets
 * usv_fill_holes_and_clear() clear the accumulators inside the fill pass
 * (no counterpart in the paper; costs 8 B per voxel of extra storage). */
#define USV_SPARE_ACCUM 0x100

typedef enum { USV_LINEAR = 0, USV_CONVEX = 1 } usv_geom;
typedef enum { USV_U8 = 0, USV_F32 = 1 } usv_dtype;

typedef struct {
    int32_t nx, ny, nz;
} usv_grid;

/* Tile shape of the insertion kernels: frames are cut into tiles of
 * tile_w columns x tile_h rows, and one thread block inserts one tile of
 * frames_per_cta consecutive frames (no counterpart in the paper; the
 * results do not depend on it, except for the FP32 summation order of the
 * trilinear mode).  USV_PNN: tile_w 64, 128 or 256, tile_h 1..1024,
 * frames_per_cta 1..16 (1..8 with tile_w 256); default 128 x 64 x 12.
 * USV_TRILINEAR: tile_w 256,
 * tile_h 1..128, frames_per_cta 1..8; default 256 x 64 x 4.  In USV_PNN,
 * frames_per_cta is an upper bound: a batch of frames too small to fill
 * the GPU is spread over more thread blocks with fewer frames each. */
typedef struct {
    int32_t tile_w, tile_h, frames_per_cta;
} usv_tile_config;

typedef struct {
    double image_to_probe[16]; /* 4x4 row-major, bottom row must be 0 0 0 1 */
    int32_t geom;              /* usv_geom */
    double sx_mm, sy_mm;       /* linear: lateral / axial pixel spacing      */
    double r0_mm, dr_mm;       /* convex: first sample radius, radial step   */
    double sector_deg;         /* convex: full sector angle (0, 180)         */
} usv_calibration;

/* ------------------------------------------------------------------------
 * usv_volume_bytes -- device bytes a volume needs: accumulators, filled
 * values, has-data bit mask, per-frame set-up scratch and the status word.
 * PNN: 8 B + 1 B + 1/8 B per voxel (+ ~1.2 MB); trilinear: 8 + 4 + 1/8;
 * with USV_SPARE_ACCUM in `mode`, 8 B more per voxel.
 * Returns 0 if the grid is invalid (any n < 1, or more than 2^31-1 voxels).
 * ---------------------------------------------------------------------- */
size_t usv_volume_bytes(usv_grid grid, int32_t mode);

/* ------------------------------------------------------------------------
 * usv_volume_create -- bind a volume to caller-provided device storage
 * (the paper's reconstruction volume, Sec. II.C).  `device_storage` must be
 * 256-byte aligned and hold usv_volume_bytes(grid, mode) bytes; it stays
 * owned by the caller and must outlive the handle.  spacing_mm > 0 and
 * finite; origin_mm finite (centre of voxel (0,0,0)).  The accumulators are
 * NOT cleared: call usv_volume_reset() before the first insert.
 * Allocates the small host-side handle and the 2 MB pinned, device-mapped
 * ring that stages host poses (usv_insert_frames); no device memory.
 * ---------------------------------------------------------------------- */
int usv_volume_create(usv_grid grid, const double spacing_mm[3], const double origin_mm[3],
                      int32_t mode, void *device_storage, size_t storage_bytes,
                      usv_volume **out);

/* Frees the host handle and its pose ring; the storage is the caller's.
 * Waits on the host for the queued set-up kernels that still read poses
 * from the ring, then frees it. */
int usv_volume_destroy(usv_volume *vol);

/* Zero the accumulators and the status word (start of a new scan). */
int usv_volume_reset(usv_volume *vol, void *stream);

/* ------------------------------------------------------------------------
 * usv_insert_frames -- insert n frames into the volume (Sec. II.C: PNN
 * reconstruction of the newly acquired frames only, on top of what the
 * volume already holds -- the paper's incremental method).
 *   images_dev  [n][H][W] uint8 (USV_U8) or float32 (USV_F32), C-order.
 *   poses_host  [n][16] float64 probe->world matrices in host memory (the
 *               tracker's output, Sec. II.B), row-major; read during the
 *               call: they are copied into the volume's pinned, device-
 *               mapped staging ring (2 MB, allocated by usv_volume_create),
 *               which the work queued on `stream` reads in place over the
 *               host link (no copy-engine transfer, so the call never waits
 *               behind the caller's own frame copies).  The call waits on
 *               the host only when the ring is still held by work the
 *               device has not done yet (more than 2 MB of poses, or 64
 *               calls, in flight).  Not allowed while
 *               `stream` is being captured into a CUDA graph
 *               (USV_ERR_UNSUPPORTED): capture usv_insert_frames_dev().
 *   cal         host struct, read during the call only.
 * USV_PNN: every pixel goes to its nearest voxel; with the per-frame map
 *   q(u,v) = C + u*A + v*B quantised to Q31.32 (each of the nine values
 *   rounded half away from zero after multiplying by 2^32; the FP64 set-up
 *   M = pose*K is summed left to right without fused multiply-add, then
 *   A = M[:,0]*sx/s, B = M[:,2]*sy/s, C = (M[:,3]-origin)/s), the voxel is
 *   floor((Q + 2^31) / 2^32) per axis; pixels outside the grid are dropped;
 *   the voxel's sum += I, count += 1.  Exact and order-independent.
 *   Needs USV_U8 and USV_LINEAR.
 * USV_TRILINEAR: each sample spreads I over its 8 neighbouring voxels with
 *   trilinear weights (weights < 2^-20 and out-of-grid corners dropped),
 *   FP32 accumulation.  USV_U8 or USV_F32; USV_LINEAR or USV_CONVEX.  A
 *   USV_F32 sample is inserted only if it is finite with |I| <= 2^64; a NaN,
 *   an infinity or a larger magnitude counts as a missing sample (no weight
 *   anywhere), so it cannot spread into other voxels.
 * A frame whose pose is not affine (bottom row != 0 0 0 1), not finite, or
 * maps outside +-2^29 voxels (|A|,|B| >= 2^14 per step) is skipped and sets
 * USV_STATUS_BAD_POSE.  Limits: 0 <= n, 1 <= H, W <= 32768.
 * ---------------------------------------------------------------------- */
int usv_insert_frames(usv_volume *vol, const void *images_dev, int32_t n, int32_t H, int32_t W,
                      int32_t dtype, const double *poses_host, const usv_calibration *cal,
                      void *stream);

/* usv_insert_frames with the poses already in device memory (poses_dev
 * [n][16] float64, 8-byte aligned, read by the device when the stream gets
 * there): no host staging, so it can be captured into a CUDA graph.  Same
 * result, arguments and errors otherwise. */
int usv_insert_frames_dev(usv_volume *vol, const void *images_dev, int32_t n, int32_t H,
                          int32_t W, int32_t dtype, const double *poses_dev,
                          const usv_calibration *cal, void *stream);

/* ------------------------------------------------------------------------
 * usv_frames_voxel_box -- the voxel box [lo, hi) (x, y, z; half-open,
 * clipped to the grid) that holds every voxel the given frames can write,
 * nearest voxel or trilinear corner, widened by `margin` >= 0 voxels on
 * every side: the region that changes when they are inserted (the paper
 * re-processes only the areas that need updating, Sec. II.C).  Pass it,
 * widened by one more voxel, to usv_fill_holes_region() and its x-y part to
 * usv_project_depth_band_region().  Computed on the host in FP64 from the
 * frames' in-plane corners (the map is affine in the image plane), with one
 * voxel of slack for rounding; frames the insertion would skip (pose not
 * affine or not finite) are ignored; with none left the box is empty
 * (lo = hi = 0).  grid, spacing_mm, origin_mm as for usv_volume_create()
 * (no volume needed, no device work); poses_host [n][16] as for
 * usv_insert_frames().
 * ---------------------------------------------------------------------- */
int usv_frames_voxel_box(usv_grid grid, const double spacing_mm[3], const double origin_mm[3],
                         const double *poses_host, int32_t n, int32_t H, int32_t W,
                         const usv_calibration *cal, int32_t margin, int32_t lo[3], int32_t hi[3]);

/* ------------------------------------------------------------------------
 * Tissue segmentation by depth of cut (the paper's Algorithms 1 and 2,
 * Sec. II.D): rows of a frame above its "depth of cut" -- the superficial
 * tissue over the bone -- are not inserted (Alg. 1 step 5, Alg. 2 step 4).
 *
 * usv_insert_frames_cut -- usv_insert_frames_dev with first_row_dev[n] (device
 *   int32): rows v < first_row_dev[f] of frame f are cut away (for a convex
 *   probe: radial samples i < first_row).  Negative values keep every row.
 *
 * usv_cut_rows_alg1 -- Alg. 1 (real-time): first_row_dev[f] = the row of
 *   depth Cut_f = K * |P_c1.x - P_cf.x - L/2| + D (Alg. 1 step 4).  P_cf is
 *   the world position of frame f's upper-left pixel, pose * calibration *
 *   (0,0,0,1); ".x" is the coordinate along spine_dir (the paper's x axis,
 *   the spine direction, given in world coordinates); P_c1 (p1_mm) is that
 *   of the scan's first frame (the neck), kept by the caller across
 *   batches.  Computed in FP64, each operation rounded in order:
 *   d = ((p1x-px)*ex + (p1y-py)*ey) + (p1z-pz)*ez; cut = K*|d - L/2| + D;
 *   row = ceil(cut / row_mm) clamped to [0, H], row_mm = sy_mm (linear) or
 *   dr_mm (convex).  K, D, L are the paper's user constants.
 *
 * usv_bone_rows_alg2 -- Alg. 2 (after the scan, uint8 frames): in rows
 *   v >= search_from_row (the lower image, step 2) the score
 *   I(v,u) * max(0, I(v,u) - I(v+drop_rows,u)) marks a bright contour with
 *   a shadow below it; per column the first row of the maximum score
 *   (search_from_row if all are 0), per frame the lower median over the
 *   columns -> bone_row_dev[f]; then the lower median over the frames
 *   [f - window/2, f + window/2] clipped to the scan (step 3, window odd)
 *   minus margin_rows, at least 0 -> first_row_dev[f].  Exact integers.
 *   H <= USV_ALG2_MAX_ROWS.
 * ---------------------------------------------------------------------- */
typedef struct {
    double K;            /* cut depth per distance from the middle of the back (mm/mm) */
    double D_mm;         /* cut depth at the middle of the back (mm) */
    double L_mm;         /* length of the back (mm) */
    double spine_dir[3]; /* unit vector along the spine (the paper's x), world coordinates */
    double p1_mm[3];     /* world position of the first frame's upper-left pixel (mm) */
} usv_alg1_params;

typedef struct {
    int32_t search_from_row; /* first row searched for the bone contour */
    int32_t drop_rows;       /* the shadow is compared this many rows below (>= 1) */
    int32_t window;          /* temporal median window in frames (odd, >= 1) */
    int32_t margin_rows;     /* rows kept above the median bone row (>= 0) */
} usv_alg2_params;

#define USV_ALG2_MAX_ROWS 8192

int usv_insert_frames_cut(usv_volume *vol, const void *images_dev, int32_t n, int32_t H,
                          int32_t W, int32_t dtype, const double *poses_dev,
                          const usv_calibration *cal, const int32_t *first_row_dev, void *stream);
int usv_cut_rows_alg1(const double *poses_dev, int32_t n, int32_t H, const usv_calibration *cal,
                      const usv_alg1_params *p, int32_t *first_row_dev, void *stream);
int usv_bone_rows_alg2(const uint8_t *images_dev, int32_t n, int32_t H, int32_t W,
                       const usv_alg2_params *p, int32_t *bone_row_dev, int32_t *first_row_dev,
                       void *stream);

/* ------------------------------------------------------------------------
 * Pose refinement (correcting the patient movement that long scans suffer,
 * Sec. I and III.A): the gradient of a depth-band projection loss with
 * respect to every frame's 6-DoF pose, through the trilinear splat.
 *
 * usv_pose_loss_grad -- vol must be USV_TRILINEAR, the probe USV_LINEAR,
 *   1 <= n <= 4096.  Clears vol and inserts the frames, then
 *     V = S / (W + eps)             (soft normalisation, differentiable)
 *     P[y][x] = mean over z in [z_lo, z_hi) of V          -> proj_dev
 *     L = sum (P - target)^2                              -> *loss_dev (FP64)
 *   and, for the left perturbation of each pose about its frame centre c
 *   (p' = R(w)(p - c) + c + t, t in mm, w a rotation vector in rad),
 *     grad_dev[f][0..2] = dL/dt,  grad_dev[f][3..5] = dL/dw  at t = w = 0
 *   (FP64 per frame; trilinear weights are piecewise linear: at a cell face
 *   the derivative from the cell floor() selects).  adj_scratch_dev holds
 *   2 * (z_hi - z_lo) * ny * nx floats.  target_dev/proj_dev: [ny][nx].
 *
 * usv_apply_pose_delta -- poses_out[f] = T(t) T(c) R(w) T(-c) poses[f] for
 *   delta[f] = (t, w) (Rodrigues), c the frame centre ((W-1)sx/2, 0,
 *   (H-1)sy/2) in world coordinates: the perturbation the gradient refers
 *   to.  Linear probes; poses_out must not alias poses.
 * ---------------------------------------------------------------------- */
int usv_pose_loss_grad(usv_volume *vol, const void *images_dev, int32_t n, int32_t H, int32_t W,
                       int32_t dtype, const double *poses_dev, const usv_calibration *cal,
                       int32_t z_lo, int32_t z_hi, float eps, const float *target_dev,
                       float *proj_dev, float *adj_scratch_dev, double *loss_dev,
                       double *grad_dev, void *stream);
int usv_apply_pose_delta(const double *poses_dev, const double *delta_dev, int32_t n, int32_t H,
                         int32_t W, const usv_calibration *cal, double *poses_out_dev,
                         void *stream);

/* ------------------------------------------------------------------------
 * usv_insert_frames_multi -- several (volume, batch of frames) jobs in one
 * go: the batches of concurrent scan sessions, each of its own size (the
 * paper processes the newly acquired frames of each scan incrementally,
 * Sec. II.C; batching sessions together has no counterpart there).  The
 * result in every volume is bit-identical to usv_insert_frames() of its job.
 * Two launches in all: one frame set-up over all jobs and one persistent
 * insertion kernel whose thread blocks walk the jobs' tiles of frames.
 * Every job: a USV_PNN volume, USV_U8 frames, a USV_LINEAR calibration,
 * 0 <= n <= 4096 frames; the arguments of a job mean what they mean for
 * usv_insert_frames_dev().  All volumes on one device, each in at most one job,
 * at most 32 jobs (USV_ERR_RANGE beyond; USV_ERR_ARG for a repeated volume
 * or volumes on different devices; USV_ERR_UNSUPPORTED for other modes or
 * geometries).  A volume's tile shape (usv_set_tile_config, usv_tune_insert)
 * applies when its tile_w is 128, else 128 x 64 x 8.
 * ---------------------------------------------------------------------- */
typedef struct {
    usv_volume *vol;
    const void *images_dev;  /* [n][H][W] uint8 */
    int32_t n, H, W;
    int32_t dtype;           /* USV_U8 */
    const double *poses_dev; /* [n][16] row-major probe->world, mm */
    const usv_calibration *cal;
    const int32_t *first_rows_dev; /* [n] first inserted row per frame, as for
                                      usv_insert_frames_cut(); NULL: all rows */
} usv_insert_job;

int usv_insert_frames_multi(const usv_insert_job *jobs, int32_t njobs, void *stream);

/* ------------------------------------------------------------------------
 * Tile shapes per frame size (no counterpart in the paper).
 * usv_tune_insert -- the insertion autotuner: inserts the first
 * min(n, 4096) of the given frames with each candidate tile shape into the
 * caller's scratch accumulators, times the insertion with CUDA events on
 * `stream` (the call waits for the stream), and keeps the fastest shape in
 * the volume for frames of H x W.  The volume's own accumulators are not
 * touched (its per-frame set-up scratch is).  Candidates: USV_PNN tile_w
 * {64, 128, 256} x tile_h {32, 48, 64, 96, 128} x frames_per_cta {4, 8, 12, 16}
 * (at most 8 with tile_w 256);
 * USV_TRILINEAR tile_h {16, 32, 64, 128} x frames_per_cta {2, 4, 8}.
 *   scratch_dev    device, 16-byte aligned, >= 8 * nx * ny * nz bytes
 *   best_out       the chosen shape (may be NULL)
 *   best_ms_out    its insertion time in ms for the frames tried (may be NULL)
 * Arguments and errors as usv_insert_frames_dev(), plus USV_ERR_NOMEM for a
 * short scratch.
 * usv_set_tile_config sets the shape for frames of H x W (cfg NULL: back to
 * the default); USV_ERR_RANGE if invalid for the volume's mode, at most 8
 * frame sizes per volume.  usv_get_tile_config reads the shape in use.
 * ---------------------------------------------------------------------- */
int usv_tune_insert(usv_volume *vol, const void *images_dev, int32_t n, int32_t H, int32_t W,
                    int32_t dtype, const double *poses_dev, const usv_calibration *cal,
                    void *scratch_dev, size_t scratch_bytes, usv_tile_config *best_out,
                    float *best_ms_out, void *stream);
int usv_set_tile_config(usv_volume *vol, int32_t H, int32_t W, const usv_tile_config *cfg);
int usv_get_tile_config(usv_volume *vol, int32_t H, int32_t W, usv_tile_config *out);

/* ------------------------------------------------------------------------
 * usv_fill_holes -- normalisation + hole filling (PNN's second stage; the
 * 3x3x3 neighbourhood is radius 1, the only radius built).  One pass that
 * reads only the accumulators, so it can be re-run after more inserts:
 *   count > 0 : value = mean (PNN: (2*sum + count) / (2*count), integer
 *               round half up, uint8; trilinear: S / W in FP32);
 *   count == 0: value = pooled mean over the non-empty in-grid neighbours
 *               among the 26 (sum of sums / sum of counts); none -> empty.
 * Writes the value volume and the has-data bit mask.
 * ---------------------------------------------------------------------- */
int usv_fill_holes(usv_volume *vol, int32_t radius, void *stream);

/* ------------------------------------------------------------------------
 * usv_fill_holes_and_clear -- usv_fill_holes(), after which the volume's
 * accumulators are zero, as after usv_volume_reset(): the call for the end
 * of a sweep, when the next sweep starts from an empty volume (no
 * counterpart in the paper).  With USV_SPARE_ACCUM in USV_PNN mode the fill
 * kernel writes zeros into the spare accumulators while it reads the
 * current ones, and the two sets swap: the clearing costs no separate pass
 * over memory.  Otherwise it is usv_fill_holes() followed by
 * usv_volume_reset().  Same arguments, errors and outputs as
 * usv_fill_holes(); usv_volume_read(USV_READ_ACCUM) afterwards reads zeros.
 * ---------------------------------------------------------------------- */
int usv_fill_holes_and_clear(usv_volume *vol, int32_t radius, void *stream);

/* ------------------------------------------------------------------------
 * usv_project_depth_band -- the VPI spine view (Sec. III.B): for every
 * (x, y) the mean of the filled values of the has-data voxels with
 * z_lo <= z < z_hi (0 where there are none), one IEEE FP32 division.
 *   out_dev    [ny][nx] float32 (required)
 *   count_dev  [ny][nx] uint16 number of voxels averaged (may be NULL)
 * Requires 0 <= z_lo < z_hi <= nz and z_hi - z_lo <= 65535.  Reads the
 * output of the last usv_fill_holes().
 * ---------------------------------------------------------------------- */
int usv_project_depth_band(usv_volume *vol, int32_t z_lo, int32_t z_hi, float *out_dev,
                           uint16_t *count_dev, void *stream);

/* ------------------------------------------------------------------------
 * Region forms, for incremental display (the paper re-processes "only the
 * areas that need to be updated" after each batch, Sec. II.C):
 * usv_fill_holes_region refreshes the filled values and mask of the voxels
 * [lo, hi) (x, y, z; clipped to the grid; x widened down to a multiple of
 * 32) from the current accumulators -- after inserting frames whose voxels
 * lie in [a, b), refreshing [a - 1, b + 1) updates everything that changed.
 * usv_project_depth_band_region recomputes the projection of columns
 * [xy_lo, xy_hi) only; the rest of out_dev / count_dev is left as it is.
 * The whole-volume calls are these with the full grid.
 * ---------------------------------------------------------------------- */
int usv_fill_holes_region(usv_volume *vol, const int32_t lo[3], const int32_t hi[3],
                          int32_t radius, void *stream);
int usv_project_depth_band_region(usv_volume *vol, int32_t z_lo, int32_t z_hi,
                                  const int32_t xy_lo[2], const int32_t xy_hi[2], float *out_dev,
                                  uint16_t *count_dev, void *stream);

/* ------------------------------------------------------------------------
 * usv_volume_read -- copy one field to caller device memory in canonical
 * [nz][ny][nx] order (the paper saves the finished volume as slices).
 *   USV_READ_ACCUM : PNN uint64 (low 32 bits sum, high 32 bits count);
 *                    trilinear float32 pairs (S, W)
 *   USV_READ_VALUES: PNN uint8; trilinear float32
 *   USV_READ_MASK  : uint8 0/1 has-data
 * USV_WRITE_ACCUM (usv_volume_write) loads accumulators back, e.g. to
 * resume a saved scan bit-exactly.
 * ---------------------------------------------------------------------- */
#define USV_READ_ACCUM 0
#define USV_READ_VALUES 1
#define USV_READ_MASK 2
int usv_volume_read(usv_volume *vol, int32_t what, void *dst_dev, void *stream);
int usv_volume_write_accum(usv_volume *vol, const void *src_dev, void *stream);

/* ------------------------------------------------------------------------
 * usv_insert_pnn_noalloc -- nearest-neighbour insertion that allocates no
 * memory at all.  The paper has no counterpart: this serves callers that
 * cannot allocate device memory on the path that feeds frames (a real-time
 * acquisition loop whose memory is fixed before the scan -- an allocation
 * can block and synchronise the device mid-scan --, a deployment that
 * forbids allocation after start-up, a plugin whose host framework owns
 * every buffer), so they cannot provide the storage usv_volume_create()
 * takes.  The result is bit-identical to usv_insert_frames() in USV_PNN.
 *   accum_dev   [nz][ny][nx] uint64 packed accumulators (low 32 bits sum,
 *               high 32 bits count, the USV_READ_ACCUM layout), owned by the
 *               caller, 8-byte aligned; zero it to start a scan.
 *   grid, spacing_mm, origin_mm   as for usv_volume_create().
 *   images_dev, n, H, W, poses_dev, cal   as for usv_insert_frames_dev(),
 *               uint8 frames of a linear probe.
 *   status_dev  optional device word: USV_STATUS_* bits are OR-ed into it
 *               (clear it first); NULL: not reported.
 * Its scratch (per-frame set-up records) is a fixed array inside the
 * library sized for USV_NOALLOC_MAX_FRAMES frames (about 160 KB that every
 * GPU which loads the library keeps until the process exits); n beyond that
 * returns USV_ERR_RANGE -- split larger batches.  The first call on each
 * device (and the first after the device's context was reset) looks up the
 * array's device address and the device's SM count; make that first call
 * before any stream capture.  All calls on one device share the array, so calls
 * that overlap on the GPU (unordered streams) race: order them on one
 * stream.  Nothing in the array has to start at zero: every call writes the
 * records it reads.  Asynchronous on `stream` like the other calls.
 * ---------------------------------------------------------------------- */
#define USV_NOALLOC_MAX_FRAMES 1024
int usv_insert_pnn_noalloc(uint64_t *accum_dev, usv_grid grid, const double spacing_mm[3],
                           const double origin_mm[3], const void *images_dev, int32_t n,
                           int32_t H, int32_t W, const double *poses_dev,
                           const usv_calibration *cal, uint32_t *status_dev, void *stream);

/* ------------------------------------------------------------------------
 * usv_test_fill_wait_timeout -- for testing the device-side failure path
 * only (no counterpart in the paper).  Runs usv_fill_holes() with the copy
 * of plane `plane` (0 <= plane < nz) never issued, so the fill kernel's
 * bounded wait for it runs out after about one second: the kernel sets
 * USV_STATUS_TIMEOUT, waits (bounded) for its copies still in flight and
 * returns.  The values and mask written by this call are undefined; the
 * accumulators are untouched and the volume stays usable.
 * USV_ERR_UNSUPPORTED unless the fill takes its tensor-copy path (USV_PNN,
 * even nx), the only one that waits on the device.
 * ---------------------------------------------------------------------- */
int usv_test_fill_wait_timeout(usv_volume *vol, int32_t plane, void *stream);

/* ------------------------------------------------------------------------
 * usv_test_insert_trilinear_carry -- for testing only (no counterpart in the
 * paper).  usv_insert_frames_dev() on a USV_TRILINEAR volume with the register
 * carry of shared corner terms between face-adjacent cells switched on
 * (carry != 0, what usv_insert_frames() does) or off (what the pose-gradient
 * path does), so that both forms of the kernel can be checked against the
 * oracle on the same frames.  Same arguments and errors as
 * usv_insert_frames_dev(); USV_ERR_UNSUPPORTED for a USV_PNN volume.
 * ---------------------------------------------------------------------- */
int usv_test_insert_trilinear_carry(usv_volume *vol, const void *images_dev, int32_t n,
                                    int32_t H, int32_t W, int32_t dtype, const double *poses_dev,
                                    const usv_calibration *cal, int32_t carry, void *stream);

/* ------------------------------------------------------------------------
 * usv_probe_red_f2 -- measurement utility (no counterpart in the paper):
 * the ceiling the trilinear insertion's float2 vector atomics are measured
 * against.  (num SMs x 8) blocks of 256 threads each add (1, 1) to
 * reds_per_thread float2 entries of buf_dev ([bytes / 8] float2, 8-byte
 * aligned, caller-owned; its contents grow): thread t of T takes entries
 * (t + k*T) mod n, so a warp's reductions are one coalesced 256-byte run.
 * Time it with events on `stream`; (T * reds_per_thread) / seconds is the
 * reduction rate for that buffer size (L2-resident or not).
 * ---------------------------------------------------------------------- */
int usv_probe_red_f2(void *buf_dev, size_t bytes, int32_t reds_per_thread, void *stream);

/* Synchronise `stream`, then return the device status bits (>= 0) and clear
 * them, or a negative USV_ERR_* code. */
int usv_status(usv_volume *vol, void *stream);

/* Human-readable text for a return code. */
const char *usv_strerror(int code);

/* Text of the CUDA error behind the calling thread's last USV_ERR_CUDA. */
const char *usv_last_cuda_error(void);

/* ABI version compiled into the library (USVOL_ABI_VERSION). */
int usv_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* USVOL_H */
