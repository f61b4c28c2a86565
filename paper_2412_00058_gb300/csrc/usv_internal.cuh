// Internal declarations shared by the usvol translation units (not part of
// the public ABI, which is include/usvol.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/usvol.h"

namespace usv {

// Checked build (compiled with -DUSV_CHECKED): every global write and atomic
// of the kernels, and every shared-memory accumulation, first tests its
// index against the buffer it writes; an index outside is skipped and sets
// USV_STATUS_OOB.  The regular build compiles the tests away.
#ifdef USV_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

__device__ __forceinline__ bool guard(unsigned long long idx, unsigned long long limit,
                                      uint32_t *status)
{
    if (!kChecked || idx < limit)
        return true;
    atomicOr(status, USV_STATUS_OOB);
    return false;
}

// Per-frame set-up record written by k_frame_setup (A0) into the volume's
// scratch area and read by the insertion kernels.
struct FrameRec {
    long long q[9];  // Q31.32 per-step map: A (per column), B (per row), C (pixel 0,0)
    double d[9];     // FP64 map; linear: same as q unquantised; convex: per-mm factors
    int valid;       // 0: frame skipped (bad pose)
    int nmax;        // upper bound on the pixels of this frame that share one voxel
    int first_row;   // rows above it are cut away (tissue segmentation); 0: keep all
    int pad;
};
static_assert(sizeof(FrameRec) == 160, "FrameRec layout");

// Host-side handle behind usv_volume*.
// Insertion tile shape (the public usv_tile_config).
using TileCfg = usv_tile_config;
// Defaults, from the whole-spine profiles: PNN 128 x 64 pixels x 8 frames,
// trilinear 256 columns x 64 rows x 4 frames.
constexpr TileCfg kPnnTileDefault = {128, 64, 12};
constexpr TileCfg kTriTileDefault = {256, 64, 4};
constexpr int kTunedCap = 8;  // frame sizes (H, W) with a chosen tile per volume

struct TunedTile {
    int H, W;
    TileCfg cfg;
};

class PoseRing;  // pinned host staging of host-side poses (usv_api.cu)

struct Volume {
    usv_grid g;
    double spacing[3];
    double origin[3];
    int mode;
    char *base;
    size_t bytes;
    void *acc;          // PNN: unsigned long long[N]; trilinear: float2[N] (S, W)
    void *spare;        // USV_SPARE_ACCUM: a second accumulator set (swaps with acc), or null
    void *val;          // PNN: uint8_t[N]; trilinear: float[N]
    uint32_t *mask;     // [nz][ny][nxw] bit words, bit x%32 of word x/32
    int nxw;
    FrameRec *rec;      // scratch: kRecCap records
    double2 *beams;     // scratch: kBeamCap (sin, cos) pairs for convex beams
    uint32_t *status;   // one word of USV_STATUS_* bits
    int num_sms;
    int device;
    TunedTile tuned[kTunedCap];  // tile shapes set or tuned per frame size
    int ntuned;
    PoseRing *ring;     // host poses staged here, read in place (owned by the handle)
};

// The tile for frames of H x W in this volume: a tuned or set one, else the
// mode's default.
TileCfg tile_for(const Volume &v, int H, int W);
bool pnn_tile_ok(const TileCfg &c);
bool tri_tile_ok(const TileCfg &c);

constexpr int kRecCap = 4096;      // frames per set-up + insert launch pair
constexpr int kBeamCap = 32768;    // max W
constexpr int kMaxDim = 32768;     // max H, W

struct Layout {
    size_t acc, val, mask, rec, beams, status, spare, total;  // spare: 0 if none
};
Layout layout_for(usv_grid g, int mode);  // mode may carry USV_SPARE_ACCUM

// Set-up parameters passed by value to k_frame_setup.
struct SetupParams {
    double K[16];
    double sx, sy;        // linear: mm per column / row; convex: 1, 1 (per mm)
    double s[3], o[3];
    int convex;
    const int32_t *first_rows;  // per-frame first inserted row, or null (all rows)
};

// Several (volume, batch of frames) jobs in one launch (usv_insert_frames_multi).
constexpr int kMaxJobs = 32;
struct SetupJob {
    const double *poses;
    SetupParams sp;
    FrameRec *rec;
    uint32_t *status;
};
struct SetupJobs {
    int njobs;
    int begin[kMaxJobs + 1];  // prefix sums of the jobs' frame counts
    SetupJob job[kMaxJobs];
};
struct InsertJob {
    const Volume *v;
    const uint8_t *img;
    int n, H, W;
    TileCfg cfg;  // tile_w must be 128
};

// Raises `func`'s dynamic shared-memory limit to dyn_smem on the current
// device, once per (kernel, device) and safely from several host threads;
// with blocks_per_sm, also returns how many blocks of `threads` threads fit
// on one SM at that size.
cudaError_t prepare_kernel(const void *func, int dyn_smem, int threads = 0,
                           int *blocks_per_sm = nullptr);

// ---- launchers (each in its own translation unit) ----
cudaError_t launch_frame_setup(const double *poses, int n, const SetupParams &sp, FrameRec *rec,
                               uint32_t *status, cudaStream_t st);
cudaError_t launch_beam_setup(double2 *beams, int W, double sector_deg, cudaStream_t st);
cudaError_t launch_frame_setup_multi(const SetupJobs &jobs, cudaStream_t st);
cudaError_t launch_insert_pnn_multi(const InsertJob *jobs, int njobs, int num_sms,
                                    cudaStream_t st);
struct Alg1Params {
    double K[16];
    double k, d_mm, half_l_mm, dir[3], p1[3], row_mm;
};
cudaError_t launch_cut_rows_alg1(const double *poses, int n, int H, const Alg1Params &p,
                                 int32_t *first_rows, cudaStream_t st);
cudaError_t launch_bone_rows_alg2(const uint8_t *img, int n, int H, int W, int from_row, int drop,
                                  int window, int margin, int32_t *bone_rows, int32_t *first_rows,
                                  cudaStream_t st);
cudaError_t launch_insert_pnn(const Volume &v, const uint8_t *img, int n, int H, int W,
                              cudaStream_t st, const TileCfg &cfg = kPnnTileDefault);
// min_rows: the fewest rows per tile a small batch may be cut to (the tile
// rows anchor each column's walk); carry: keep the corner terms two
// face-adjacent cells share in registers across the step
cudaError_t launch_insert_trilinear(const Volume &v, const void *img, int is_f32, int n, int H,
                                    int W, int convex, double r0, double dr, cudaStream_t st,
                                    const TileCfg &cfg = kTriTileDefault, int min_rows = 8,
                                    bool carry = true);
// fill / project a region: voxels [lo, hi) (clipped to the grid; the fill
// needs lo[0] a multiple of 32), columns [rlo, rhi)
// clear: accumulators to zero in the pass; withhold: test hook (a plane whose
// copy is never issued, so the kernel's bounded wait for it runs out)
cudaError_t launch_fill_pnn(const Volume &v, const int *lo, const int *hi, cudaStream_t st,
                            void *clear = nullptr, int withhold = -1);
cudaError_t launch_fill_trilinear(const Volume &v, const int *lo, const int *hi, cudaStream_t st);
cudaError_t launch_project_u8(const Volume &v, int lo, int hi, const int *rlo, const int *rhi,
                              float *out, uint16_t *cnt, cudaStream_t st);
cudaError_t launch_project_f32(const Volume &v, int lo, int hi, const int *rlo, const int *rhi,
                               float *out, uint16_t *cnt, cudaStream_t st);
cudaError_t launch_zero(void *p, size_t bytes, int num_sms, cudaStream_t st);
cudaError_t launch_red_f2_probe(void *buf, size_t bytes, int reds, int num_sms, cudaStream_t st);
cudaError_t launch_zero_f64(double *p, int n, cudaStream_t st);
cudaError_t launch_soft_project_adjoint(const Volume &v, int lo, int hi, float eps,
                                        const float *target, float *proj, float2 *adj,
                                        double *loss, cudaStream_t st);
cudaError_t launch_pose_grad(const Volume &v, const void *img, int is_f32, int n, int H, int W,
                             int lo, int hi, const float2 *adj, double *grad, cudaStream_t st);
cudaError_t launch_apply_pose_delta(const double *poses, const double *delta, int n, double cx,
                                    double cz, const double *K, double *out, cudaStream_t st);
cudaError_t launch_unpack_mask(const Volume &v, uint8_t *dst, cudaStream_t st);

// Trilinear factors (f, 1 - f) of one axis from the Q.47 fraction bits fr
// (f = fr / 2^47, fr in [0, 2^47)): the smaller of the two, s <= 1/2, is
// converted correctly rounded -- its 46 bits split into two halves of at
// most 23 bits, each made exact in the mantissa of a float, joined by one
// fused multiply-add -- and the larger is 1 - s, rounded.  Both keep a
// relative error below 1.5 * 2^-24, which a small factor needs (the weighted
// mean of a voxel reached only by far corners), and the work stays on the
// integer and FP32 units: a 64-bit integer-to-float conversion runs on the
// FP64 units.
__device__ __forceinline__ void tri_factors(long long fr, float &w1, float &w0)
{
    const unsigned long long p = (unsigned long long)fr & ((1ull << 47) - 1);
    const bool upper = (p >> 46) != 0;                              // f >= 1/2
    const unsigned long long sm = upper ? (1ull << 47) - p : p;     // <= 2^46
    const unsigned hi = (unsigned)(sm >> 23), lo = (unsigned)sm & 0x7FFFFFu;  // hi <= 2^23
    const float fh = __int_as_float(0x4B000000 + (int)hi) - 8388608.0f;
    const float fl = __int_as_float(0x4B000000 + (int)lo) - 8388608.0f;
    const float small = fmaf(fh, 5.9604644775390625e-08f, fl * 7.105427357601002e-15f);
    const float big = 1.0f - small;
    w1 = upper ? big : small;
    w0 = upper ? small : big;
}

// A byte as an exact float: 2^23 + b in the mantissa, minus 2^23.
__device__ __forceinline__ float u8_to_float(unsigned b)
{
    return __int_as_float(0x4B000000 | (int)b) - 8388608.0f;
}

}  // namespace usv
