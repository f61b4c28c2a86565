// Tissue segmentation by depth of cut (the paper's Algorithms 1 and 2): per
// frame, the first image row that is inserted; rows above it (superficial
// tissue over the bone) are cut away by the insertion kernels.
//
// Algorithm 1 (real-time, Table I): the cut depth follows the probe's
// position along the spine,
//     Cut_n = K * |P_c1.x - P_cn.x - L/2| + D,
// where P_cn is the position of frame n's upper-left pixel and .x the
// coordinate along the spine (Alg. 1 steps 2-4).  Evaluated in FP64 with
// separately rounded operations in a fixed order:
//   p_a   = M[a][3] of M = pose * K (as in the set-up kernel),
//   d     = ((p1_x - p_x) * e_x + (p1_y - p_y) * e_y) + (p1_z - p_z) * e_z,
//   cut   = k * |d - L/2| + D   (mm),   row = ceil(cut / row_mm), clamped to [0, H].
//
// Algorithm 2 (post-acquisition, Table II): in the lower part of each frame
// find the contour with a large intensity drop and a bright value (the bone
// cortex is bright and shadows what lies below it), take its depth per
// frame, median-filter the depths over the frames, cut there.  Integer
// arithmetic:
//   score(v, u) = I(v, u) * max(0, I(v, u) - I(v + drop, u))  for v in [from, H - drop)
//   b(u)  = first v of the maximum score (from if every score is 0)
//   b_n   = lower median of b(u) over the columns of frame n
//   m_n   = lower median of b_k over k in [n - w/2, n + w/2] clipped to the scan
//   row_n = max(0, m_n - margin).
#include "usv_internal.cuh"

namespace usv {

namespace {

__global__ void k_cut_rows_alg1(const double *__restrict__ poses, int n, int H, Alg1Params p,
                                int32_t *__restrict__ rows)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n)
        return;
    const double *P = poses + (size_t)f * 16;
    double pos[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double acc = __dmul_rn(P[a * 4 + 0], p.K[0 * 4 + 3]);
        acc = __dadd_rn(acc, __dmul_rn(P[a * 4 + 1], p.K[1 * 4 + 3]));
        acc = __dadd_rn(acc, __dmul_rn(P[a * 4 + 2], p.K[2 * 4 + 3]));
        acc = __dadd_rn(acc, __dmul_rn(P[a * 4 + 3], p.K[3 * 4 + 3]));
        pos[a] = acc;
    }
    double d = __dmul_rn(__dsub_rn(p.p1[0], pos[0]), p.dir[0]);
    d = __dadd_rn(d, __dmul_rn(__dsub_rn(p.p1[1], pos[1]), p.dir[1]));
    d = __dadd_rn(d, __dmul_rn(__dsub_rn(p.p1[2], pos[2]), p.dir[2]));
    const double cut = __dadd_rn(__dmul_rn(p.k, fabs(__dsub_rn(d, p.half_l_mm))), p.d_mm);
    const double row = ceil(__ddiv_rn(cut, p.row_mm));
    int r;
    if (!(row > 0.0))  // also NaN
        r = 0;
    else if (row >= (double)H)
        r = H;
    else
        r = (int)row;
    rows[f] = r;
}

constexpr int kBoneThreads = 256;
constexpr int kMaxBoneH = 8192;

// one CTA per frame: per-column contour row, then the lower median over
// the columns from a histogram of rows
__global__ void __launch_bounds__(kBoneThreads) k_bone_rows(const uint8_t *__restrict__ img,
                                                            int H, int W, int from, int drop,
                                                            int32_t *__restrict__ bone)
{
    __shared__ unsigned hist[kMaxBoneH];
    __shared__ int s_med;
    const int f = blockIdx.x;
    for (int i = threadIdx.x; i < H; i += kBoneThreads)
        hist[i] = 0u;
    __syncthreads();
    const uint8_t *fr = img + (size_t)f * H * W;
    for (int u = threadIdx.x; u < W; u += kBoneThreads) {
        int best = -1, brow = from;
        for (int v = from; v + drop < H; ++v) {
            const int a = fr[(size_t)v * W + u], b = fr[(size_t)(v + drop) * W + u];
            const int s = a * (a > b ? a - b : 0);
            if (s > best) {
                best = s;
                brow = v;
            }
        }
        if (best <= 0)
            brow = from;
        atomicAdd(&hist[brow], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned m = (unsigned)(W - 1) / 2;  // lower median: m-th smallest (0-based)
        unsigned acc = 0;
        int med = 0;
        for (int v = 0; v < H; ++v) {
            acc += hist[v];
            if (acc > m) {
                med = v;
                break;
            }
        }
        s_med = med;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        bone[f] = s_med;
}

// lower median of bone[k] over the window around each frame, minus margin
__global__ void k_bone_filter(const int32_t *__restrict__ bone, int n, int half, int margin,
                              int32_t *__restrict__ rows)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n)
        return;
    const int k0 = max(0, f - half), k1 = min(n - 1, f + half);
    const int len = k1 - k0 + 1, m = (len - 1) / 2;
    int med = bone[f];
    for (int i = k0; i <= k1; ++i) {
        const int e = bone[i];
        int less = 0, le = 0;
        for (int k = k0; k <= k1; ++k) {
            less += bone[k] < e;
            le += bone[k] <= e;
        }
        if (less <= m && m < le) {
            med = e;
            break;
        }
    }
    rows[f] = max(0, med - margin);
}

}  // namespace

cudaError_t launch_cut_rows_alg1(const double *poses, int n, int H, const Alg1Params &p,
                                 int32_t *first_rows, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_cut_rows_alg1<<<(n + 127) / 128, 128, 0, st>>>(poses, n, H, p, first_rows);
    return cudaGetLastError();
}

cudaError_t launch_bone_rows_alg2(const uint8_t *img, int n, int H, int W, int from_row, int drop,
                                  int window, int margin, int32_t *bone_rows, int32_t *first_rows,
                                  cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    if (H > kMaxBoneH)
        return cudaErrorInvalidValue;
    k_bone_rows<<<n, kBoneThreads, 0, st>>>(img, H, W, from_row, drop, bone_rows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    k_bone_filter<<<(n + 127) / 128, 128, 0, st>>>(bone_rows, n, window / 2, margin, first_rows);
    return cudaGetLastError();
}

}  // namespace usv
