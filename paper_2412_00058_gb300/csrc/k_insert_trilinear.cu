// A1' (variant): trilinear splatting with the convex-probe scan conversion
// fused into insertion.  The paper reconstructs with PNN (Sec. II.C) after
// weighing it against the distance-weighted methods surveyed by Solberg et
// al.; this is the distance-weighted alternative: every sample spreads its
// intensity over the 8 voxels around its position q with the trilinear
// weights w = prod_a (1 - f_a | f_a), f = q - floor(q), into an FP32
// (S, W) pair per voxel.  Out-of-grid corners and weights below 2^-20 are
// dropped.
//
// Positions: each thread owns one image column j (a beam for a convex
// probe) and walks down its rows, along which the position is affine:
// q(i) = q(i0) + (i - i0)*d.  The start q(i0) is evaluated in FP64 and split
// into an integer voxel and a fraction; the fraction and the step d are then
// carried in Q16.47 fixed point, so after 128 steps the position is still
// within ~1e-12 voxel of the FP64 value, and both trilinear factors of an
// axis, f and 1 - f, are formed from exact integers (no cancellation when f
// is close to 1).  Columns whose step exceeds 256 voxels re-anchor every row.
#include "usv_internal.cuh"

namespace usv {

namespace {

constexpr int kThreads = 256;

struct TriArgs {
    const void *img;
    int is_f32;
    int n, H, W;
    const FrameRec *rec;
    const double2 *beams;
    float2 *acc;
    int nx, ny, nz;
    int convex;
    double r0, dr;
    int th;          // rows per CTA
    int tiles_x;     // column tiles of kThreads columns
};

constexpr long long kOne47 = 1LL << 47;
constexpr long long kMask47 = kOne47 - 1;
constexpr float kInv47 = 7.105427357601002e-15f;  // 2^-47

// q (FP64, |q| < 2^30) -> integer voxel floor(q) and Q16.47 fraction
__device__ __forceinline__ void anchor(double q, int &i0, long long &fq)
{
    const double fl = floor(q);
    i0 = (int)fl;
    fq = __double2ll_rn((q - fl) * 140737488355328.0);  // (q - floor q) * 2^47, exact split
}

__global__ void __launch_bounds__(kThreads) k_insert_trilinear(TriArgs a)
{
    const int tx = blockIdx.x % a.tiles_x, ty = blockIdx.x / a.tiles_x;
    const int j = tx * kThreads + threadIdx.x;
    const int f = blockIdx.y;
    if (j >= a.W)
        return;
    const FrameRec *r = a.rec + f;
    if (!r->valid)
        return;
    const int v0 = ty * a.th, v1 = min(a.H, v0 + a.th);

    // FP64 position of sample (v, j) and its per-row step, per axis
    double base[3], step[3];
    if (a.convex) {
        const double2 sc = a.beams[j];
        for (int ax = 0; ax < 3; ++ax) {
            const double dA = r->d[ax], dB = r->d[3 + ax], C = r->d[6 + ax];
            const double rr = a.r0 + (double)v0 * a.dr;
            base[ax] = C + (rr * sc.x) * dA + (rr * sc.y - a.r0) * dB;
            step[ax] = a.dr * (sc.x * dA + sc.y * dB);
        }
    } else {
        for (int ax = 0; ax < 3; ++ax) {
            base[ax] = r->d[6 + ax] + (double)j * r->d[ax] + (double)v0 * r->d[3 + ax];
            step[ax] = r->d[3 + ax];
        }
    }
    const bool steep = fabs(step[0]) > 256.0 || fabs(step[1]) > 256.0 || fabs(step[2]) > 256.0;
    int i0[3];
    long long fq[3], dq[3];
    for (int ax = 0; ax < 3; ++ax) {
        anchor(base[ax], i0[ax], fq[ax]);
        dq[ax] = __double2ll_rn(step[ax] * 140737488355328.0);
    }
    const size_t fbase = (size_t)f * a.H * a.W;
    const float wmin = 9.5367431640625e-07f;  // 2^-20
    for (int v = v0; v < v1; ++v) {
        if (steep && v > v0)
            for (int ax = 0; ax < 3; ++ax)
                anchor(base[ax] + (double)(v - v0) * step[ax], i0[ax], fq[ax]);
        const size_t pi = fbase + (size_t)v * a.W + j;
        const float I = a.is_f32 ? __ldcs(static_cast<const float *>(a.img) + pi)
                                 : (float)__ldcs(static_cast<const uint8_t *>(a.img) + pi);
        int ix[3];
        float w1[3], w0[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            ix[ax] = i0[ax] + (int)(fq[ax] >> 47);
            const long long fr = fq[ax] & kMask47;
            w1[ax] = __ll2float_rn(fr) * kInv47;
            w0[ax] = __ll2float_rn(kOne47 - fr) * kInv47;
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
            const int X = ix[0] + cx, Y = ix[1] + cy, Z = ix[2] + cz;
            if ((unsigned)X >= (unsigned)a.nx || (unsigned)Y >= (unsigned)a.ny ||
                (unsigned)Z >= (unsigned)a.nz)
                continue;
            const float w = (cx ? w1[0] : w0[0]) * (cy ? w1[1] : w0[1]) * (cz ? w1[2] : w0[2]);
            if (w < wmin)
                continue;
            atomicAdd(a.acc + ((size_t)Z * a.ny + Y) * a.nx + X, make_float2(w * I, w));
        }
        if (!steep) {
            fq[0] += dq[0];
            fq[1] += dq[1];
            fq[2] += dq[2];
        }
    }
}

}  // namespace

cudaError_t launch_insert_trilinear(const Volume &v, const void *img, int is_f32, int n, int H,
                                    int W, int convex, double r0, double dr, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    TriArgs a;
    a.img = img;
    a.is_f32 = is_f32;
    a.n = n;
    a.H = H;
    a.W = W;
    a.rec = v.rec;
    a.beams = v.beams;
    a.acc = static_cast<float2 *>(v.acc);
    a.nx = v.g.nx;
    a.ny = v.g.ny;
    a.nz = v.g.nz;
    a.convex = convex;
    a.r0 = r0;
    a.dr = dr;
    a.th = 128;
    a.tiles_x = (W + kThreads - 1) / kThreads;
    const int tiles_y = (H + a.th - 1) / a.th;
    dim3 grid(a.tiles_x * tiles_y, n);
    k_insert_trilinear<<<grid, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace usv
