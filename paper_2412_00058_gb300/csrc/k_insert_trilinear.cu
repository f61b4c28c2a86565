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
// carried in Q16.47 fixed point, so after 16 steps the position is still
// within ~1e-12 voxel of the FP64 value.  The trilinear factors of an axis,
// f and 1 - f, are formed from that integer fraction with a relative error
// below 1.5 * 2^-24 each (no cancellation when f is close to 1, and no 64-bit
// integer-to-float conversion).  Columns whose step exceeds 256 voxels
// re-anchor every row.
//
// GB300 design: a CTA takes a tile of 256 columns x 64 rows of 4 consecutive
// frames; each thread walks one column through the 64 rows, merging the 8
// corner terms of consecutive samples that stay in one cell (about 1.7
// samples per 0.4 mm cell along a 0.235 mm-step beam) in registers, and
// sends each cell's terms to HBM with one vector atomic (S, W) per corner.
// When the beam steps into a face-adjacent cell, the 4 corner voxels the two
// cells share keep their terms in registers (moved to the new cell's
// corners), and only the 4 corners left behind are sent: about 40 % fewer
// atomics on the convex sweep.  This carry costs work on every cell
// change; it pays where the atomics miss L2, and a launch can leave it out
// (the pose-gradient path, whose smaller volume keeps its atomics in L2).
// A conservative voxel box of the tile (FP64 extremes of the patch -- for a
// convex fan the depth extreme can sit on the central beam -- plus a
// one-voxel margin) decides whether the tile touches the grid at all and
// whether its corners need bounds checks.
//
// Samples: a uint8 sample is always inserted; a float32 sample only if it is
// finite with |I| <= 2^64 (one compare at load; a rejected sample adds no
// weight).  This keeps every register sum of a column walk finite, so the
// 0/1-mask carry below never multiplies an infinity by zero.
#include <cfloat>
#include <climits>

#include "usv_internal.cuh"

namespace usv {

namespace {

constexpr int kThreads = 256;
constexpr int kCols = 256;                   // columns per tile (one per thread)
constexpr int kMaxFpc = 8;                   // frames per CTA, at most

struct TriArgs {
    const void *img;
    int is_f32;
    int n, H, W;
    const FrameRec *rec;
    const double2 *beams;
    float2 *acc;
    uint32_t *status;  // checked build: USV_STATUS_OOB
    int nx, ny, nz;
    int convex;
    double r0, dr;
    int tiles_x;     // column tiles
    int rows;        // rows per tile
    int fpc;         // frames per CTA
};

constexpr long long kOne47 = 1LL << 47;
constexpr long long kMask47 = kOne47 - 1;
constexpr float kWmin = 9.5367431640625e-07f;     // 2^-20
constexpr float kMaxSample = 18446744073709551616.0f;  // 2^64: larger |I| is not inserted

// q (FP64, |q| < 2^30) -> integer voxel floor(q) and Q16.47 fraction
__device__ __forceinline__ void anchor(double q, int &i0, long long &fq)
{
    const double fl = floor(q);
    i0 = (int)fl;
    fq = __double2ll_rn((q - fl) * 140737488355328.0);  // (q - floor q) * 2^47
}

// FP64 position (voxel units) of sample (row v, column j) of frame r, and
// its per-row step.
__device__ __forceinline__ void sample_line(const TriArgs &a, const FrameRec *r, int j, int v,
                                            double (&base)[3], double (&step)[3])
{
    if (a.convex) {
        const double2 sc = a.beams[j];
        const double rr = a.r0 + (double)v * a.dr;
        for (int ax = 0; ax < 3; ++ax) {
            const double dA = r->d[ax], dB = r->d[3 + ax], C = r->d[6 + ax];
            base[ax] = C + (rr * sc.x) * dA + (rr * sc.y - a.r0) * dB;
            step[ax] = a.dr * (sc.x * dA + sc.y * dB);
        }
    } else {
        for (int ax = 0; ax < 3; ++ax) {
            base[ax] = r->d[6 + ax] + (double)j * r->d[ax] + (double)v * r->d[3 + ax];
            step[ax] = r->d[3 + ax];
        }
    }
}

// Conservative voxel range of frame r's samples in columns [j0, j1) x rows
// [v0, v1): the in-plane (x, z) extremes of the patch, mapped through the
// affine per-mm (convex) or per-pixel (linear) map.
__device__ void patch_box(const TriArgs &a, const FrameRec *r, int j0, int j1, int v0, int v1,
                          double (&lo)[3], double (&hi)[3])
{
    double xs[2], zs[2];
    if (a.convex) {
        const double ra = a.r0 + (double)v0 * a.dr, rb = a.r0 + (double)(v1 - 1) * a.dr;
        const double2 sa = a.beams[j0], sb = a.beams[j1 - 1];
        // x = r sin(theta): monotone in theta, extremes at corners
        const double x1 = ra * sa.x, x2 = rb * sa.x, x3 = ra * sb.x, x4 = rb * sb.x;
        xs[0] = fmin(fmin(x1, x2), fmin(x3, x4));
        xs[1] = fmax(fmax(x1, x2), fmax(x3, x4));
        // z = r cos(theta) - r0: minimum at a corner, maximum on the central
        // beam if the patch straddles it
        const double cmin = fmin(sa.y, sb.y);
        const double cmax = (sa.x <= 0.0 && sb.x >= 0.0) ? 1.0 : fmax(sa.y, sb.y);
        zs[0] = ra * cmin - a.r0;
        zs[1] = rb * cmax - a.r0;
    } else {
        xs[0] = (double)j0;  // linear: the map is per pixel, (u, v) directly
        xs[1] = (double)(j1 - 1);
        zs[0] = (double)v0;
        zs[1] = (double)(v1 - 1);
    }
    for (int ax = 0; ax < 3; ++ax) {
        lo[ax] = DBL_MAX;
        hi[ax] = -DBL_MAX;
        for (int c = 0; c < 4; ++c) {
            const double q = r->d[6 + ax] + xs[c & 1] * r->d[ax] + zs[c >> 1] * r->d[3 + ax];
            lo[ax] = fmin(lo[ax], q);
            hi[ax] = fmax(hi[ax], q);
        }
    }
}

// Corners of a cell that a step to a face-adjacent cell leaves behind, as
// a bit mask over the 8 corners (bit c: corner c): the step moves by one
// along the axis of corner bit `abit`, up or down; moving up, the corners
// with that bit clear stay behind (the others become the new cell's corners
// with the bit clear), moving down the corners with the bit set.  Any other
// step (or the end of a column) leaves all 8 behind.
__device__ __forceinline__ unsigned left_behind(bool face, int abit, bool up)
{
    if (!face)
        return 0xFFu;
    const unsigned clear = abit == 1 ? 0x55u : abit == 2 ? 0x33u : 0x0Fu;
    return up ? clear : 0xFFu & ~clear;
}

// Send the corners in `send` of the cell at (lx, ly, lz) to HBM, one vector
// atomic (S, W) per corner that holds a term.  The corner addresses are the
// cell's base offset plus 0 or 1 entry, the row pitch and the plane pitch,
// formed once per cell; in tiles the grid clips, corners outside it are
// dropped by one mask per axis.
template <bool CHECK>
__device__ __forceinline__ void splat(float2 *acc, uint32_t *status, unsigned ex, unsigned ey,
                                      unsigned ez, int lx, int ly, int lz, const float (&cS)[8],
                                      const float (&cW)[8], unsigned send = 0xFFu)
{
    if (CHECK) {
        const unsigned okx = ((unsigned)lx < ex ? 0x55u : 0u) | ((unsigned)(lx + 1) < ex ? 0xAAu : 0u);
        const unsigned oky = ((unsigned)ly < ey ? 0x33u : 0u) | ((unsigned)(ly + 1) < ey ? 0xCCu : 0u);
        const unsigned okz = ((unsigned)lz < ez ? 0x0Fu : 0u) | ((unsigned)(lz + 1) < ez ? 0xF0u : 0u);
        send &= okx & oky & okz;
    }
    // entry offsets of corner 0 and of the +y, +z and +y+z corners (signed:
    // in a clipped tile corner 0 itself may lie outside the grid)
    const long long plane = (long long)ex * ey;
    const long long i0 = ((long long)lz * ey + ly) * (long long)ex + lx;
    const long long off[4] = {i0, i0 + ex, i0 + plane, i0 + plane + ex};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long i = off[c >> 1] + (c & 1);
        const bool go = ((send >> c) & 1u) && cW[c] != 0.0f;
        if constexpr (kChecked) {
            const unsigned X = (unsigned)(lx + (c & 1)), Y = (unsigned)(ly + ((c >> 1) & 1)),
                           Z = (unsigned)(lz + (c >> 2));
            if (go && !(guard(X, ex, status) && guard(Y, ey, status) && guard(Z, ez, status)))
                continue;
        }
        if (go)
            atomicAdd(acc + i, make_float2(cS[c], cW[c]));
    }
}

template <bool CHECK, bool CARRY>
__device__ __forceinline__ void walk(const TriArgs &a, const FrameRec *recs, int f0, int f1,
                                     int j, int v0, int v1, unsigned ex, unsigned ey,
                                     unsigned ez)
{
    for (int f = f0; f < f1; ++f) {
        const FrameRec *r = recs + (f - f0);
        if (!r->valid)
            continue;
        const int vs = max(v0, r->first_row);  // rows above the cut are not inserted
        if (vs >= v1)
            continue;
        double base[3], step[3];
        sample_line(a, r, j, vs, base, step);
        const bool steep =
            fabs(step[0]) > 256.0 || fabs(step[1]) > 256.0 || fabs(step[2]) > 256.0;
        int i0[3];
        long long fq[3], dq[3];
        for (int ax = 0; ax < 3; ++ax) {
            anchor(base[ax], i0[ax], fq[ax]);
            dq[ax] = __double2ll_rn(step[ax] * 140737488355328.0);
        }
        const size_t fbase = (size_t)f * a.H * a.W;
        // register accumulation of the current cell's 8 corner terms
        float cS[8], cW[8];
#pragma unroll
        for (int c = 0; c < 8; ++c)
            cS[c] = cW[c] = 0.0f;
        int cx0 = INT_MIN, cy0 = 0, cz0 = 0;
        // the next row's sample is loaded while this row is splatted
        auto sample = [&](int v) {
            const size_t pi = fbase + (size_t)v * a.W + j;
            return a.is_f32 ? __ldcs(static_cast<const float *>(a.img) + pi)
                            : u8_to_float(__ldcs(static_cast<const uint8_t *>(a.img) + pi));
        };
        float In = sample(vs);
        for (int v = vs; v < v1; ++v) {
            if (steep && v > vs)
                for (int ax = 0; ax < 3; ++ax)
                    anchor(base[ax] + (double)(v - vs) * step[ax], i0[ax], fq[ax]);
            const float I = In;
            if (v + 1 < v1)
                In = sample(v + 1);
            // a float32 sample that is not finite or exceeds 2^64 is not
            // inserted (uint8 samples always pass)
            const bool admit = fabsf(I) <= kMaxSample;
            int ix[3];
            float w1[3], w0[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                ix[ax] = i0[ax] + (int)(fq[ax] >> 47);
                const long long fr = fq[ax] & kMask47;
                tri_factors(fr, w1[ax], w0[ax]);
            }
            if (ix[0] != cx0 || ix[1] != cy0 || ix[2] != cz0) {
                // a step to a face-adjacent cell keeps the 4 corner voxels the
                // two cells share: their terms move to the new cell's corners
                // and go out with it; only the corners left behind are sent
                // (unsigned differences: the first cell's INT_MIN must not overflow)
                const int dx = (int)((unsigned)ix[0] - (unsigned)cx0);
                const int dy = (int)((unsigned)ix[1] - (unsigned)cy0);
                const int dz = (int)((unsigned)ix[2] - (unsigned)cz0);
                const bool face = CARRY && cx0 != INT_MIN && abs(dx) + abs(dy) + abs(dz) == 1;
                const int abit = dx != 0 ? 1 : dy != 0 ? 2 : 4;
                const bool up = dx + dy + dz > 0;
                if (cx0 != INT_MIN)
                    splat<CHECK>(a.acc, a.status, ex, ey, ez, cx0, cy0, cz0, cS, cW,
                                 left_behind(face, abit, up));
                // new corner c is old corner c ^ abit when it receives: 0/1
                // masks and multiply-adds (exact: one term is kept, the others
                // are multiplied by zero) keep this off the integer pipe
                if constexpr (CARRY) {
                    // receiving along axis bit b: the corners with b clear
                    // on a step up, with b set on a step down -- fixed per
                    // corner, so one mask per axis and direction
                    const float xl = face && abit == 1 && up ? 1.0f : 0.0f;
                    const float xh = face && abit == 1 && !up ? 1.0f : 0.0f;
                    const float yl = face && abit == 2 && up ? 1.0f : 0.0f;
                    const float yh = face && abit == 2 && !up ? 1.0f : 0.0f;
                    const float zl = face && abit == 4 && up ? 1.0f : 0.0f;
                    const float zh = face && abit == 4 && !up ? 1.0f : 0.0f;
                    float nS[8], nW[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float kx = (c & 1) ? xh : xl, ky = (c & 2) ? yh : yl;
                        const float kz = (c & 4) ? zh : zl;
                        nS[c] = fmaf(kx, cS[c ^ 1], fmaf(ky, cS[c ^ 2], kz * cS[c ^ 4]));
                        nW[c] = fmaf(kx, cW[c ^ 1], fmaf(ky, cW[c ^ 2], kz * cW[c ^ 4]));
                    }
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        cS[c] = nS[c];
                        cW[c] = nW[c];
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        cS[c] = cW[c] = 0.0f;
                }
                cx0 = ix[0];
                cy0 = ix[1];
                cz0 = ix[2];
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float w = ((c & 1) ? w1[0] : w0[0]) * (((c >> 1) & 1) ? w1[1] : w0[1]) *
                                ((c >> 2) ? w1[2] : w0[2]);
                if (admit && w >= kWmin) {
                    cS[c] += w * I;
                    cW[c] += w;
                }
            }
            if (!steep) {
                fq[0] += dq[0];
                fq[1] += dq[1];
                fq[2] += dq[2];
            }
        }
        if (cx0 != INT_MIN)
            splat<CHECK>(a.acc, a.status, ex, ey, ez, cx0, cy0, cz0, cS, cW);
    }
}

template <bool CARRY>
__global__ void __launch_bounds__(kThreads, 3) k_insert_trilinear(TriArgs a)
{
    __shared__ FrameRec s_rec[kMaxFpc];
    __shared__ int s_mode, s_check;
    const int tx = blockIdx.x % a.tiles_x, ty = blockIdx.x / a.tiles_x;
    const int j0 = tx * kCols, j1 = min(a.W, j0 + kCols);
    const int v0 = ty * a.rows, v1 = min(a.H, v0 + a.rows);
    const int f0 = blockIdx.y * a.fpc, f1 = min(a.n, f0 + a.fpc);

    for (int i = threadIdx.x; i < (f1 - f0) * (int)(sizeof(FrameRec) / 8); i += kThreads)
        reinterpret_cast<unsigned long long *>(s_rec)[i] =
            reinterpret_cast<const unsigned long long *>(a.rec + f0)[i];
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
        int any = 0;
        if (lane < f1 - f0 && s_rec[lane].valid) {
            patch_box(a, s_rec + lane, j0, j1, v0, v1, lo, hi);
            any = 1;
        }
        // reduce over the frames (lanes)
        for (int off = 16; off > 0; off >>= 1) {
            any |= __shfl_xor_sync(0xFFFFFFFFu, any, off);
            for (int ax = 0; ax < 3; ++ax) {
                lo[ax] = fmin(lo[ax], __shfl_xor_sync(0xFFFFFFFFu, lo[ax], off));
                hi[ax] = fmax(hi[ax], __shfl_xor_sync(0xFFFFFFFFu, hi[ax], off));
            }
        }
        if (lane == 0) {
            int mode = 0, check = 0;
            if (any) {
                const int n[3] = {a.nx, a.ny, a.nz};
                mode = 1;
                for (int ax = 0; ax < 3; ++ax) {
                    // corners reach floor(q) + 1; one voxel of margin each side
                    const long long l0 = (long long)floor(lo[ax]) - 1;
                    const long long h0 = (long long)floor(hi[ax]) + 2;
                    const long long l = l0 < 0 ? 0 : l0, h = h0 > n[ax] - 1 ? n[ax] - 1 : h0;
                    if (l > h)
                        mode = 0;
                    if (l != l0 || h != h0)
                        check = 1;
                }
            }
            s_mode = mode;
            s_check = check;
        }
    }
    __syncthreads();
    if (s_mode == 0)
        return;
    const int j = j0 + threadIdx.x;
    // corner bounds checks only in tiles whose voxel box the grid clips
    if (j < j1 && v0 < v1) {
        if (s_check)
            walk<true, CARRY>(a, s_rec, f0, f1, j, v0, v1, (unsigned)a.nx, (unsigned)a.ny,
                              (unsigned)a.nz);
        else
            walk<false, CARRY>(a, s_rec, f0, f1, j, v0, v1, (unsigned)a.nx, (unsigned)a.ny,
                               (unsigned)a.nz);
    }
}

}  // namespace

// A column walks at most tile_h rows from its anchor with steps below 256
// voxels, so the Q16.47 position stays below 128 * 256 = 2^15 voxels (no
// overflow of the 64-bit fraction) and drifts by under 2^-41 voxel.
bool tri_tile_ok(const TileCfg &c)
{
    return c.tile_w == kCols && c.tile_h >= 1 && c.tile_h <= 128 && c.frames_per_cta >= 1 &&
           c.frames_per_cta <= kMaxFpc;
}

cudaError_t launch_insert_trilinear(const Volume &v, const void *img, int is_f32, int n, int H,
                                    int W, int convex, double r0, double dr, cudaStream_t st,
                                    const TileCfg &cfg, int min_rows, bool carry)
{
    if (n <= 0)
        return cudaSuccess;
    if (!tri_tile_ok(cfg))
        return cudaErrorInvalidValue;
    TriArgs a;
    a.img = img;
    a.is_f32 = is_f32;
    a.n = n;
    a.H = H;
    a.W = W;
    a.rec = v.rec;
    a.beams = v.beams;
    a.acc = static_cast<float2 *>(v.acc);
    a.status = v.status;
    a.nx = v.g.nx;
    a.ny = v.g.ny;
    a.nz = v.g.nz;
    a.convex = convex;
    a.r0 = r0;
    a.dr = dr;
    a.tiles_x = (W + kCols - 1) / kCols;
    a.rows = cfg.tile_h;
    a.fpc = cfg.frames_per_cta;
    // a batch too small to fill the GPU's resident blocks (3 per SM at this
    // kernel's registers) takes fewer frames per block, then fewer rows per
    // tile (down to max(8, min_rows)), so that more blocks share it.  The
    // tile rows fix where each column's walk is anchored, so callers that
    // must reproduce the positions (the pose gradient) keep them.
    const int floor_rows = min_rows > 8 ? min_rows : 8;
    const long long resident = (long long)v.num_sms * 3;
    auto blocks = [&] {
        return (long long)a.tiles_x * ((H + a.rows - 1) / a.rows) * ((n + a.fpc - 1) / a.fpc);
    };
    while (blocks() < resident && (a.fpc > 1 || a.rows > floor_rows)) {
        if (a.fpc > 1)
            a.fpc = (a.fpc + 1) / 2;
        else
            a.rows = (a.rows + 1) / 2 < floor_rows ? floor_rows : (a.rows + 1) / 2;
    }
    const int tiles_y = (H + a.rows - 1) / a.rows;
    const long long groups = (n + a.fpc - 1) / a.fpc;
    if (groups > 65535)
        return cudaErrorInvalidConfiguration;
    dim3 grid(a.tiles_x * tiles_y, (unsigned)groups);
    if (carry)
        k_insert_trilinear<true><<<grid, kThreads, 0, st>>>(a);
    else
        k_insert_trilinear<false><<<grid, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace usv
