/*
 * CPU ORACLE for the free-hand ultrasound volume path -- TEST INFRASTRUCTURE.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py (cpu_baseline leg and the
 * reference arm) may load this file.  The product path (the CUDA library
 * under paper_2412_00058_gb300/) never calls it and shares no code with it.
 *
 * Plain, slow, obviously-correct C in FP64 / exact integers.  One function
 * per step of the path, each following the definition it cites:
 *
 *   ora_frame_affine_q32   per-frame pixel->voxel affine map (Alg. 1 steps
 *                          2, 3, 6: a pixel is carried into the reference
 *                          frame by the tracked transform T_T^W applied after
 *                          the image calibration), quantised to Q31.32.
 *   ora_insert_pnn         pixel-nearest-neighbour insertion (Sec. II.C: PNN
 *                          after Solberg et al.; every pixel goes to its
 *                          nearest voxel, which accumulates intensity and a
 *                          hit count).
 *   ora_fill_pnn           normalisation (bin value = sum / count) and the
 *                          3x3x3 hole-filling pass of PNN (Sec. II.C, PNN's
 *                          second stage).
 *   ora_project_u8         depth-band projection, the VPI spine view at a
 *                          fixed depth (Sec. III.B, Fig. 6).
 *   ora_insert_trilinear   distance-weighted (trilinear) splatting variant,
 *   ora_fill_trilinear     its normalisation + hole fill, and
 *   ora_project_f64        its depth-band projection, all in FP64.
 *   ora_cut_rows_alg1      Algorithm 1 (real-time depth of cut from the
 *                          probe position along the spine, Table I).
 *   ora_bone_rows_alg2     Algorithm 2 (depth of cut from the bone contour
 *                          and a median filter over frames, Table II).
 *   ora_insert_pnn_rows    PNN insertion of the rows below each frame's
 *   ora_insert_trilinear_rows  depth of cut (Alg. 1 step 5-6, Alg. 2 4-5).
 *
 * Where the paper is silent the reading taken is stated at the function.
 * Build with -ffp-contract=off: the affine set-up is defined as separately
 * rounded IEEE multiplies and adds (no fused multiply-add).
 */
#include "usv_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO32 4294967296.0

/* Host threads for the multi-core forms (ora_insert_pnn_rows_mt, and the
 * fill and projection loops, which split their independent outputs).  1
 * (the default) runs everything on the calling thread, exactly the plain
 * loops below.  Without OpenMP the count stays 1. */
static int g_threads = 1;

int ora_set_threads(int n)
{
#ifdef _OPENMP
    g_threads = n < 1 ? 1 : n;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

/* Round half away from zero, exactly.  x - trunc(x) is exact in binary
 * floating point, so the comparison with 0.5 decides the tie rule. */
int64_t ora_round_half_away(double x)
{
    double t = trunc(x);
    double r = x - t;
    if (r >= 0.5)
        t += 1.0;
    else if (r <= -0.5)
        t -= 1.0;
    return (int64_t)t;
}

/* floor(a / b) for b > 0, written out (C division truncates toward zero). */
static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0)
        q -= 1;
    return q;
}

/* M = P * K restricted to the top three rows; every entry is the four
 * products summed left to right, each operation rounded (no FMA). */
static void pose_times_calib(const double P[16], const double K[16], double M[3][4])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 4; ++j) {
            double acc = P[i * 4 + 0] * K[0 * 4 + j];
            acc = acc + P[i * 4 + 1] * K[1 * 4 + j];
            acc = acc + P[i * 4 + 2] * K[2 * 4 + j];
            acc = acc + P[i * 4 + 3] * K[3 * 4 + j];
            M[i][j] = acc;
        }
}

/*
 * Per-frame affine map from pixel (u, v) to continuous voxel coordinates
 *     q(u, v) = C + u*A + v*B
 * where the world point of the pixel is p = P K (u*sx, 0, v*sy, 1)^T
 * (Alg. 1 steps 2-3 and 6: the image point is carried to the world by the
 * calibration and the tracked probe pose T_T^W) and q = (p - origin)/spacing:
 *     A_a = (M[a][0]*sx)/s_a,  B_a = (M[a][2]*sy)/s_a,  C_a = (M[a][3]-o_a)/s_a.
 * The nine values are quantised to Q31.32 (round half away from zero of
 * value * 2^32).  coef = {A_x,A_y,A_z, B_x,B_y,B_z, C_x,C_y,C_z}.
 *
 * Reading (the paper fixes no precision): the quantised map *defines* the
 * nearest-neighbour result.  A frame is valid iff the pose's bottom row is
 * exactly (0,0,0,1), all nine values are finite, |A_a| < 2^14, |B_a| < 2^14
 * and |C_a| < 2^29; invalid frames are skipped.  Returns 1 if valid.
 */
int ora_frame_affine_q32(const double P[16], const double K[16], double sx, double sy,
                         const double spacing[3], const double origin[3], int64_t coef[9])
{
    double M[3][4];
    double A[3], B[3], C[3];
    int ok = P[12] == 0.0 && P[13] == 0.0 && P[14] == 0.0 && P[15] == 1.0;
    pose_times_calib(P, K, M);
    for (int a = 0; a < 3; ++a) {
        A[a] = (M[a][0] * sx) / spacing[a];
        B[a] = (M[a][2] * sy) / spacing[a];
        C[a] = (M[a][3] - origin[a]) / spacing[a];
        if (!isfinite(A[a]) || !isfinite(B[a]) || !isfinite(C[a]))
            ok = 0;
        else if (fabs(A[a]) >= 16384.0 || fabs(B[a]) >= 16384.0 || fabs(C[a]) >= 536870912.0)
            ok = 0;
    }
    for (int a = 0; a < 3; ++a) {
        coef[a] = ok ? ora_round_half_away(A[a] * TWO32) : 0;
        coef[3 + a] = ok ? ora_round_half_away(B[a] * TWO32) : 0;
        coef[6 + a] = ok ? ora_round_half_away(C[a] * TWO32) : 0;
    }
    return ok;
}

/*
 * PNN insertion (Sec. II.C).  For every pixel of every valid frame:
 *   Q_a = C_a + u*A_a + v*B_a                (exact int64, Q31.32)
 *   i_a = floor((Q_a + 2^31) / 2^32)        (nearest voxel; ties go up)
 * and if 0 <= i_a < n_a on all axes, sum[i] += I(u, v) and cnt[i] += 1.
 * Every pixel is inserted, zeros included.  Volume order [nz][ny][nx].
 * Returns the number of frames skipped as invalid.
 */
int64_t ora_insert_pnn(uint64_t *sum, uint32_t *cnt, int nx, int ny, int nz,
                       const uint8_t *images, int n, int H, int W, const double *poses,
                       const double K[16], double sx, double sy,
                       const double spacing[3], const double origin[3])
{
    return ora_insert_pnn_rows(sum, cnt, nx, ny, nz, images, n, H, W, poses, K, sx, sy, spacing,
                               origin, 0);
}

/* As ora_insert_pnn, inserting only rows v >= first_rows[f] of frame f
 * (all rows if first_rows is NULL): the image below the depth of cut. */
int64_t ora_insert_pnn_rows(uint64_t *sum, uint32_t *cnt, int nx, int ny, int nz,
                            const uint8_t *images, int n, int H, int W, const double *poses,
                            const double K[16], double sx, double sy,
                            const double spacing[3], const double origin[3],
                            const int32_t *first_rows)
{
    int64_t skipped = 0;
    const int64_t half = (int64_t)1 << 31;
    const int64_t one = (int64_t)1 << 32;
    for (int f = 0; f < n; ++f) {
        int64_t c[9];
        if (!ora_frame_affine_q32(poses + (size_t)f * 16, K, sx, sy, spacing, origin, c)) {
            ++skipped;
            continue;
        }
        const uint8_t *img = images + (size_t)f * H * W;
        const int v_first = first_rows ? (first_rows[f] > 0 ? first_rows[f] : 0) : 0;
        for (int v = v_first; v < H; ++v)
            for (int u = 0; u < W; ++u) {
                int64_t idx[3];
                for (int a = 0; a < 3; ++a) {
                    int64_t Q = c[6 + a] + (int64_t)u * c[a] + (int64_t)v * c[3 + a];
                    idx[a] = floor_div(Q + half, one);
                }
                if (idx[0] < 0 || idx[0] >= nx || idx[1] < 0 || idx[1] >= ny || idx[2] < 0 ||
                    idx[2] >= nz)
                    continue;
                size_t lin = ((size_t)idx[2] * ny + (size_t)idx[1]) * nx + (size_t)idx[0];
                sum[lin] += img[(size_t)v * W + u];
                cnt[lin] += 1;
            }
    }
    return skipped;
}

/* ora_insert_pnn_rows on g_threads host threads: the frames are split into
 * contiguous ranges and every accumulator update is an atomic integer add,
 * so the result is the same bits as the plain loop whatever the order. */
int64_t ora_insert_pnn_rows_mt(uint64_t *sum, uint32_t *cnt, int nx, int ny, int nz,
                               const uint8_t *images, int n, int H, int W, const double *poses,
                               const double K[16], double sx, double sy,
                               const double spacing[3], const double origin[3],
                               const int32_t *first_rows)
{
    int64_t skipped = 0;
    const int64_t half = (int64_t)1 << 31;
    const int64_t one = (int64_t)1 << 32;
#pragma omp parallel for schedule(static) num_threads(g_threads) reduction(+ : skipped)
    for (int f = 0; f < n; ++f) {
        int64_t c[9];
        if (!ora_frame_affine_q32(poses + (size_t)f * 16, K, sx, sy, spacing, origin, c)) {
            ++skipped;
            continue;
        }
        const uint8_t *img = images + (size_t)f * H * W;
        const int v_first = first_rows ? (first_rows[f] > 0 ? first_rows[f] : 0) : 0;
        for (int v = v_first; v < H; ++v)
            for (int u = 0; u < W; ++u) {
                int64_t idx[3];
                for (int a = 0; a < 3; ++a) {
                    int64_t Q = c[6 + a] + (int64_t)u * c[a] + (int64_t)v * c[3 + a];
                    idx[a] = floor_div(Q + half, one);
                }
                if (idx[0] < 0 || idx[0] >= nx || idx[1] < 0 || idx[1] >= ny || idx[2] < 0 ||
                    idx[2] >= nz)
                    continue;
                size_t lin = ((size_t)idx[2] * ny + (size_t)idx[1]) * nx + (size_t)idx[0];
                const uint64_t I = img[(size_t)v * W + u];
#pragma omp atomic
                sum[lin] += I;
#pragma omp atomic
                cnt[lin] += 1;
            }
    }
    return skipped;
}

/* round-half-up mean of integer data: floor(s/c + 1/2) = (2s + c) / (2c) */
static uint8_t mean_u8(uint64_t s, uint64_t c)
{
    uint64_t q = (2 * s + c) / (2 * c);
    return (uint8_t)(q > 255 ? 255 : q);
}

/*
 * Normalisation and 3x3x3 hole filling for PNN (Sec. II.C: PNN's bin
 * value is the mean of the pixels that fell into it; empty bins are then
 * filled from their neighbourhood).  Reading: one pass that reads only the
 * accumulators; an empty voxel takes the pooled, count-weighted mean
 * (sum of neighbour sums over sum of neighbour counts) of its non-empty
 * in-grid neighbours among the 26; with none it stays empty (has = 0,
 * val = 0).  Means round half up.
 */
void ora_fill_pnn(const uint64_t *sum, const uint32_t *cnt, int nx, int ny, int nz,
                  uint8_t *val, uint8_t *has)
{
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = ((size_t)z * ny + y) * nx + x;
                if (cnt[i] > 0) {
                    val[i] = mean_u8(sum[i], cnt[i]);
                    has[i] = 1;
                    continue;
                }
                uint64_t S = 0, C = 0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (dx == 0 && dy == 0 && dz == 0)
                                continue;
                            int X = x + dx, Y = y + dy, Z = z + dz;
                            if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz)
                                continue;
                            size_t j = ((size_t)Z * ny + Y) * nx + X;
                            if (cnt[j] > 0) {
                                S += sum[j];
                                C += cnt[j];
                            }
                        }
                if (C > 0) {
                    val[i] = mean_u8(S, C);
                    has[i] = 1;
                } else {
                    val[i] = 0;
                    has[i] = 0;
                }
            }
}

/*
 * Depth-band projection (the VPI view at a fixed depth, Sec. III.B).
 * Reading: for every (x, y) the mean of the has-data voxels with z in the
 * half-open band [lo, hi), as a float (0 where there are none); cnt gets the
 * number of voxels averaged.
 */
void ora_project_u8(const uint8_t *val, const uint8_t *has, int nx, int ny, int nz, int lo,
                    int hi, float *out, uint16_t *cnt)
{
    (void)nz;
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            uint64_t s = 0, c = 0;
            for (int z = lo; z < hi; ++z) {
                size_t i = ((size_t)z * ny + y) * nx + x;
                if (has[i]) {
                    s += val[i];
                    c += 1;
                }
            }
            out[(size_t)y * nx + x] = c ? (float)((double)s / (double)c) : 0.0f;
            if (cnt)
                cnt[(size_t)y * nx + x] = (uint16_t)c;
        }
}

/* ------------------------------------------------------------------------- */
/* Trilinear (distance-weighted) variant, FP64 throughout.                    */
/* ------------------------------------------------------------------------- */

/*
 * In-plane point (mm, image frame) of sample (row i, column j).
 *   linear: (j*sx, 0, i*sy)
 *   convex: r = r0 + i*dr, theta = -sector/2 + j*sector/(W-1);
 *           (r sin(theta), 0, r cos(theta) - r0)   [origin at the centre of
 *           the transducer face, z pointing into the body]
 * Reading: the paper's 6C1 convex probe (Sec. III.A) gives no radius; r0 is
 * a parameter and the beams are spread evenly over the sector, both ends
 * included.
 */
static void sample_point(const ora_geometry *g, int W, int i, int j, double *xi, double *zi)
{
    if (g->convex) {
        const double pi = 3.14159265358979323846;
        double half = g->sector_deg * pi / 360.0;
        double th = -half + (double)j * (2.0 * half / (double)(W - 1));
        double r = g->r0 + (double)i * g->dr;
        *xi = r * sin(th);
        *zi = r * cos(th) - g->r0;
    } else {
        *xi = (double)j * g->sx;
        *zi = (double)i * g->sy;
    }
}

/*
 * Trilinear splatting.  Each sample at continuous voxel position q spreads
 * its intensity over the 8 voxels around it with the trilinear weights
 * w = prod_a (1 - f_a or f_a), f = q - floor(q):  S += w*I, Wt += w.
 * Readings: corners outside the grid are dropped without renormalising;
 * weights below 2^-20 are dropped; a voxel is empty iff Wt == 0.  Frames are
 * skipped when invalid: the pose's bottom row must be exactly (0,0,0,1)
 * and, per axis, the map's values must be finite with |C_a| < 2^29 and the
 * per-step (linear: per pixel, A_a = M[a][0]*sx/s_a, B_a = M[a][2]*sy/s_a)
 * or per-mm (convex: M[a][0]/s_a, M[a][2]/s_a) factors below 2^14.
 * images: uint8 (is_f32 == 0) or float32, [n][H][W].  Reading for float32
 * samples (the paper's images are 8-bit, so it says nothing about them): a
 * sample is inserted only if it is finite with |I| <= 2^64; any other is
 * treated as absent and adds no weight.
 */
int64_t ora_insert_trilinear(double *S, double *Wt, int nx, int ny, int nz,
                             const void *images, int is_f32, int n, int H, int W,
                             const double *poses, const double K[16], const ora_geometry *g,
                             const double spacing[3], const double origin[3])
{
    return ora_insert_trilinear_rows(S, Wt, nx, ny, nz, images, is_f32, n, H, W, poses, K, g,
                                     spacing, origin, 0);
}

/* As ora_insert_trilinear, skipping rows i < first_rows[f] of frame f. */
int64_t ora_insert_trilinear_rows(double *S, double *Wt, int nx, int ny, int nz,
                                  const void *images, int is_f32, int n, int H, int W,
                                  const double *poses, const double K[16],
                                  const ora_geometry *g, const double spacing[3],
                                  const double origin[3], const int32_t *first_rows)
{
    int64_t skipped = 0;
    const double wmin = 1.0 / 1048576.0; /* 2^-20 */
    for (int f = 0; f < n; ++f) {
        const double *P = poses + (size_t)f * 16;
        double M[3][4];
        int ok = P[12] == 0.0 && P[13] == 0.0 && P[14] == 0.0 && P[15] == 1.0;
        pose_times_calib(P, K, M);
        for (int a = 0; a < 3; ++a) {
            double A = g->convex ? M[a][0] / spacing[a] : (M[a][0] * g->sx) / spacing[a];
            double B = g->convex ? M[a][2] / spacing[a] : (M[a][2] * g->sy) / spacing[a];
            double C = (M[a][3] - origin[a]) / spacing[a];
            if (!isfinite(A) || !isfinite(B) || !isfinite(C))
                ok = 0;
            else if (fabs(A) >= 16384.0 || fabs(B) >= 16384.0 || fabs(C) >= 536870912.0)
                ok = 0;
        }
        if (!ok) {
            ++skipped;
            continue;
        }
        const int i_first = first_rows ? (first_rows[f] > 0 ? first_rows[f] : 0) : 0;
        for (int i = i_first; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                double xi, zi, q[3], fr[3];
                int64_t i0[3];
                sample_point(g, W, i, j, &xi, &zi);
                for (int a = 0; a < 3; ++a) {
                    double p = M[a][0] * xi + M[a][2] * zi + M[a][3];
                    q[a] = (p - origin[a]) / spacing[a];
                    double fl = floor(q[a]);
                    i0[a] = (int64_t)fl;
                    fr[a] = q[a] - fl;
                }
                double I = is_f32 ? (double)((const float *)images)[((size_t)f * H + i) * W + j]
                                  : (double)((const uint8_t *)images)[((size_t)f * H + i) * W + j];
                if (!(fabs(I) <= 18446744073709551616.0)) /* not finite, or above 2^64 */
                    continue;
                for (int cz = 0; cz < 2; ++cz)
                    for (int cy = 0; cy < 2; ++cy)
                        for (int cx = 0; cx < 2; ++cx) {
                            int64_t X = i0[0] + cx, Y = i0[1] + cy, Z = i0[2] + cz;
                            if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz)
                                continue;
                            double w = (cx ? fr[0] : 1.0 - fr[0]) * (cy ? fr[1] : 1.0 - fr[1]) *
                                       (cz ? fr[2] : 1.0 - fr[2]);
                            if (w < wmin)
                                continue;
                            size_t lin = ((size_t)Z * ny + (size_t)Y) * nx + (size_t)X;
                            S[lin] += w * I;
                            Wt[lin] += w;
                        }
            }
    }
    return skipped;
}

/*
 * Normalisation + 3x3x3 hole fill for the weighted variant: a voxel with
 * Wt > 0 takes S/Wt; an empty one takes (sum of neighbour S)/(sum of
 * neighbour Wt) over its non-empty in-grid neighbours among the 26; with
 * none it stays empty.
 */
void ora_fill_trilinear(const double *S, const double *Wt, int nx, int ny, int nz, double *val,
                        uint8_t *has)
{
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = ((size_t)z * ny + y) * nx + x;
                if (Wt[i] > 0.0) {
                    val[i] = S[i] / Wt[i];
                    has[i] = 1;
                    continue;
                }
                double SS = 0.0, WW = 0.0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (dx == 0 && dy == 0 && dz == 0)
                                continue;
                            int X = x + dx, Y = y + dy, Z = z + dz;
                            if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz)
                                continue;
                            size_t j = ((size_t)Z * ny + Y) * nx + X;
                            if (Wt[j] > 0.0) {
                                SS += S[j];
                                WW += Wt[j];
                            }
                        }
                if (WW > 0.0) {
                    val[i] = SS / WW;
                    has[i] = 1;
                } else {
                    val[i] = 0.0;
                    has[i] = 0;
                }
            }
}

/* Depth-band mean of a real-valued volume over has-data voxels, FP64. */
void ora_project_f64(const double *val, const uint8_t *has, int nx, int ny, int nz, int lo,
                     int hi, double *out, uint16_t *cnt)
{
    (void)nz;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double s = 0.0;
            uint64_t c = 0;
            for (int z = lo; z < hi; ++z) {
                size_t i = ((size_t)z * ny + y) * nx + x;
                if (has[i]) {
                    s += val[i];
                    c += 1;
                }
            }
            out[(size_t)y * nx + x] = c ? s / (double)c : 0.0;
            if (cnt)
                cnt[(size_t)y * nx + x] = (uint16_t)c;
        }
}

/* ------------------------------------------------------------------------- */
/* Tissue segmentation: depth of cut (Algorithms 1 and 2).                    */
/* ------------------------------------------------------------------------- */

/*
 * Algorithm 1 (Table I): Cut_n = K |P_c1.x - P_cn.x - L/2| + D, where P_cn
 * is the position of frame n's upper-left pixel (step 3) and .x the
 * coordinate along the spine (step 4).  Reading: P_cn = pose * calib *
 * (0,0,0,1), ".x" = dot with the unit spine direction e, P_c1 = p1 (the
 * scan's first frame); the first row kept is ceil(Cut_n / row_mm), clamped
 * to [0, H].  FP64, operations in this order, no fused multiply-add.
 */
void ora_cut_rows_alg1(const double *poses, int n, int H, const double K[16], double k,
                       double d_mm, double l_mm, const double e[3], const double p1[3],
                       double row_mm, int32_t *rows, double *cut_mm)
{
    for (int f = 0; f < n; ++f) {
        const double *P = poses + (size_t)f * 16;
        double M[3][4], pos[3];
        pose_times_calib(P, K, M);
        for (int a = 0; a < 3; ++a)
            pos[a] = M[a][3];
        double d = (p1[0] - pos[0]) * e[0];
        d = d + (p1[1] - pos[1]) * e[1];
        d = d + (p1[2] - pos[2]) * e[2];
        const double cut = k * fabs(d - l_mm * 0.5) + d_mm;
        const double row = ceil(cut / row_mm);
        int r = 0;
        if (row > 0.0)
            r = row >= (double)H ? H : (int)row;
        rows[f] = r;
        if (cut_mm)
            cut_mm[f] = cut;
    }
}

static int cmp_i32(const void *a, const void *b)
{
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Algorithm 2 (Table II).  Step 2 -- contours at the bottom of the image
 * with a large gradient and a high value: in rows v >= from, score(v, u) =
 * I(v,u) * max(0, I(v,u) - I(v+drop,u)) (a bright cortex over its acoustic
 * shadow); the column's contour row is the first v of the maximum score
 * (from if all scores are 0); the frame's bone row is the lower median over
 * its columns.  Step 3 -- median filtering over all frames: the lower
 * median of the bone rows in [n - window/2, n + window/2] clipped to the
 * scan.  The depth of cut keeps `margin` rows above it (at least row 0).
 */
void ora_bone_rows_alg2(const uint8_t *images, int n, int H, int W, int from, int drop,
                        int window, int margin, int32_t *bone, int32_t *rows)
{
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(W > window ? W : window));
    for (int f = 0; f < n; ++f) {
        const uint8_t *img = images + (size_t)f * H * W;
        for (int u = 0; u < W; ++u) {
            long best = -1;
            int brow = from;
            for (int v = from; v + drop < H; ++v) {
                const int a = img[(size_t)v * W + u];
                const int b = img[(size_t)(v + drop) * W + u];
                const long s = (long)a * (a > b ? a - b : 0);
                if (s > best) {
                    best = s;
                    brow = v;
                }
            }
            col[u] = best > 0 ? brow : from;
        }
        qsort(col, (size_t)W, sizeof(int32_t), cmp_i32);
        bone[f] = col[(W - 1) / 2];
    }
    for (int f = 0; f < n; ++f) {
        const int k0 = f - window / 2 < 0 ? 0 : f - window / 2;
        const int k1 = f + window / 2 > n - 1 ? n - 1 : f + window / 2;
        const int len = k1 - k0 + 1;
        for (int k = 0; k < len; ++k)
            col[k] = bone[k0 + k];
        qsort(col, (size_t)len, sizeof(int32_t), cmp_i32);
        const int med = col[(len - 1) / 2];
        rows[f] = med - margin > 0 ? med - margin : 0;
    }
    free(col);
}
