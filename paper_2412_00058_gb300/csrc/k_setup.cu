// A0: per-frame pixel->voxel map, computed on the device in FP64.
//
// The world point of an image point x is p = pose * K * x (Alg. 1 steps
// 2-3 and 6: the tracked probe pose T_T^W applied after the image
// calibration).  In voxel units q = (p - origin) / spacing, which is affine
// in the pixel indices:  q(u, v) = C + u*A + v*B.
//
// Every operation is an explicitly rounded IEEE FP64 intrinsic (no
// contraction into fused multiply-adds), in a fixed order, so the result is
// identical on any IEEE machine that follows the same order:
//   M[i][j] = ((P[i][0]K[0][j] + P[i][1]K[1][j]) + P[i][2]K[2][j]) + P[i][3]K[3][j]
//   A_a = (M[a][0]*sx)/s_a,  B_a = (M[a][2]*sy)/s_a,  C_a = (M[a][3]-o_a)/s_a
// and each value times 2^32 is rounded half away from zero to int64 (Q31.32).
#include "usv_internal.cuh"

namespace usv {

namespace {

__device__ __forceinline__ long long q32_round(double x)
{
    // x * 2^32 is exact (power-of-two scale).  x - trunc(x) is exact, so
    // comparing it with 1/2 implements "half away from zero".
    const double y = __dmul_rn(x, 4294967296.0);
    double t = trunc(y);
    const double r = __dsub_rn(y, t);
    if (r >= 0.5)
        t = __dadd_rn(t, 1.0);
    else if (r <= -0.5)
        t = __dsub_rn(t, 1.0);
    return (long long)t;
}

// Upper bound on how many pixels of one frame can land in the same voxel.
// Two such pixels differ by du*A + dv*B with every component in (-1, 1), so
// |dv| < sqrt(3)|A| / |A x B| (the distance of B from the line of A) and,
// within one row, at most ceil(1 / max_a |A_a|) columns fit in a unit
// interval:  N <= (floor(sqrt(3)|A|/|AxB|) + 1) * ceil(1/|A|_inf).
// Computed on the unquantised map with a 1e-6 relative margin (the
// quantised map differs by < 2^-33 per entry, and the cross product is
// trusted only when A and B are more than 1e-6 rad from parallel);
// saturates at 2^20.
__device__ int pixels_per_voxel_bound(const double *d)
{
    const double ax = d[0], ay = d[1], az = d[2], bx = d[3], by = d[4], bz = d[5];
    const double cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
    const double det = sqrt(cx * cx + cy * cy + cz * cz);
    const double na = sqrt(ax * ax + ay * ay + az * az);
    const double nb = sqrt(bx * bx + by * by + bz * bz);
    const double ninf = fmax(fabs(ax), fmax(fabs(ay), fabs(az)));
    // nearly parallel A, B: the cross product loses relative accuracy
    if (!(det > 1e-6 * na * nb) || !(ninf > 1e-9))
        return 1 << 20;
    const double rows = floor(1.7320508075688772 * na / det * (1.0 + 1e-6)) + 1.0;
    const double cols = ceil(1.0 / ninf * (1.0 + 1e-6));
    const double n = rows * cols;
    return n >= 1048576.0 ? (1 << 20) : (int)n;
}

// Frame f's record from its pose P (16 FP64, row-major).
__device__ void setup_frame(const double *__restrict__ P, int f, const SetupParams &sp,
                            FrameRec *__restrict__ rec, uint32_t *status)
{
    double p[16];
#pragma unroll
    for (int i = 0; i < 16; ++i)
        p[i] = P[i];
    bool ok = p[12] == 0.0 && p[13] == 0.0 && p[14] == 0.0 && p[15] == 1.0;
    FrameRec r;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double m[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double acc = __dmul_rn(p[a * 4 + 0], sp.K[0 * 4 + j]);
            acc = __dadd_rn(acc, __dmul_rn(p[a * 4 + 1], sp.K[1 * 4 + j]));
            acc = __dadd_rn(acc, __dmul_rn(p[a * 4 + 2], sp.K[2 * 4 + j]));
            acc = __dadd_rn(acc, __dmul_rn(p[a * 4 + 3], sp.K[3 * 4 + j]));
            m[j] = acc;
        }
        const double A = __ddiv_rn(__dmul_rn(m[0], sp.sx), sp.s[a]);
        const double B = __ddiv_rn(__dmul_rn(m[2], sp.sy), sp.s[a]);
        const double C = __ddiv_rn(__dsub_rn(m[3], sp.o[a]), sp.s[a]);
        if (!isfinite(A) || !isfinite(B) || !isfinite(C))
            ok = false;
        else if (fabs(A) >= 16384.0 || fabs(B) >= 16384.0 || fabs(C) >= 536870912.0)
            ok = false;
        r.d[a] = A;
        r.d[3 + a] = B;
        r.d[6 + a] = C;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i)
        r.q[i] = ok ? q32_round(r.d[i]) : 0;
    r.valid = ok ? 1 : 0;
    r.nmax = ok ? pixels_per_voxel_bound(r.d) : (1 << 20);
    r.first_row = sp.first_rows ? max(sp.first_rows[f], 0) : 0;
    r.pad = 0;
    rec[f] = r;
    if (!ok)
        atomicOr(status, USV_STATUS_BAD_POSE);
}

__global__ void k_frame_setup(const double *__restrict__ poses, int n, SetupParams sp,
                              FrameRec *__restrict__ rec, uint32_t *status)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < n)
        setup_frame(poses + (size_t)f * 16, f, sp, rec, status);
}

// All jobs' frames in one launch: thread t takes frame t - begin[j] of the
// job j with begin[j] <= t < begin[j + 1].
__global__ void k_frame_setup_multi(const __grid_constant__ SetupJobs J)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= J.begin[J.njobs])
        return;
    int j = 0;
    while (t >= J.begin[j + 1])
        ++j;
    const int f = t - J.begin[j];
    const SetupJob &b = J.job[j];
    setup_frame(b.poses + (size_t)f * 16, f, b.sp, b.rec, b.status);
}

// Beam directions of a convex probe: theta_j = -sector/2 + j*sector/(W-1)
// (beams spread evenly over the sector, both ends included).
__global__ void k_beam_setup(double2 *beams, int W, double half_rad, double step_rad)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= W)
        return;
    const double th = __dadd_rn(-half_rad, __dmul_rn((double)j, step_rad));
    double s, c;
    sincos(th, &s, &c);
    beams[j] = make_double2(s, c);
}

}  // namespace

cudaError_t launch_frame_setup(const double *poses, int n, const SetupParams &sp, FrameRec *rec,
                               uint32_t *status, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    // one warp per block: the FP64 work per frame is long, so spread the
    // frames over as many SMs as possible
    k_frame_setup<<<(n + 31) / 32, 32, 0, st>>>(poses, n, sp, rec, status);
    return cudaGetLastError();
}

cudaError_t launch_frame_setup_multi(const SetupJobs &jobs, cudaStream_t st)
{
    const int total = jobs.begin[jobs.njobs];
    if (total <= 0)
        return cudaSuccess;
    k_frame_setup_multi<<<(total + 31) / 32, 32, 0, st>>>(jobs);
    return cudaGetLastError();
}

cudaError_t launch_beam_setup(double2 *beams, int W, double sector_deg, cudaStream_t st)
{
    const double pi = 3.14159265358979323846;
    const double half = sector_deg * pi / 360.0;
    const double step = W > 1 ? (2.0 * half) / (double)(W - 1) : 0.0;
    k_beam_setup<<<(W + 127) / 128, 128, 0, st>>>(beams, W, half, step);
    return cudaGetLastError();
}

}  // namespace usv
