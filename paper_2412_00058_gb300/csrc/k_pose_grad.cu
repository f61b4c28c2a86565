// Pose refinement: gradient of a depth-band projection loss with respect to
// each frame's 6-DoF pose, through the trilinear splat.  The paper's
// patients move during long scans (Sec. I, III.A); a loss between the
// projection of the current reconstruction and a target view lets poses be
// corrected by gradient descent.
//
// Forward (differentiable by construction):
//   S_v, W_v      trilinear splat of every sample (k_insert_trilinear)
//   V_v           = S_v / (W_v + eps)            (soft normalisation)
//   P_xy          = (1/B) sum_{z in band} V_v     (B = band length)
//   L             = sum_xy (P_xy - T_xy)^2
// Backward:
//   g_xy = 2 (P_xy - T_xy);  dL/dS_v = g / (B (W+eps));  dL/dW_v = -g S / (B (W+eps)^2)
//   per sample s, with corner weights w_c = prod_a phi_a (phi = 1-f or f):
//     dL/dq_s,a = sum_c (I_s dL/dS_c + dL/dW_c) * dw_c/dq_a   (right derivative at
//     cell faces, matching floor), over corners kept by the forward (in grid,
//     w >= 2^-20); dL/dp_s = dL/dq_s / spacing
//   per frame, for the left perturbation p' = R(w) (p - c) + c + t about the
//   frame centre c: dL/dt = sum_s dL/dp_s,  dL/dw = sum_s (p_s - c) x dL/dp_s.
// Samples reuse the insertion kernel's exact fixed-point positions and its
// sample rule (float32 samples that are not finite or exceed 2^64 are not
// inserted), so forward and backward see identical cells.
#include <cfloat>

#include "usv_internal.cuh"

namespace usv {

namespace {

constexpr long long kOne47 = 1LL << 47;
constexpr long long kMask47 = kOne47 - 1;
constexpr float kWmin = 9.5367431640625e-07f;     // 2^-20
constexpr float kMaxSample = 18446744073709551616.0f;  // 2^64, as the insertion

__device__ __forceinline__ void anchor(double q, int &i0, long long &fq)
{
    const double fl = floor(q);
    i0 = (int)fl;
    fq = __double2ll_rn((q - fl) * 140737488355328.0);
}

struct SoftArgs {
    const float2 *acc;
    const float *target;
    float *proj;
    float2 *adj;        // [band][ny][nx] (dL/dS, dL/dW)
    double *loss;
    int nx, ny, lo, hi;
    float eps;
    uint32_t *status;   // checked build: USV_STATUS_OOB
};

__global__ void __launch_bounds__(256) k_soft_project_adjoint(SoftArgs a)
{
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    double l = 0.0;
    if (x < a.nx && y < a.ny) {
        const size_t plane = (size_t)a.nx * a.ny, i0 = (size_t)y * a.nx + x;
        const float invB = 1.0f / (float)(a.hi - a.lo);
        float P = 0.0f;
        for (int z = a.lo; z < a.hi; ++z) {
            const float2 sw = a.acc[(size_t)z * plane + i0];
            P += __fdiv_rn(sw.x, sw.y + a.eps);
        }
        P *= invB;
        if (guard(i0, plane, a.status))
            a.proj[i0] = P;
        const float d = P - a.target[i0];
        l = (double)d * (double)d;
        const float g = 2.0f * d * invB;
        for (int z = a.lo; z < a.hi; ++z) {
            const float2 sw = a.acc[(size_t)z * plane + i0];
            const float den = sw.y + a.eps;
            const float gs = __fdiv_rn(g, den);
            const size_t ai = (size_t)(z - a.lo) * plane + i0;
            if (guard(ai, (size_t)(a.hi - a.lo) * plane, a.status))
                a.adj[ai] = make_float2(gs, -gs * __fdiv_rn(sw.x, den));
        }
    }
    // block reduction of the loss
    for (int off = 16; off > 0; off >>= 1)
        l += __shfl_xor_sync(0xFFFFFFFFu, l, off);
    __shared__ double part[8];
    if ((threadIdx.x & 31) == 0)
        part[threadIdx.y] = l;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k)
            s += part[k];
        atomicAdd(a.loss, s);
    }
}

struct GradArgs {
    const void *img;
    int is_f32;
    int n, H, W;
    const FrameRec *rec;
    const float2 *adj;
    double *grad;       // [n][6]: dL/dt (mm), dL/dw (rad)
    uint32_t *status;   // checked build: USV_STATUS_OOB
    int nx, ny, nz, lo, hi;
    double s[3];        // voxel spacing (mm)
};

// one CTA per (frame, 256-column tile x 64-row tile); thread = column
__global__ void __launch_bounds__(256) k_pose_grad(GradArgs a, int tiles_x)
{
    const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int j = tx * 256 + threadIdx.x;
    const int f = blockIdx.y;
    const FrameRec *r = a.rec + f;
    float acc[6] = {0, 0, 0, 0, 0, 0};
    if (r->valid && j < a.W) {
        const int v0 = max(ty * 64, r->first_row), v1 = min(a.H, ty * 64 + 64);
        if (v0 < v1) {
            double base[3], step[3], pivot[3];
            for (int ax = 0; ax < 3; ++ax) {
                base[ax] = r->d[6 + ax] + (double)j * r->d[ax] + (double)v0 * r->d[3 + ax];
                step[ax] = r->d[3 + ax];
                // frame centre ((W-1)/2, (H-1)/2) in voxel units
                pivot[ax] = r->d[6 + ax] + 0.5 * (double)(a.W - 1) * r->d[ax] +
                            0.5 * (double)(a.H - 1) * r->d[3 + ax];
            }
            const bool steep =
                fabs(step[0]) > 256.0 || fabs(step[1]) > 256.0 || fabs(step[2]) > 256.0;
            int i0[3];
            long long fq[3], dq[3];
            float off[3];
            for (int ax = 0; ax < 3; ++ax) {
                anchor(base[ax], i0[ax], fq[ax]);
                dq[ax] = __double2ll_rn(step[ax] * 140737488355328.0);
                off[ax] = (float)((double)i0[ax] - pivot[ax]);  // i0 - pivot (voxels)
            }
            const int i0s[3] = {i0[0], i0[1], i0[2]};
            const size_t plane = (size_t)a.nx * a.ny;
            for (int v = v0; v < v1; ++v) {
                if (steep && v > v0)
                    for (int ax = 0; ax < 3; ++ax)
                        anchor(base[ax] + (double)(v - v0) * step[ax], i0[ax], fq[ax]);
                const size_t pi = ((size_t)f * a.H + v) * a.W + j;
                const float I = a.is_f32 ? __ldg(static_cast<const float *>(a.img) + pi)
                                         : u8_to_float(__ldg(static_cast<const uint8_t *>(a.img) + pi));
                // the insertion's sample rule: a float32 sample that is not
                // finite or exceeds 2^64 was not inserted, so it has no gradient
                const bool admit = fabsf(I) <= kMaxSample;
                int ix[3];
                float w1[3], w0[3], rel[3];
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    const int whole = (int)(fq[ax] >> 47);
                    ix[ax] = i0[ax] + whole;
                    const long long fr = fq[ax] & kMask47;
                    tri_factors(fr, w1[ax], w0[ax]);
                    // position relative to the pivot (voxels): (i0s - pivot) + (ix - i0s) + f
                    rel[ax] = off[ax] + (float)(ix[ax] - i0s[ax]) + w1[ax];
                }
                float gq[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
                    const int X = ix[0] + cx, Y = ix[1] + cy, Z = ix[2] + cz;
                    if ((unsigned)X >= (unsigned)a.nx || (unsigned)Y >= (unsigned)a.ny ||
                        Z < a.lo || Z >= a.hi)
                        continue;
                    const float px = cx ? w1[0] : w0[0], py = cy ? w1[1] : w0[1],
                                pz = cz ? w1[2] : w0[2];
                    if (!admit || px * py * pz < kWmin)
                        continue;
                    const float2 ad = __ldg(a.adj + (size_t)(Z - a.lo) * plane +
                                            (size_t)Y * a.nx + X);
                    const float g = I * ad.x + ad.y;
                    gq[0] += g * (cx ? 1.0f : -1.0f) * py * pz;
                    gq[1] += g * (cy ? 1.0f : -1.0f) * px * pz;
                    gq[2] += g * (cz ? 1.0f : -1.0f) * px * py;
                }
                // to mm: dL/dp = dL/dq / s; lever arm r = rel * s
                float gp[3], rm[3];
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    gp[ax] = gq[ax] / (float)a.s[ax];
                    rm[ax] = rel[ax] * (float)a.s[ax];
                }
                acc[0] += gp[0];
                acc[1] += gp[1];
                acc[2] += gp[2];
                acc[3] += rm[1] * gp[2] - rm[2] * gp[1];
                acc[4] += rm[2] * gp[0] - rm[0] * gp[2];
                acc[5] += rm[0] * gp[1] - rm[1] * gp[0];
                if (!steep) {
                    fq[0] += dq[0];
                    fq[1] += dq[1];
                    fq[2] += dq[2];
                }
            }
        }
    }
    // block reduction -> one FP64 atomic per component
    __shared__ float part[8][6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float vsum = acc[k];
        for (int o = 16; o > 0; o >>= 1)
            vsum += __shfl_xor_sync(0xFFFFFFFFu, vsum, o);
        if ((threadIdx.x & 31) == 0)
            part[threadIdx.x >> 5][k] = vsum;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w)
            s += (double)part[w][threadIdx.x];
        if (guard(f, a.n, a.status))
            atomicAdd(a.grad + (size_t)f * 6 + threadIdx.x, s);
    }
}

// P' = T(t) T(c) R(w) T(-c) P, c = the frame centre in world coordinates
__global__ void k_apply_pose_delta(const double *poses, const double *delta, int n, double cx,
                                   double cz, double K00, double K01, double K02, double K03,
                                   double K10, double K11, double K12, double K13, double K20,
                                   double K21, double K22, double K23, double *out)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n)
        return;
    const double *P = poses + (size_t)f * 16;
    const double *d = delta + (size_t)f * 6;
    // centre in the probe frame: K * (cx, 0, cz, 1); then world: P * that
    const double kc[3] = {K00 * cx + K02 * cz + K03, K10 * cx + K12 * cz + K13,
                          K20 * cx + K22 * cz + K23};
    (void)K01;
    (void)K11;
    (void)K21;
    double c[3];
    for (int a = 0; a < 3; ++a)
        c[a] = P[a * 4 + 0] * kc[0] + P[a * 4 + 1] * kc[1] + P[a * 4 + 2] * kc[2] + P[a * 4 + 3];
    // Rodrigues
    const double wx = d[3], wy = d[4], wz = d[5];
    const double th = sqrt(wx * wx + wy * wy + wz * wz);
    double R[9];
    if (th < 1e-12) {
        R[0] = 1; R[1] = -wz; R[2] = wy;
        R[3] = wz; R[4] = 1; R[5] = -wx;
        R[6] = -wy; R[7] = wx; R[8] = 1;
    } else {
        const double kx = wx / th, ky = wy / th, kz = wz / th;
        const double s = sin(th), cth = cos(th), v = 1.0 - cth;
        R[0] = cth + kx * kx * v;      R[1] = kx * ky * v - kz * s; R[2] = kx * kz * v + ky * s;
        R[3] = ky * kx * v + kz * s;   R[4] = cth + ky * ky * v;    R[5] = ky * kz * v - kx * s;
        R[6] = kz * kx * v - ky * s;   R[7] = kz * ky * v + kx * s; R[8] = cth + kz * kz * v;
    }
    double* o = out + (size_t)f * 16;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 4; ++b)
            o[a * 4 + b] = R[a * 3 + 0] * P[0 * 4 + b] + R[a * 3 + 1] * P[1 * 4 + b] +
                           R[a * 3 + 2] * P[2 * 4 + b];
        // translation: R (P_t - c) + c + t
        o[a * 4 + 3] = R[a * 3 + 0] * (P[3] - c[0]) + R[a * 3 + 1] * (P[7] - c[1]) +
                       R[a * 3 + 2] * (P[11] - c[2]) + c[a] + d[a];
    }
    o[12] = 0.0; o[13] = 0.0; o[14] = 0.0; o[15] = 1.0;
}

__global__ void k_zero_f64(double *p, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        p[i] = 0.0;
}

}  // namespace

cudaError_t launch_zero_f64(double *p, int n, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_zero_f64<<<(n + 255) / 256, 256, 0, st>>>(p, n);
    return cudaGetLastError();
}

cudaError_t launch_soft_project_adjoint(const Volume &v, int lo, int hi, float eps,
                                        const float *target, float *proj, float2 *adj,
                                        double *loss, cudaStream_t st)
{
    SoftArgs a{static_cast<const float2 *>(v.acc), target, proj, adj, loss,
               v.g.nx, v.g.ny, lo, hi, eps, v.status};
    dim3 grid((v.g.nx + 31) / 32, (v.g.ny + 7) / 8);
    k_soft_project_adjoint<<<grid, dim3(32, 8), 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pose_grad(const Volume &v, const void *img, int is_f32, int n, int H, int W,
                             int lo, int hi, const float2 *adj, double *grad, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    GradArgs a;
    a.img = img;
    a.is_f32 = is_f32;
    a.n = n;
    a.H = H;
    a.W = W;
    a.rec = v.rec;
    a.adj = adj;
    a.grad = grad;
    a.status = v.status;
    a.nx = v.g.nx;
    a.ny = v.g.ny;
    a.nz = v.g.nz;
    a.lo = lo;
    a.hi = hi;
    for (int k = 0; k < 3; ++k)
        a.s[k] = v.spacing[k];
    const int tiles_x = (W + 255) / 256, tiles_y = (H + 63) / 64;
    dim3 grid(tiles_x * tiles_y, n);
    k_pose_grad<<<grid, 256, 0, st>>>(a, tiles_x);
    return cudaGetLastError();
}

cudaError_t launch_apply_pose_delta(const double *poses, const double *delta, int n, double cx,
                                    double cz, const double *K, double *out, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_apply_pose_delta<<<(n + 127) / 128, 128, 0, st>>>(poses, delta, n, cx, cz, K[0], K[1], K[2],
                                                         K[3], K[4], K[5], K[6], K[7], K[8], K[9],
                                                         K[10], K[11], out);
    return cudaGetLastError();
}

}  // namespace usv
