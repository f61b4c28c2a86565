// A4: depth-band projection -- the VPI spine view at a fixed depth (Sec.
// III.B, Fig. 6: coronal images from a fixed depth of 35 or 45 mm).  For
// every (x, y), the mean of the filled values of the has-data voxels with
// z in [lo, hi), 0 where there are none; one IEEE FP32 division.
//
// GB300 design: one thread per (x, y) column marching down the band; a warp
// reads 32 consecutive bytes of a row per plane and shares one mask word.
// The band is a few MB, so this kernel is latency-bound rather than
// HBM-bound: each thread issues the loads of 8 planes before it uses any of
// them (the sums still run in ascending z), so their latencies overlap.  It
// is kept separate so several bands can be projected from one filled
// volume.
#include "usv_internal.cuh"

namespace usv {

namespace {

constexpr int kUnroll = 8;  // planes whose loads are in flight together

struct ProjArgs {
    const void *val;
    const uint32_t *mask;
    float *out;
    uint16_t *cnt;
    int nx, ny, nxw, lo, hi;
    int rx0, ry0, rx1, ry1;  // refreshed columns [rx0, rx1) x [ry0, ry1)
    uint32_t *status;        // checked build: USV_STATUS_OOB
};

__global__ void __launch_bounds__(256) k_project_u8(ProjArgs a)
{
    const int x = a.rx0 + blockIdx.x * 32 + threadIdx.x, y = a.ry0 + blockIdx.y * 8 + threadIdx.y;
    if (x >= a.rx1 || y >= a.ry1)
        return;
    const auto *val = static_cast<const uint8_t *>(a.val);
    const size_t plane = (size_t)a.ny * a.nx, mplane = (size_t)a.ny * a.nxw;
    const size_t i0 = (size_t)y * a.nx + x, m0 = (size_t)y * a.nxw + (x >> 5);
    unsigned s = 0, c = 0;
    int z = a.lo;
    for (; z + kUnroll <= a.hi; z += kUnroll) {
        unsigned m[kUnroll], v[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            m[k] = __ldg(a.mask + m0 + (size_t)(z + k) * mplane);
            v[k] = __ldg(val + i0 + (size_t)(z + k) * plane);
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const unsigned bit = (m[k] >> (x & 31)) & 1u;
            s += bit ? v[k] : 0u;
            c += bit;
        }
    }
    for (; z < a.hi; ++z) {
        const unsigned bit = (__ldg(a.mask + m0 + (size_t)z * mplane) >> (x & 31)) & 1u;
        const unsigned v = __ldg(val + i0 + (size_t)z * plane);
        s += bit ? v : 0u;
        c += bit;
    }
    if (!guard(i0, plane, a.status))
        return;
    a.out[i0] = c ? __fdiv_rn((float)s, (float)c) : 0.0f;
    if (a.cnt)
        a.cnt[i0] = (uint16_t)c;
}

__global__ void __launch_bounds__(256) k_project_f32(ProjArgs a)
{
    const int x = a.rx0 + blockIdx.x * 32 + threadIdx.x, y = a.ry0 + blockIdx.y * 8 + threadIdx.y;
    if (x >= a.rx1 || y >= a.ry1)
        return;
    const auto *val = static_cast<const float *>(a.val);
    const size_t plane = (size_t)a.ny * a.nx, mplane = (size_t)a.ny * a.nxw;
    const size_t i0 = (size_t)y * a.nx + x, m0 = (size_t)y * a.nxw + (x >> 5);
    float s = 0.0f;
    unsigned c = 0;
    int z = a.lo;
    for (; z + kUnroll <= a.hi; z += kUnroll) {
        unsigned m[kUnroll];
        float v[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            m[k] = __ldg(a.mask + m0 + (size_t)(z + k) * mplane);
            v[k] = __ldg(val + i0 + (size_t)(z + k) * plane);
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k)
            if ((m[k] >> (x & 31)) & 1u) {  // ascending z, as one plane at a time
                s += v[k];
                c += 1;
            }
    }
    for (; z < a.hi; ++z) {
        const unsigned bit = (__ldg(a.mask + m0 + (size_t)z * mplane) >> (x & 31)) & 1u;
        if (bit) {
            s += __ldg(val + i0 + (size_t)z * plane);
            c += 1;
        }
    }
    if (!guard(i0, plane, a.status))
        return;
    a.out[i0] = c ? __fdiv_rn(s, (float)c) : 0.0f;
    if (a.cnt)
        a.cnt[i0] = (uint16_t)c;
}

}  // namespace

cudaError_t launch_project_u8(const Volume &v, int lo, int hi, const int *rlo, const int *rhi,
                              float *out, uint16_t *cnt, cudaStream_t st)
{
    ProjArgs a{v.val, v.mask, out, cnt, v.g.nx, v.g.ny, v.nxw, lo, hi,
               rlo[0], rlo[1], rhi[0], rhi[1], v.status};
    dim3 grid((rhi[0] - rlo[0] + 31) / 32, (rhi[1] - rlo[1] + 7) / 8);
    if (grid.x == 0 || grid.y == 0)
        return cudaSuccess;
    k_project_u8<<<grid, dim3(32, 8), 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_project_f32(const Volume &v, int lo, int hi, const int *rlo, const int *rhi,
                               float *out, uint16_t *cnt, cudaStream_t st)
{
    ProjArgs a{v.val, v.mask, out, cnt, v.g.nx, v.g.ny, v.nxw, lo, hi,
               rlo[0], rlo[1], rhi[0], rhi[1], v.status};
    dim3 grid((rhi[0] - rlo[0] + 31) / 32, (rhi[1] - rlo[1] + 7) / 8);
    if (grid.x == 0 || grid.y == 0)
        return cudaSuccess;
    k_project_f32<<<grid, dim3(32, 8), 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace usv
