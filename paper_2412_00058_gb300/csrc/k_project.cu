// A4: depth-band projection -- the VPI spine view at a fixed depth (Sec.
// III.B, Fig. 6: coronal images from a fixed depth of 35 or 45 mm).  For
// every (x, y), the mean of the filled values of the has-data voxels with
// z in [lo, hi), 0 where there are none; one IEEE FP32 division.
//
// GB300 design: the band is a few MB, so the kernel is latency-bound rather
// than HBM-bound; each thread issues the loads of 8 planes before it uses
// any of them (the sums still run in ascending z), so their latencies
// overlap.  A whole-plane projection of uint8 values takes 4 consecutive
// columns of the flattened (y, x) plane per thread: one 32-bit load per
// plane (a warp reads 128 consecutive bytes) and the at most two mask words
// its 4 columns fall in (a row end or a 32-column boundary can split them).
// A region, or a plane whose size or base does not allow 32-bit words,
// takes one thread per (x, y) column (a warp reads 32 consecutive bytes of
// a row per plane and shares one mask word).  It is kept separate so
// several bands can be projected from one filled volume.
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

// Whole plane, 4 consecutive columns i0 .. i0+3 of the flattened plane per
// thread (the plane's size a multiple of 4, nx not 1 or 2 mod 32).  Column
// k's has-data bit is in mask word A (the word of column i0) or B (the word
// of column i0 + 3).
__global__ void __launch_bounds__(256) k_project_u8_w4(ProjArgs a, int vec_out)
{
    const size_t plane = (size_t)a.ny * a.nx, nw = plane / 4;
    const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw)
        return;
    const size_t i0 = 4 * w;
    const size_t mplane = (size_t)a.ny * a.nxw;
    // mask words and bits of the 4 columns
    size_t mo[4];
    unsigned sh[4];
    {
        unsigned y = (unsigned)(i0 / (size_t)a.nx), x = (unsigned)(i0 - (size_t)y * a.nx);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            mo[k] = (size_t)y * a.nxw + (x >> 5);
            sh[k] = x & 31u;
            if (++x == (unsigned)a.nx) {
                x = 0;
                ++y;
            }
        }
    }
    const size_t mA = mo[0], mB = mo[3];
    unsigned useB = 0;  // bit k: column k's bit is in word B
#pragma unroll
    for (int k = 0; k < 4; ++k)
        useB |= (mo[k] != mA ? 1u : 0u) << k;
    const auto *vw = static_cast<const uint32_t *>(a.val);
    unsigned s[4] = {0u, 0u, 0u, 0u}, c[4] = {0u, 0u, 0u, 0u};
    auto add = [&](unsigned v, unsigned ma, unsigned mb) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned bit = ((((useB >> k) & 1u) ? mb : ma) >> sh[k]) & 1u;
            s[k] += bit ? (v >> (8 * k)) & 0xFFu : 0u;
            c[k] += bit;
        }
    };
    int z = a.lo;
    for (; z + kUnroll <= a.hi; z += kUnroll) {
        unsigned v[kUnroll], ma[kUnroll], mb[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            v[k] = __ldg(vw + w + (size_t)(z + k) * nw);
            ma[k] = __ldg(a.mask + mA + (size_t)(z + k) * mplane);
            mb[k] = __ldg(a.mask + mB + (size_t)(z + k) * mplane);
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k)
            add(v[k], ma[k], mb[k]);
    }
    for (; z < a.hi; ++z)
        add(__ldg(vw + w + (size_t)z * nw), __ldg(a.mask + mA + (size_t)z * mplane),
            __ldg(a.mask + mB + (size_t)z * mplane));
    if (!guard(i0 + 3, plane, a.status))
        return;
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        o[k] = c[k] ? __fdiv_rn((float)s[k], (float)c[k]) : 0.0f;
    if (vec_out) {
        *reinterpret_cast<float4 *>(a.out + i0) = make_float4(o[0], o[1], o[2], o[3]);
        if (a.cnt)
            *reinterpret_cast<uint2 *>(a.cnt + i0) =
                make_uint2(c[0] | (c[1] << 16), c[2] | (c[3] << 16));
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a.out[i0 + k] = o[k];
            if (a.cnt)
                a.cnt[i0 + k] = (uint16_t)c[k];
        }
    }
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
    const size_t plane = (size_t)v.g.nx * v.g.ny;
    // (with nx = 1 or 2 mod 32 a group of 4 columns can span a 32-column
    // boundary and a row end, three mask words: those grids take the other
    // kernel)
    if (rlo[0] == 0 && rlo[1] == 0 && rhi[0] == v.g.nx && rhi[1] == v.g.ny && plane % 4 == 0 &&
        v.g.nx % 32 != 1 && v.g.nx % 32 != 2 &&
        (reinterpret_cast<uintptr_t>(v.val) & 3) == 0 &&
        (reinterpret_cast<uintptr_t>(out) & 3) == 0 && (reinterpret_cast<uintptr_t>(cnt) & 1) == 0) {
        // whole plane, 32-bit words; 16-byte stores where out and cnt allow
        const int vec = (reinterpret_cast<uintptr_t>(out) & 15) == 0 &&
                        (reinterpret_cast<uintptr_t>(cnt) & 7) == 0;
        const size_t nw = plane / 4;
        k_project_u8_w4<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(a, vec);
        return cudaGetLastError();
    }
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
