// A2 + A3: normalisation and 3x3x3 hole filling (PNN's second stage after
// bin-filling; Sec. II.C chooses PNN).  One Jacobi pass that reads only the
// accumulators, so re-running it after more inserts stays exact:
//   count > 0  -> value = mean of the voxel's own samples
//   count == 0 -> value = pooled mean over its 26 in-grid neighbours
//                 (sum of sums / sum of counts; empty neighbours add zero)
//   neither    -> empty (mask bit 0, value 0)
// PNN means round half up in exact integer arithmetic; the weighted variant
// divides in IEEE FP32.
//
// GB300 design: HBM-bound stencil.  A CTA owns a 32 x 8 (x, y) column tile
// and marches along z through a slab of planes, keeping three halo'd planes
// of accumulators in a shared-memory ring, so every accumulator is read from
// HBM once (plus a thin halo that neighbouring CTAs share through L2).  The
// has-data mask is one warp ballot per 32 voxels of a row.
#include "usv_internal.cuh"

namespace usv {

namespace {

constexpr int TX = 32, TY = 8, PX = TX + 2, PY = TY + 2;

// floor(S/C + 1/2) clamped to 255, exact.  The quotient q = floor(N/D) with
// N = 2S + C, D = 2C is at most 255 for valid data, so an FP32 estimate is
// off by at most one and one integer correction in each direction fixes it.
__device__ __forceinline__ unsigned mean_round_u8(unsigned long long S, unsigned long long C)
{
    const unsigned long long N = 2ull * S + C, D = 2ull * C;
    const float qf = __fdiv_rn(__ull2float_rn(N), __ull2float_rn(D));
    if (qf >= 257.0f)
        return 255u;
    unsigned long long q = (unsigned long long)qf;
    if (q > 0 && q * D > N)
        --q;
    if ((q + 1) * D <= N)
        ++q;
    return q > 255 ? 255u : (unsigned)q;
}

struct FillArgs {
    const void *acc;
    void *val;
    uint32_t *mask;
    uint32_t *status;
    int nx, ny, nz, nxw, zchunk;
};

template <typename T>
__device__ __forceinline__ void load_plane(T (*pl)[PX], const T *acc, int z, const FillArgs &a,
                                           int x0, int y0, int tid)
{
    for (int i = tid; i < PX * PY; i += TX * TY) {
        const int ly = i / PX, lx = i - ly * PX;
        const int X = x0 - 1 + lx, Y = y0 - 1 + ly;
        T v{};
        if (z >= 0 && z < a.nz && X >= 0 && X < a.nx && Y >= 0 && Y < a.ny)
            v = __ldcg(acc + ((size_t)z * a.ny + Y) * a.nx + X);
        pl[ly][lx] = v;
    }
}

__global__ void __launch_bounds__(TX *TY) k_fill_pnn(FillArgs a)
{
    __shared__ unsigned long long pl[3][PY][PX];
    const auto *acc = static_cast<const unsigned long long *>(a.acc);
    auto *val = static_cast<uint8_t *>(a.val);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zchunk, z1 = min(a.nz, z0 + a.zchunk);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x = x0 + tx, y = y0 + ty;
    const bool inside = x < a.nx && y < a.ny;
    bool saturated = false;

    load_plane(pl[(z0 + 2) % 3], acc, z0 - 1, a, x0, y0, tid);
    load_plane(pl[z0 % 3], acc, z0, a, x0, y0, tid);
    for (int z = z0; z < z1; ++z) {
        load_plane(pl[(z + 1) % 3], acc, z + 1, a, x0, y0, tid);
        __syncthreads();
        const unsigned long long c0 = pl[z % 3][ty + 1][tx + 1];
        unsigned v = 0;
        bool has;
        if ((c0 >> 32) != 0) {
            saturated |= (c0 >> 32) >= (1u << 24);
            v = mean_round_u8(c0 & 0xFFFFFFFFull, c0 >> 32);
            has = true;
        } else {
            unsigned long long S = 0, C = 0;
#pragma unroll
            for (int dz = 0; dz < 3; ++dz) {
                const int slot = (z + 2 + dz) % 3;  // planes z-1, z, z+1
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const unsigned long long w = pl[slot][ty + dy][tx + dx];
                        S += w & 0xFFFFFFFFull;
                        C += w >> 32;
                    }
            }
            has = C != 0;
            if (has)
                v = mean_round_u8(S, C);
        }
        const size_t i = ((size_t)z * a.ny + y) * a.nx + x;
        if (inside)
            val[i] = (uint8_t)v;
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, inside && has);
        if (tx == 0 && y < a.ny)
            a.mask[((size_t)z * a.ny + y) * a.nxw + blockIdx.x] = bits;
        __syncthreads();
    }
    if (__syncthreads_or(saturated) && tid == 0)
        atomicOr(a.status, USV_STATUS_SATURATED);
}

__global__ void __launch_bounds__(TX *TY) k_fill_f32(FillArgs a)
{
    __shared__ float2 pl[3][PY][PX];
    const auto *acc = static_cast<const float2 *>(a.acc);
    auto *val = static_cast<float *>(a.val);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zchunk, z1 = min(a.nz, z0 + a.zchunk);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x = x0 + tx, y = y0 + ty;
    const bool inside = x < a.nx && y < a.ny;

    load_plane(pl[(z0 + 2) % 3], acc, z0 - 1, a, x0, y0, tid);
    load_plane(pl[z0 % 3], acc, z0, a, x0, y0, tid);
    for (int z = z0; z < z1; ++z) {
        load_plane(pl[(z + 1) % 3], acc, z + 1, a, x0, y0, tid);
        __syncthreads();
        const float2 c0 = pl[z % 3][ty + 1][tx + 1];
        float v = 0.0f;
        bool has;
        if (c0.y > 0.0f) {
            v = __fdiv_rn(c0.x, c0.y);
            has = true;
        } else {
            float S = 0.0f, W = 0.0f;
#pragma unroll
            for (int dz = 0; dz < 3; ++dz) {
                const int slot = (z + 2 + dz) % 3;
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const float2 w = pl[slot][ty + dy][tx + dx];
                        if (w.y > 0.0f) {
                            S += w.x;
                            W += w.y;
                        }
                    }
            }
            has = W > 0.0f;
            if (has)
                v = __fdiv_rn(S, W);
        }
        const size_t i = ((size_t)z * a.ny + y) * a.nx + x;
        if (inside)
            val[i] = v;
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, inside && has);
        if (tx == 0 && y < a.ny)
            a.mask[((size_t)z * a.ny + y) * a.nxw + blockIdx.x] = bits;
        __syncthreads();
    }
}

dim3 fill_grid(const Volume &v, int *zchunk)
{
    const int gx = (v.g.nx + TX - 1) / TX, gy = (v.g.ny + TY - 1) / TY;
    // enough CTAs for ~8 waves of 8 resident CTAs per SM, slabs >= 16 planes
    const long long want = (long long)v.num_sms * 8 * 8;
    long long zc = ((long long)gx * gy * v.g.nz + want - 1) / want;
    zc = zc < 16 ? 16 : zc;
    zc = zc > v.g.nz ? v.g.nz : zc;
    *zchunk = (int)zc;
    return dim3(gx, gy, (v.g.nz + (int)zc - 1) / (int)zc);
}

}  // namespace

cudaError_t launch_fill_pnn(const Volume &v, cudaStream_t st)
{
    FillArgs a{v.acc, v.val, v.mask, v.status, v.g.nx, v.g.ny, v.g.nz, v.nxw, 0};
    const dim3 grid = fill_grid(v, &a.zchunk);
    k_fill_pnn<<<grid, dim3(TX, TY), 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fill_trilinear(const Volume &v, cudaStream_t st)
{
    FillArgs a{v.acc, v.val, v.mask, v.status, v.g.nx, v.g.ny, v.g.nz, v.nxw, 0};
    const dim3 grid = fill_grid(v, &a.zchunk);
    k_fill_f32<<<grid, dim3(TX, TY), 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace usv
