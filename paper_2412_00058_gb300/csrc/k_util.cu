// Small device utilities: clearing accumulators (start of a scan) and
// unpacking the has-data bit mask to one byte per voxel for usv_volume_read.
#include "usv_internal.cuh"

namespace usv {

namespace {

// Grid-stride clear with 16-byte stores; `bytes` is a multiple of 16 and
// `p` 16-byte aligned (the storage layout guarantees both).
__global__ void __launch_bounds__(256) k_zero16(uint4 *p, size_t n16)
{
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16;
         i += (size_t)gridDim.x * blockDim.x)
        __stcs(p + i, z);
}

__global__ void __launch_bounds__(256) k_unpack_mask(const uint32_t *mask, uint8_t *dst, int nx,
                                                     int ny, int nz, int nxw)
{
    const size_t n = (size_t)nx * ny * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / nx;
        const int x = (int)(i - row * nx);
        dst[i] = (uint8_t)((mask[row * nxw + (x >> 5)] >> (x & 31)) & 1u);
    }
}

// Vector-atomic rate probe: thread t of T adds (1, 1) to float2 entries
// (t + k*T) mod n for k < reds -- a warp's 32 reductions are one coalesced
// 256-byte run, and the runs sweep the buffer.  With a buffer that fits in
// L2 this is the L2's float2 reduction throughput; with one far larger than
// L2 every reduction also reads and writes HBM.
__global__ void __launch_bounds__(256) k_red_f2_probe(float2 *buf, unsigned long long n, int reds)
{
    const unsigned long long T = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int k = 0; k < reds; ++k) {
        atomicAdd(buf + (i % n), make_float2(1.0f, 1.0f));
        i += T;
    }
}

}  // namespace

cudaError_t launch_red_f2_probe(void *buf, size_t bytes, int reds, int num_sms, cudaStream_t st)
{
    const unsigned long long n = bytes / sizeof(float2);
    if (n == 0 || reds <= 0)
        return cudaSuccess;
    k_red_f2_probe<<<(unsigned)num_sms * 8, 256, 0, st>>>(static_cast<float2 *>(buf), n, reds);
    return cudaGetLastError();
}

cudaError_t launch_zero(void *p, size_t bytes, int num_sms, cudaStream_t st)
{
    const size_t n16 = bytes / 16;
    if (n16 == 0)
        return cudaSuccess;
    size_t blocks = (n16 + 255) / 256;
    const size_t cap = (size_t)num_sms * 8;
    blocks = blocks < cap ? blocks : cap;
    k_zero16<<<(unsigned)blocks, 256, 0, st>>>(static_cast<uint4 *>(p), n16);
    return cudaGetLastError();
}

cudaError_t launch_unpack_mask(const Volume &v, uint8_t *dst, cudaStream_t st)
{
    const size_t n = (size_t)v.g.nx * v.g.ny * v.g.nz;
    size_t blocks = (n + 255) / 256;
    const size_t cap = (size_t)v.num_sms * 16;
    blocks = blocks < cap ? blocks : cap;
    k_unpack_mask<<<(unsigned)blocks, 256, 0, st>>>(v.mask, dst, v.g.nx, v.g.ny, v.g.nz, v.nxw);
    return cudaGetLastError();
}

}  // namespace usv
