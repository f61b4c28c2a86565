// A1: pixel-nearest-neighbour insertion (Sec. II.C: PNN reconstruction of the
// newly acquired frames).  Every pixel goes to the voxel
//     i_a = floor((Q_a + 2^31) / 2^32),   Q_a = C_a + u*A_a + v*B_a  (Q31.32)
// and, if inside the grid, adds (count 1, sum I) to that voxel's packed
// accumulator (low 32 bits: sum, high 32 bits: count).  All arithmetic is
// integer, so the result is exact and independent of execution order.
//
// GB300 design:
//  * one CTA = a tile of TH rows x (16*TWC) columns of FPC consecutive
//    frames; each thread reads 16 pixels per 128-bit load (coalesced);
//  * the tile's voxel bounding box over its frames is exact (the map is
//    affine, so the extremes sit at the tile corners) -> the CTA accumulates
//    into a dense shared-memory box (separate 32-bit sum and count arrays:
//    native shared atomics; a CTA sees at most 4*8192 pixels, so neither
//    word can wrap), then adds each touched box entry to HBM with one
//    packed 64-bit global atomic;
//  * within a thread, consecutive pixels that hit the same voxel are merged
//    in registers (about 3.6 pixels per voxel along a row for the
//    whole-spine probe) before touching shared memory;
//  * coordinates advance by exact 64-bit adds (two 32-bit ops per axis);
//    bounds checks run only in tiles whose box was clipped by the grid;
//  * tiles whose box does not fit in shared memory (pixels as coarse as
//    voxels, or steep poses) send each run straight to HBM atomics.
#include <climits>

#include "usv_internal.cuh"

namespace usv {

namespace {

constexpr int kThreads = 256;
constexpr unsigned kOut = 0xFFFFFFFEu;   // run key of pixels outside the box
constexpr unsigned kNone = 0xFFFFFFFFu;  // no run open

struct PnnArgs {
    const uint8_t *img;
    int n, H, W;
    const FrameRec *rec;
    unsigned long long *acc;
    int nx, ny, nz;
    int twc, th;            // tile: twc 16-pixel chunks wide, th rows high
    int tiles_x, tiles_y;   // tiles per frame
    int fpc;                // frames per CTA
    int box_cap;            // shared box capacity (entries)
};

__device__ __forceinline__ int hi32(long long q) { return (int)(q >> 32); }

__device__ __forceinline__ unsigned long long pack(unsigned s, unsigned c)
{
    return ((unsigned long long)c << 32) | (unsigned long long)s;
}

// Target of a run: the CTA's shared box (sum and count words) or, in direct
// mode, the packed HBM accumulators.
struct Target {
    unsigned *bsum;
    unsigned *bcnt;
    unsigned long long *acc;
};

template <bool SHARED>
__device__ __forceinline__ void add_run(const Target &t, unsigned key, unsigned s, unsigned c)
{
    if (SHARED) {
        atomicAdd(t.bsum + key, s);
        atomicAdd(t.bcnt + key, c);
    } else {
        atomicAdd(t.acc + key, pack(s, c));
    }
}

// Walk one run of up to 16 pixels along a row.  q*: box-local Q31.32
// coordinates (+2^31 already applied) of the first pixel; a*: per-column
// steps.  Key = box-local linear index (ex*ey*ez box), or kOut.
template <bool VEC, bool CHECK, bool SHARED>
__device__ __forceinline__ void walk_chunk(const uint32_t (&pw)[4], int npx, long long qx,
                                           long long qy, long long qz, long long ax, long long ay,
                                           long long az, unsigned ex, unsigned ey, unsigned ez,
                                           const Target &t)
{
    unsigned cur = kNone, rs = 0;
    int start = 0;
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        if (!VEC && p >= npx)
            break;
        const int lx = hi32(qx), ly = hi32(qy), lz = hi32(qz);
        unsigned key;
        if (CHECK) {
            const bool in = (unsigned)lx < ex && (unsigned)ly < ey && (unsigned)lz < ez;
            key = in ? ((unsigned)lz * ey + (unsigned)ly) * ex + (unsigned)lx : kOut;
        } else {
            key = ((unsigned)lz * ey + (unsigned)ly) * ex + (unsigned)lx;
        }
        if (key != cur) {
            if (p != 0 && cur != kOut)
                add_run<SHARED>(t, cur, rs, (unsigned)(p - start));
            cur = key;
            rs = 0;
            start = p;
        }
        rs += (pw[p >> 2] >> (8 * (p & 3))) & 0xFFu;
        qx += ax;
        qy += ay;
        qz += az;
    }
    if (cur != kOut)
        add_run<SHARED>(t, cur, rs, (unsigned)((VEC ? 16 : npx) - start));
}

template <bool VEC, bool CHECK, bool SHARED>
__device__ __forceinline__ void run_frames(const PnnArgs &a, int f0, int f1, int u0, int u1, int v0, int v1,
                           const long long (&off)[3], unsigned ex, unsigned ey, unsigned ez,
                           const Target &target)
{
    const int cpr = (u1 - u0 + 15) >> 4;  // chunks per row
    const int nchunks = cpr * (v1 - v0);
    for (int f = f0; f < f1; ++f) {
        const FrameRec *r = a.rec + f;
        if (!r->valid)
            continue;
        const long long Ax = r->q[0], Ay = r->q[1], Az = r->q[2];
        const long long Bx = r->q[3], By = r->q[4], Bz = r->q[5];
        const long long Cx = r->q[6] + off[0], Cy = r->q[7] + off[1], Cz = r->q[8] + off[2];
        const uint8_t *img = a.img + (size_t)f * a.H * a.W;
        for (int k = threadIdx.x; k < nchunks; k += kThreads) {
            const int row = k / cpr;
            const int u = u0 + ((k - row * cpr) << 4);
            const int v = v0 + row;
            const uint8_t *src = img + (size_t)v * a.W + u;
            uint32_t pw[4];
            int npx = 16;
            if (VEC) {
                const uint4 q = __ldcs(reinterpret_cast<const uint4 *>(src));
                pw[0] = q.x;
                pw[1] = q.y;
                pw[2] = q.z;
                pw[3] = q.w;
            } else {
                npx = min(16, u1 - u);
                pw[0] = pw[1] = pw[2] = pw[3] = 0;
                for (int p = 0; p < npx; ++p)
                    pw[p >> 2] |= (uint32_t)__ldcs(src + p) << (8 * (p & 3));
            }
            const long long qx = Cx + (long long)u * Ax + (long long)v * Bx;
            const long long qy = Cy + (long long)u * Ay + (long long)v * By;
            const long long qz = Cz + (long long)u * Az + (long long)v * Bz;
            walk_chunk<VEC, CHECK, SHARED>(pw, npx, qx, qy, qz, Ax, Ay, Az, ex, ey, ez, target);
        }
    }
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_insert_pnn(PnnArgs a)
{
    extern __shared__ unsigned box[];  // [box_cap] sums, then [box_cap] counts
    __shared__ int s_lo[3], s_ext[3], s_mode, s_check;

    const int tile = blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int u0 = tx * a.twc * 16, v0 = ty * a.th;
    const int u1 = min(a.W, u0 + a.twc * 16), v1 = min(a.H, v0 + a.th);
    const int f0 = blockIdx.y * a.fpc, f1 = min(a.n, f0 + a.fpc);

    if (threadIdx.x == 0) {
        long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX};
        long long hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
        bool any = false;
        for (int f = f0; f < f1; ++f) {
            const FrameRec *r = a.rec + f;
            if (!r->valid)
                continue;
            any = true;
            for (int c = 0; c < 4; ++c) {
                const long long u = (c & 1) ? u1 - 1 : u0;
                const long long v = (c & 2) ? v1 - 1 : v0;
                for (int ax = 0; ax < 3; ++ax) {
                    const long long Q = r->q[6 + ax] + u * r->q[ax] + v * r->q[3 + ax];
                    const long long i = (Q + (1LL << 31)) >> 32;  // arithmetic: floor
                    lo[ax] = min(lo[ax], i);
                    hi[ax] = max(hi[ax], i);
                }
            }
        }
        int mode = 0, check = 0;
        if (any) {
            const long long n[3] = {a.nx, a.ny, a.nz};
            long long vol = 1;
            mode = 1;
            for (int ax = 0; ax < 3; ++ax) {
                const long long l = max(lo[ax], 0LL), h = min(hi[ax], n[ax] - 1);
                if (l > h)
                    mode = 0;
                if (l != lo[ax] || h != hi[ax])
                    check = 1;
                s_lo[ax] = (int)l;
                s_ext[ax] = (int)max(h - l + 1, 0LL);
                vol *= max(h - l + 1, 0LL);
            }
            if (mode == 1 && vol > a.box_cap)
                mode = 2;
        }
        s_mode = mode;
        s_check = check;
    }
    __syncthreads();
    const int mode = s_mode;
    if (mode == 0)
        return;

    if (mode == 1) {
        const unsigned ex = s_ext[0], ey = s_ext[1], ez = s_ext[2];
        const unsigned bvol = ex * ey * ez;
        const Target t{box, box + a.box_cap, nullptr};
        for (unsigned i = threadIdx.x; i < bvol; i += kThreads) {
            t.bsum[i] = 0u;
            t.bcnt[i] = 0u;
        }
        __syncthreads();
        const long long off[3] = {(1LL << 31) - ((long long)s_lo[0] << 32),
                                  (1LL << 31) - ((long long)s_lo[1] << 32),
                                  (1LL << 31) - ((long long)s_lo[2] << 32)};
        if (s_check)
            run_frames<VEC, true, true>(a, f0, f1, u0, u1, v0, v1, off, ex, ey, ez, t);
        else
            run_frames<VEC, false, true>(a, f0, f1, u0, u1, v0, v1, off, ex, ey, ez, t);
        __syncthreads();
        // Flush: one warp per box row (fixed y, z), lanes along x.
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (unsigned row = warp; row < ey * ez; row += kThreads / 32) {
            const unsigned ly = row % ey, lz = row / ey;
            unsigned long long *dst =
                a.acc + ((size_t)(lz + s_lo[2]) * a.ny + (ly + s_lo[1])) * a.nx + s_lo[0];
            const unsigned *src_s = t.bsum + (size_t)row * ex;
            const unsigned *src_c = t.bcnt + (size_t)row * ex;
            for (unsigned lx = lane; lx < ex; lx += 32) {
                const unsigned c = src_c[lx];
                if (c != 0u)
                    atomicAdd(dst + lx, pack(src_s[lx], c));
            }
        }
    } else {
        // Direct mode: keys are global linear indices into the whole grid.
        const long long off[3] = {1LL << 31, 1LL << 31, 1LL << 31};
        const Target t{nullptr, nullptr, a.acc};
        run_frames<VEC, true, false>(a, f0, f1, u0, u1, v0, v1, off, (unsigned)a.nx,
                                     (unsigned)a.ny, (unsigned)a.nz, t);
    }
}

}  // namespace

cudaError_t launch_insert_pnn(const Volume &v, const uint8_t *img, int n, int H, int W,
                              cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    PnnArgs a;
    a.img = img;
    a.n = n;
    a.H = H;
    a.W = W;
    a.rec = v.rec;
    a.acc = reinterpret_cast<unsigned long long *>(v.acc);
    a.nx = v.g.nx;
    a.ny = v.g.ny;
    a.nz = v.g.nz;
    // Tile: 128 columns x 64 rows (smaller frames: the whole width / height).
    a.twc = min(8, (W + 15) / 16);
    a.th = min(64, H);
    a.tiles_x = (W + a.twc * 16 - 1) / (a.twc * 16);
    a.tiles_y = (H + a.th - 1) / a.th;
    a.fpc = 4;
    const int smem = 48 * 1024;
    a.box_cap = smem / 8;  // entries: one 32-bit sum + one 32-bit count each
    const bool vec = (W % 16 == 0) && ((reinterpret_cast<uintptr_t>(img) & 15) == 0);
    const long long groups = (n + a.fpc - 1) / a.fpc;
    if (groups > 65535)
        return cudaErrorInvalidConfiguration;
    dim3 grid(a.tiles_x * a.tiles_y, (unsigned)groups);
    // The box plus the CTA's few static words exceed the 48 KB default.
    static int attr_device = -1;
    int dev = -1;
    cudaGetDevice(&dev);
    if (attr_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_insert_pnn<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_insert_pnn<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess)
            return e;
        attr_device = dev;
    }
    if (vec)
        k_insert_pnn<true><<<grid, kThreads, smem, st>>>(a);
    else
        k_insert_pnn<false><<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace usv
