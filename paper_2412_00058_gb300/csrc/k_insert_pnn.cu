// A1: pixel-nearest-neighbour insertion (Sec. II.C: PNN reconstruction of the
// newly acquired frames).  Every pixel goes to the voxel
//     i_a = floor((Q_a + 2^31) / 2^32),   Q_a = C_a + u*A_a + v*B_a  (Q31.32)
// and, if inside the grid, adds (count 1, sum I) to that voxel's packed
// accumulator (low 32 bits: sum, high 32 bits: count).  All arithmetic is
// integer, so the result is exact and independent of execution order.
//
// GB300 design:
//  * one CTA = a tile of TW columns x TH rows of FPC consecutive frames
//    (default 128 x 64 x 8; TW is 64, 128 or 256, the shape is set per frame
//    size or chosen by the autotuner); a row segment of TW pixels is TW/16
//    lanes, each lane sixteen consecutive pixels read with one coalesced
//    128-bit load (the next row's load is issued before the current row is
//    processed).  With the default a quarter-warp covers one row and the
//    CTA's 32 quarter-warps take every 32nd row.  The near-square tile keeps the box
//    small: the frames are tilted in plane, and an axis-aligned box around a
//    tilted 128 x 64 patch holds about 0.09 entries per pixel against 0.13
//    for a 256 x 32 patch;
//  * the tile's voxel bounding box over its frames is exact (the map is
//    affine, so the extremes sit at the tile corners), so the CTA can
//    accumulate into a dense shared-memory box and then add each touched
//    entry to HBM with one packed 64-bit global atomic;
//  * per pixel: three exact 64-bit coordinate adds, the box index, one
//    native 32-bit shared atomic.  In one step the lanes of a row segment
//    handle pixels 16 columns apart (different voxels), so the atomics do
//    not diverge; lanes of the warp's other rows may meet them in a voxel
//    (a bank conflict, not a divergence);
//  * box entry layout: if the frames' bound on pixels per voxel (set-up
//    kernel) keeps every count of the CTA below 1024, one word holds
//    count (10 bits) | sum (22 bits) -> one atomic per pixel; otherwise
//    two words (sum, count) -> two atomics; if the box does not fit in
//    shared memory (pixels as coarse as voxels, steep poses) every pixel
//    goes straight to an HBM atomic;
//  * bounds checks run only in tiles whose box was clipped by the grid, and
//    there once per 16-pixel group: along a row every voxel index is monotone,
//    so a group whose two end pixels are inside the box is inside.
#include <climits>

#include "usv_internal.cuh"

namespace usv {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPix = 16;             // pixels per lane per row (one 128-bit load)
constexpr int kSmem = 48 * 1024;     // dynamic shared memory per CTA (the box)
constexpr int kMaxFpc = 8;           // frames per CTA (warp 0 takes 4 corners x 8 frames)

// Tile geometry for a tile width TW (64, 128 or 256 columns): a row segment
// of TW pixels is TW/8 lanes, so a warp covers 32/(TW/8) rows per pass.
template <int TW>
struct Tile {
    static constexpr int kRowLanes = TW / kPix;            // lanes per row segment
    static constexpr int kWarpRows = 32 / kRowLanes;       // rows per warp per pass
    static constexpr int kPassRows = kWarps * kWarpRows;   // rows per CTA per pass
};
constexpr int kCountShift = 22;      // packed entry: count << 22 | sum
constexpr int kPackedMaxCount = 1023;

enum { MODE_SKIP = 0, MODE_PACKED = 1, MODE_SPLIT = 2, MODE_DIRECT = 3 };

struct PnnArgs {
    const uint8_t *img;
    int n, H, W;
    const FrameRec *rec;
    unsigned long long *acc;
    int nx, ny, nz;
    int th;                 // rows per tile
    int tiles_x;            // tiles per frame along u
    int fpc;                // frames per CTA
};

__device__ __forceinline__ int hi32(long long q) { return (int)(q >> 32); }

// Division by a CTA-uniform d in [1, 2^16] of numerators n < 2^16:
// with m = floor(2^32 / d) + 1 = 2^32/d + e, 0 < e <= 1,
//     n*m / 2^32 = n/d + n*e/2^32,   n*e/2^32 < 2^-16 <= 1/d,
// and the fractional part of n/d is at most 1 - 1/d, so floor(n*m / 2^32)
// = floor(n/d).  (d = 1 would need m = 2^32 + 1, so it is taken apart.)
__device__ __forceinline__ unsigned div_magic(unsigned d)
{
    return d > 1u ? (unsigned)(0x100000000ull / d) + 1u : 0u;
}

__device__ __forceinline__ unsigned div_by(unsigned n, unsigned d, unsigned m)
{
    return d > 1u ? __umulhi(n, m) : n;
}

__device__ __forceinline__ unsigned long long pack64(unsigned s, unsigned c)
{
    return ((unsigned long long)c << 32) | (unsigned long long)s;
}

// Byte B of `word` in bits 0-7, the other bytes taken from `hi` (bytes
// 1-3 of hi land in bytes 1-3): one byte permute gives the packed box entry
// (count 1 << 22 | I) or, with hi = 0, the plain intensity.
template <int B>
__device__ __forceinline__ unsigned byte_with(unsigned word, unsigned hi)
{
    unsigned d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(word), "r"(hi), "n"(0x7650 | B));
    return d;
}

// One pixel: box-local voxel from the coordinates, then the accumulate.
template <bool CHECK, int MODE, int B>
__device__ __forceinline__ void put(unsigned *box, unsigned cap, unsigned long long *acc,
                                    long long qx, long long qy, long long qz, unsigned ex,
                                    unsigned ey, unsigned ez, unsigned word)
{
    const unsigned lx = (unsigned)hi32(qx), ly = (unsigned)hi32(qy), lz = (unsigned)hi32(qz);
    if (CHECK && !(lx < ex && ly < ey && lz < ez))
        return;
    const unsigned key = (lz * ey + ly) * ex + lx;
    if (MODE == MODE_PACKED) {
        atomicAdd(box + key, byte_with<B>(word, 1u << kCountShift));
    } else if (MODE == MODE_SPLIT) {
        atomicAdd(box + key, byte_with<B>(word, 0u));
        atomicAdd(box + cap + key, 1u);
    } else {
        atomicAdd(acc + key, pack64(byte_with<B>(word, 0u), 1u));
    }
}

template <int J, bool CHECK, int MODE>
__device__ __forceinline__ void put_px(unsigned *box, unsigned cap, unsigned long long *acc,
                                       long long qx, long long qy, long long qz, long long Ax,
                                       long long Ay, long long Az, unsigned ex, unsigned ey,
                                       unsigned ez, uint4 w, int npx)
{
    if constexpr (J < kPix) {
        if (J < npx)
            put<CHECK, MODE, J & 3>(box, cap, acc, qx, qy, qz, ex, ey, ez,
                                    J < 4 ? w.x : J < 8 ? w.y : J < 12 ? w.z : w.w);
        put_px<J + 1, CHECK, MODE>(box, cap, acc, qx + Ax, qy + Ay, qz + Az, Ax, Ay, Az, ex, ey,
                                   ez, w, npx);
    }
}

template <bool CHECK, int MODE>
__device__ __forceinline__ void put_group(unsigned *box, unsigned cap, unsigned long long *acc,
                                          long long qx, long long qy, long long qz, long long Ax,
                                          long long Ay, long long Az, unsigned ex, unsigned ey,
                                          unsigned ez, uint4 w, int npx)
{
    put_px<0, CHECK, MODE>(box, cap, acc, qx, qy, qz, Ax, Ay, Az, ex, ey, ez, w, npx);
}

template <int TW, bool VEC, bool CHECK, int MODE>
__device__ __forceinline__ void run_frames(const PnnArgs &a, int f0, int f1, int u0, int u1,
                                           int v0, int v1, const long long (&off)[3],
                                           unsigned ex, unsigned ey, unsigned ez, unsigned *box,
                                           unsigned cap, const FrameRec *recs)
{
    constexpr int kRowLanes = Tile<TW>::kRowLanes, kWarpRows = Tile<TW>::kWarpRows;
    constexpr int kPassRows = Tile<TW>::kPassRows;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int u = u0 + kPix * (lane % kRowLanes);
    const int vs = v0 + warp * kWarpRows + lane / kRowLanes;  // this lane's first row
    if (u >= u1 || vs >= v1)
        return;
    const int npx = VEC ? kPix : min(kPix, u1 - u);
    const size_t rstep = (size_t)kPassRows * a.W;
    for (int f = f0; f < f1; ++f) {
        const FrameRec *r = recs + (f - f0);
        if (!r->valid)
            continue;
        const long long Ax = r->q[0], Ay = r->q[1], Az = r->q[2];
        const long long Bx = r->q[3], By = r->q[4], Bz = r->q[5];
        // rows above first_row are cut away (tissue segmentation)
        const int fr = r->first_row;
        if (fr >= v1)
            continue;
        int v = vs;
        if (v < fr)
            v += (fr - v + kPassRows - 1) / kPassRows * kPassRows;
        if (v >= v1)
            continue;
        const long long qx0 = r->q[6] + off[0] + (long long)u * Ax + (long long)v * Bx;
        const long long qy0 = r->q[7] + off[1] + (long long)u * Ay + (long long)v * By;
        const long long qz0 = r->q[8] + off[2] + (long long)u * Az + (long long)v * Bz;
        const long long Rx = kPassRows * Bx, Ry = kPassRows * By, Rz = kPassRows * Bz;
        const long long Ex = (kPix - 1) * Ax, Ey = (kPix - 1) * Ay, Ez = (kPix - 1) * Az;
        long long qx = qx0, qy = qy0, qz = qz0;
        const uint8_t *src = a.img + ((size_t)f * a.H + v) * a.W + u;
        auto load = [&](const uint8_t *p) {
            uint4 w;
            if (VEC) {
                w = __ldcs(reinterpret_cast<const uint4 *>(p));
            } else {
                w = make_uint4(0u, 0u, 0u, 0u);
                for (int j = 0; j < npx; ++j) {
                    const unsigned b = __ldcs(p + j) << (8 * (j & 3));
                    if (j < 4)
                        w.x |= b;
                    else if (j < 8)
                        w.y |= b;
                    else if (j < 12)
                        w.z |= b;
                    else
                        w.w |= b;
                }
            }
            return w;
        };
        uint4 w = load(src);
        for (; v < v1; v += kPassRows) {
            const bool more = v + kPassRows < v1;
            uint4 wn = make_uint4(0u, 0u, 0u, 0u);
            if (more)
                wn = load(src + rstep);
            bool inside = true;
            if (CHECK) {
                const long long lx = qx + Ex, ly = qy + Ey, lz = qz + Ez;
                inside = (unsigned)hi32(qx) < ex && (unsigned)hi32(qy) < ey &&
                         (unsigned)hi32(qz) < ez && (unsigned)hi32(lx) < ex &&
                         (unsigned)hi32(ly) < ey && (unsigned)hi32(lz) < ez;
            }
            if (!CHECK || inside)
                put_group<false, MODE>(box, cap, a.acc, qx, qy, qz, Ax, Ay, Az, ex, ey, ez, w,
                                       npx);
            else
                put_group<true, MODE>(box, cap, a.acc, qx, qy, qz, Ax, Ay, Az, ex, ey, ez, w,
                                      npx);
            qx += Rx;
            qy += Ry;
            qz += Rz;
            src += rstep;
            w = wn;
        }
    }
}

// One CTA's work: tile `tile` of the frame group `group` (frames
// group*fpc ..).  Every thread of the CTA calls it with the same arguments;
// it leaves shared memory to be reused only after a barrier.
template <int TW, bool VEC>
__device__ __forceinline__ void insert_tile(const PnnArgs &a, int tile, int group)
{
    extern __shared__ unsigned box[];
    __shared__ int s_lo[3], s_ext[3], s_mode, s_check;
    __shared__ FrameRec s_rec[kMaxFpc];

    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int u0 = tx * TW, v0 = ty * a.th;
    const int u1 = min(a.W, u0 + TW), v1 = min(a.H, v0 + a.th);
    const int f0 = group * a.fpc, f1 = min(a.n, f0 + a.fpc);

    // the CTA's frame records, copied once into shared memory
    for (int i = threadIdx.x; i < (f1 - f0) * (int)(sizeof(FrameRec) / 8); i += kThreads)
        reinterpret_cast<unsigned long long *>(s_rec)[i] =
            reinterpret_cast<const unsigned long long *>(a.rec + f0)[i];
    __syncthreads();
    if (threadIdx.x < 32) {
        // lane i: corner i & 3 of frame f0 + (i >> 2) (up to 8 frames)
        const int lane = threadIdx.x;
        const int f = f0 + (lane >> 2);
        int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
        int cnt = 0, valid = 0;
        if (f < f1 && s_rec[f - f0].valid) {
            const FrameRec *r = s_rec + (f - f0);
            const long long u = (lane & 1) ? u1 - 1 : u0;
            const long long v = (lane & 2) ? v1 - 1 : v0;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const long long Q = r->q[6 + ax] + u * r->q[ax] + v * r->q[3 + ax];
                lo[ax] = hi[ax] = (int)((Q + (1LL << 31)) >> 32);  // arithmetic: floor
            }
            valid = 1;
            cnt = (lane & 3) == 0 ? r->nmax : 0;
        }
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            lo[ax] = __reduce_min_sync(0xFFFFFFFFu, lo[ax]);
            hi[ax] = __reduce_max_sync(0xFFFFFFFFu, hi[ax]);
        }
        const unsigned any = __reduce_or_sync(0xFFFFFFFFu, (unsigned)valid);
        const unsigned nsum = __reduce_add_sync(0xFFFFFFFFu, (unsigned)cnt);
        if (lane == 0) {
            int mode = MODE_SKIP, check = 0;
            if (any) {
                const int n[3] = {a.nx, a.ny, a.nz};
                long long vol = 1;
                mode = MODE_PACKED;
                for (int ax = 0; ax < 3; ++ax) {
                    const int l = max(lo[ax], 0), h = min(hi[ax], n[ax] - 1);
                    if (l > h)
                        mode = MODE_SKIP;
                    if (l != lo[ax] || h != hi[ax])
                        check = 1;
                    s_lo[ax] = l;
                    s_ext[ax] = max(h - l + 1, 0);
                    vol *= max(h - l + 1, 0);
                }
                if (mode != MODE_SKIP) {
                    if (nsum <= kPackedMaxCount && vol <= kSmem / 4)
                        mode = MODE_PACKED;
                    else if (vol <= kSmem / 8)
                        mode = MODE_SPLIT;
                    else
                        mode = MODE_DIRECT;
                }
            }
            s_mode = mode;
            s_check = check;
        }
    }
    __syncthreads();
    const int mode = s_mode;
    if (mode == MODE_SKIP)
        return;

    if (mode == MODE_DIRECT) {
        // keys are global linear indices into the whole grid
        const long long off[3] = {1LL << 31, 1LL << 31, 1LL << 31};
        run_frames<TW, VEC, true, MODE_DIRECT>(a, f0, f1, u0, u1, v0, v1, off, (unsigned)a.nx,
                                           (unsigned)a.ny, (unsigned)a.nz, nullptr, 0, s_rec);
        return;
    }
    const unsigned ex = s_ext[0], ey = s_ext[1], ez = s_ext[2];
    const unsigned bvol = ex * ey * ez;
    const unsigned cap = kSmem / 8;
    for (unsigned i = threadIdx.x; i < bvol; i += kThreads) {
        box[i] = 0u;
        if (mode == MODE_SPLIT)
            box[cap + i] = 0u;
    }
    __syncthreads();
    const long long off[3] = {(1LL << 31) - ((long long)s_lo[0] << 32),
                              (1LL << 31) - ((long long)s_lo[1] << 32),
                              (1LL << 31) - ((long long)s_lo[2] << 32)};
    if (mode == MODE_PACKED) {
        if (s_check)
            run_frames<TW, VEC, true, MODE_PACKED>(a, f0, f1, u0, u1, v0, v1, off, ex, ey, ez, box, 0,
                                               s_rec);
        else
            run_frames<TW, VEC, false, MODE_PACKED>(a, f0, f1, u0, u1, v0, v1, off, ex, ey, ez, box,
                                                0, s_rec);
    } else {
        if (s_check)
            run_frames<TW, VEC, true, MODE_SPLIT>(a, f0, f1, u0, u1, v0, v1, off, ex, ey, ez, box,
                                              cap, s_rec);
        else
            run_frames<TW, VEC, false, MODE_SPLIT>(a, f0, f1, u0, u1, v0, v1, off, ex, ey, ez, box,
                                               cap, s_rec);
    }
    __syncthreads();
    // Flush: the box in linear order, all threads busy; each touched entry
    // goes to HBM with one packed 64-bit atomic.  Box coordinates come from
    // the linear index by an exact multiply-high division (below).
    const unsigned mx = div_magic(ex), my = div_magic(ey);
    const size_t nxy = (size_t)a.nx * a.ny;
    unsigned long long *base =
        a.acc + ((size_t)s_lo[2] * a.ny + s_lo[1]) * a.nx + s_lo[0];
    for (unsigned i = threadIdx.x; i < bvol; i += kThreads) {
        const unsigned e = box[i];
        unsigned s, c;
        if (mode == MODE_PACKED) {
            s = e & ((1u << kCountShift) - 1);
            c = e >> kCountShift;
        } else {
            s = e;
            c = box[cap + i];
        }
        if (c != 0u) {
            const unsigned row = div_by(i, ex, mx), lx = i - row * ex;
            const unsigned lz = div_by(row, ey, my), ly = row - lz * ey;
            atomicAdd(base + lz * nxy + (size_t)ly * a.nx + lx, pack64(s, c));
        }
    }
}

template <int TW, bool VEC>
__global__ void __launch_bounds__(kThreads) k_insert_pnn(PnnArgs a)
{
    insert_tile<TW, VEC>(a, blockIdx.x, blockIdx.y);
}

// Several (volume, frames) jobs in one persistent launch: the work items
// are all jobs' (frame group, tile) pairs, job after job; each CTA takes
// items blockIdx.x, blockIdx.x + gridDim.x, ... so consecutive items (tiles
// of one frame group) run side by side.
struct PnnJobs {
    int njobs;
    long long begin[kMaxJobs + 1];  // prefix sums of the jobs' item counts
    int tiles[kMaxJobs];            // tiles per frame group
    int vec[kMaxJobs];
    PnnArgs args[kMaxJobs];
};

__global__ void __launch_bounds__(kThreads) k_insert_pnn_multi(const __grid_constant__ PnnJobs J)
{
    const long long total = J.begin[J.njobs];
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
        int j = 0;
        while (item >= J.begin[j + 1])
            ++j;
        const long long local = item - J.begin[j];
        const int tile = (int)(local % J.tiles[j]), group = (int)(local / J.tiles[j]);
        if (J.vec[j])
            insert_tile<128, true>(J.args[j], tile, group);
        else
            insert_tile<128, false>(J.args[j], tile, group);
        __syncthreads();  // the next item reuses the box and the CTA's words
    }
}

}  // namespace

namespace {

template <int TW>
cudaError_t launch_tw(const PnnArgs &a, dim3 grid, bool vec, cudaStream_t st)
{
    // the box plus the CTA's static words exceed the 48 KB default
    cudaError_t e = prepare_kernel(reinterpret_cast<const void *>(k_insert_pnn<TW, true>), kSmem);
    if (e == cudaSuccess)
        e = prepare_kernel(reinterpret_cast<const void *>(k_insert_pnn<TW, false>), kSmem);
    if (e != cudaSuccess)
        return e;
    if (vec)
        k_insert_pnn<TW, true><<<grid, kThreads, kSmem, st>>>(a);
    else
        k_insert_pnn<TW, false><<<grid, kThreads, kSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool pnn_tile_ok(const TileCfg &c)
{
    return (c.tile_w == 64 || c.tile_w == 128 || c.tile_w == 256) && c.tile_h >= 1 &&
           c.tile_h <= 1024 && c.frames_per_cta >= 1 && c.frames_per_cta <= kMaxFpc;
}

namespace {

PnnArgs make_args(const Volume &v, const uint8_t *img, int n, int H, int W, const TileCfg &cfg)
{
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
    a.th = min(cfg.tile_h, H);
    a.tiles_x = (W + cfg.tile_w - 1) / cfg.tile_w;
    a.fpc = cfg.frames_per_cta;
    return a;
}

bool vec_ok(const uint8_t *img, int W)
{
    return (W % kPix == 0) && ((reinterpret_cast<uintptr_t>(img) & (kPix - 1)) == 0);
}

}  // namespace

cudaError_t launch_insert_pnn_multi(const InsertJob *jobs, int njobs, int num_sms,
                                    cudaStream_t st)
{
    if (njobs < 0 || njobs > kMaxJobs)
        return cudaErrorInvalidValue;
    int per_sm = 1;
    const cudaError_t e = prepare_kernel(reinterpret_cast<const void *>(k_insert_pnn_multi), kSmem,
                                         kThreads, &per_sm);
    if (e != cudaSuccess)
        return e;
    const long long resident = (long long)num_sms * per_sm;
    PnnJobs J;
    J.njobs = njobs;
    J.begin[0] = 0;
    for (int j = 0; j < njobs; ++j) {
        const InsertJob &b = jobs[j];
        if (b.cfg.tile_w != 128 || !pnn_tile_ok(b.cfg))
            return cudaErrorInvalidValue;
        J.args[j] = make_args(*b.v, b.img, b.n, b.H, b.W, b.cfg);
        const int tiles_y = (b.H + J.args[j].th - 1) / J.args[j].th;
        J.tiles[j] = J.args[j].tiles_x * tiles_y;
        J.vec[j] = vec_ok(b.img, b.W) ? 1 : 0;
    }
    // frames per block are upper bounds: while all jobs' work items cannot
    // fill the resident blocks, every job takes fewer frames per block
    long long total = 0;
    for (bool shrink = true; shrink;) {
        total = 0;
        bool can = false;
        for (int j = 0; j < njobs; ++j) {
            const int n = J.args[j].n, f = J.args[j].fpc;
            J.begin[j + 1] = J.begin[j] + (long long)(n > 0 ? (n + f - 1) / f : 0) * J.tiles[j];
            can |= f > 1;
        }
        total = J.begin[njobs];
        shrink = can && total < resident;
        if (shrink)
            for (int j = 0; j < njobs; ++j)
                J.args[j].fpc = (J.args[j].fpc + 1) / 2;
    }
    if (total == 0)
        return cudaSuccess;
    const unsigned grid = (unsigned)(total < resident ? total : resident);
    k_insert_pnn_multi<<<grid, kThreads, kSmem, st>>>(J);
    return cudaGetLastError();
}

cudaError_t launch_insert_pnn(const Volume &v, const uint8_t *img, int n, int H, int W,
                              cudaStream_t st, const TileCfg &cfg)
{
    if (n <= 0)
        return cudaSuccess;
    if (!pnn_tile_ok(cfg))
        return cudaErrorInvalidValue;
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
    a.th = min(cfg.tile_h, H);
    a.tiles_x = (W + cfg.tile_w - 1) / cfg.tile_w;
    const int tiles_y = (H + a.th - 1) / a.th;
    // frames_per_cta is an upper bound: a batch too small to fill the GPU's
    // resident blocks (4 per SM at the 48 KB box) takes fewer frames per
    // block, down to one, so that more blocks share it
    a.fpc = cfg.frames_per_cta;
    const long long resident = (long long)v.num_sms * 4;
    while (a.fpc > 1 && (long long)((n + a.fpc - 1) / a.fpc) * a.tiles_x * tiles_y < resident)
        a.fpc = (a.fpc + 1) / 2;
    const bool vec = (W % kPix == 0) && ((reinterpret_cast<uintptr_t>(img) & (kPix - 1)) == 0);
    const long long groups = (n + a.fpc - 1) / a.fpc;
    if (groups > 65535 || (long long)a.tiles_x * tiles_y > 0x7FFFFFFFLL)
        return cudaErrorInvalidConfiguration;
    const dim3 grid(a.tiles_x * tiles_y, (unsigned)groups);
    switch (cfg.tile_w) {
    case 64: return launch_tw<64>(a, grid, vec, st);
    case 256: return launch_tw<256>(a, grid, vec, st);
    default: return launch_tw<128>(a, grid, vec, st);
    }
}

}  // namespace usv
