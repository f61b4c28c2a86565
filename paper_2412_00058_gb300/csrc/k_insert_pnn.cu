// A1: pixel-nearest-neighbour insertion (Sec. II.C: PNN reconstruction of the
// newly acquired frames).  Every pixel goes to the voxel
//     i_a = floor((Q_a + 2^31) / 2^32),   Q_a = C_a + u*A_a + v*B_a  (Q31.32)
// and, if inside the grid, adds (count 1, sum I) to that voxel's packed
// accumulator (low 32 bits: sum, high 32 bits: count).  All arithmetic is
// integer, so the result is exact and independent of execution order.
//
// GB300 design:
//  * one CTA = a tile of TW columns x TH rows of FPC consecutive frames
//    (default 128 x 64 x 12; TW is 64, 128 or 256, FPC up to 16, 8 with
//    TW 256; the shape is set per frame size or chosen by the autotuner).
//    More frames per box means fewer flushes of each voxel and less set-up
//    per pixel; a group of more than 8 frames whose box is too large for
//    packed entries is done as two passes (its first 8 frames, then the
//    rest), each with its own box.  A row of the tile is cut into
//    segments of 32 pixels, each read by one lane with two coalesced 16-byte
//    loads (a whole 32-byte sector); the next wanted frame's segment is
//    loaded while this one is inserted;
//  * the lanes of a warp take segments of rows 4 apart (rows ordered 0, 4,
//    8, ..., then 1, 5, ...): at 3 to 4 rows per voxel in depth, no two lanes
//    of one step meet in a voxel, so a warp step's shared atomics do not
//    serialise on one address;
//  * the tile's voxel bounding box over its frames is exact (the map is
//    affine, so the extremes sit at the tile corners), so the CTA can
//    accumulate into a dense shared-memory box and then add each touched
//    entry to HBM with one packed 64-bit global atomic.  Box rows are padded
//    to 4 words and planes to 4 mod 8 words: 16-byte clears and flush loads,
//    and the depth offsets of a warp's lanes fall on different banks;
//  * per pixel (the inner loop is hand-written PTX, so the instruction mix
//    is fixed): the box word from the three exact coordinates (two
//    multiply-adds and a shift-add), one byte permute, one native 32-bit
//    shared reduction, and the coordinate steps.  GB300's integer ALU and
//    multiply-add units each take a warp instruction every other cycle, so
//    the steps are split between them: x and z, when below half a voxel per
//    pixel, advance by one wide multiply-add each (a 64-bit add of a
//    sign-extended 32-bit step), y by a 64-bit add.  Where every lane of a
//    warp stays in one y layer for its segment (frames tilted by a degree or
//    less), y and its multiply-add drop out of the loop;
//  * box entry layout: if the frames' bound on pixels per voxel (set-up
//    kernel) keeps every count of the CTA below 1024, one word holds
//    count (10 bits) | sum (22 bits) -> one atomic per pixel; otherwise
//    two words (sum, count) -> two atomics; if the box does not fit in
//    shared memory (pixels as coarse as voxels, steep poses) every pixel
//    goes straight to an HBM atomic;
//  * a tile that the grid clips keeps its whole (unclipped) box when that
//    fits: its pixels outside the grid land in box entries outside the grid,
//    which the flush drops, so every segment takes the checked-free inner
//    loop (a segment cut by the grid would otherwise run a per-pixel checked
//    loop, and with it every warp that holds one, beside the fast one);
//  * only when the whole box does not fit is the box clipped to the grid;
//    bounds checks then run once per segment: along a row every voxel index
//    is monotone, so a segment whose two end pixels are inside the box is
//    inside;
//  * the flush takes the box 4 entries at a time (one 16-byte load), in row
//    order, with exact multiply-high divisions for the row indices; it is
//    compiled per box mode, so its loop holds no mode tests.
#include <climits>
#include <cstddef>

#include "usv_internal.cuh"

namespace usv {

namespace {

constexpr int kThreads = 256;
constexpr int kSeg = 32;             // pixels per lane segment (two 16-byte loads)
constexpr int kSmem = 52 * 1024;     // dynamic shared memory per CTA (the box)
constexpr int kBoxWords = kSmem / 4;
constexpr int kMaxFpc = 16;          // frames per CTA (8 with 256-column tiles)
constexpr int kHalfFpc = 8;          // warp 0 takes 4 corners x 8 frames, twice
constexpr int kCountShift = 22;      // packed entry: count << 22 | sum
constexpr int kPackedMaxCount = 1023;

enum { MODE_SKIP = 0, MODE_PACKED = 1, MODE_SPLIT = 2, MODE_DIRECT = 3 };

struct PnnArgs {
    const uint8_t *img;
    int n, H, W;
    const FrameRec *rec;
    unsigned long long *acc;
    uint32_t *status;       // checked build: USV_STATUS_OOB
    int nx, ny, nz;
    int th;                 // rows per tile
    int tiles_x;            // tiles per frame along u
    int fpc;                // frames per CTA
};

// The part of a frame record the insertion reads (its map and flags),
// copied into shared memory.
struct PnnRec {
    long long q[9];
    int valid, nmax, first_row, pad;
};
static_assert(offsetof(FrameRec, valid) == 144 && sizeof(PnnRec) == 88, "record layout");

// How a CTA accumulates one pass over frames [fa, fb) of its group: box
// origin and extents, strides, mode, checks.
struct Plan {
    int lo[3], ext[3], zs, ex4, mode, check, spill, fa, fb;
};

__device__ __forceinline__ unsigned hi32(long long q) { return (unsigned)(q >> 32); }

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

// Box geometry of a CTA: extents and word strides.  Rows (fixed y, z) are
// ex4 = ex rounded up to 4 words apart, planes zs words apart with
// zs = 4 mod 8: the box is 16-byte aligned quad by quad (16-byte clears and
// flush loads), and the depth offsets of a warp's lanes fall on 8 different
// groups of 4 banks.
struct Box {
    unsigned ex, ey, ez, zs, ex4;
    unsigned long long words;  // entries the keys may address (checked build)
    uint32_t *status;
};

// 64-bit C + k*A for a 32-bit k: one wide multiply-add of A's low word and
// one multiply-add of its high word into the result's high word (exact
// modulo 2^64, which covers every map a valid frame can have).
__device__ __forceinline__ long long mad64(unsigned k, long long A, long long C)
{
    long long d;
    asm("{\n\t.reg .u32 dl, dh;\n\t"
        "mad.wide.u32 %0, %1, %2, %3;\n\t"
        "mov.b64 {dl, dh}, %0;\n\t"
        "mad.lo.u32 dh, %1, %4, dh;\n\t"
        "mov.b64 %0, {dl, dh};\n\t}"
        : "=l"(d)
        : "r"(k), "r"((unsigned)A), "l"(C), "r"((unsigned)((unsigned long long)A >> 32)));
    return d;
}

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

// One pixel: box-local voxel from the coordinates, then the accumulate.
template <bool CHECK, int MODE, int B>
__device__ __forceinline__ void put(unsigned *box, unsigned cap, unsigned long long *acc,
                                    long long qx, long long qy, long long qz, const Box &bx,
                                    unsigned word)
{
    const unsigned lx = hi32(qx), ly = hi32(qy), lz = hi32(qz);
    if (CHECK && !(lx < bx.ex && ly < bx.ey && lz < bx.ez))
        return;
    const unsigned key = lz * bx.zs + ly * bx.ex4 + lx;
    if (!guard(key, bx.words, bx.status))
        return;
    if (MODE == MODE_PACKED) {
        atomicAdd(box + key, byte_with<B>(word, 1u << kCountShift));
    } else if (MODE == MODE_SPLIT) {
        atomicAdd(box + key, byte_with<B>(word, 0u));
        atomicAdd(box + cap + key, 1u);
    } else {
        atomicAdd(acc + key, pack64(byte_with<B>(word, 0u), 1u));
    }
}

// The pixels [J, NPX) of a segment, Q stepping by A per pixel.
template <int J, int NPX, bool CHECK, int MODE>
__device__ __forceinline__ void put_run(unsigned *box, unsigned cap, unsigned long long *acc,
                                        long long qx, long long qy, long long qz, long long Ax,
                                        long long Ay, long long Az, const Box &bx, uint4 w0,
                                        uint4 w1)
{
    if constexpr (J < NPX) {
        constexpr int k = J & 15;
        const uint4 &w = J < 16 ? w0 : w1;
        const unsigned word = k < 4 ? w.x : k < 8 ? w.y : k < 12 ? w.z : w.w;
        put<CHECK, MODE, J & 3>(box, cap, acc, qx, qy, qz, bx, word);
        put_run<J + 1, NPX, CHECK, MODE>(box, cap, acc, qx + Ax, qy + Ay, qz + Az, Ax, Ay, Az,
                                         bx, w0, w1);
    }
}

// A segment of npx pixels (VEC: 16 or 32) starting at Q.
template <bool VEC, bool CHECK, int MODE>
__device__ __forceinline__ void put_segment(unsigned *box, unsigned cap, unsigned long long *acc,
                                            long long qx, long long qy, long long qz,
                                            long long Ax, long long Ay, long long Az,
                                            const Box &bx, uint4 w0, uint4 w1, int npx)
{
    if (VEC) {
        if (npx == kSeg)
            put_run<0, 32, CHECK, MODE>(box, cap, acc, qx, qy, qz, Ax, Ay, Az, bx, w0, w1);
        else
            put_run<0, 16, CHECK, MODE>(box, cap, acc, qx, qy, qz, Ax, Ay, Az, bx, w0, w1);
    } else {
        // scalar-loaded segment of 1..32 pixels: pixels past npx carry no data
        // and are skipped one by one
        unsigned wd[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int j = 0; j < kSeg; ++j) {
            if (j < npx) {
                const unsigned word = wd[j >> 2];
                switch (j & 3) {
                case 0: put<CHECK, MODE, 0>(box, cap, acc, qx, qy, qz, bx, word); break;
                case 1: put<CHECK, MODE, 1>(box, cap, acc, qx, qy, qz, bx, word); break;
                case 2: put<CHECK, MODE, 2>(box, cap, acc, qx, qy, qz, bx, word); break;
                default: put<CHECK, MODE, 3>(box, cap, acc, qx, qy, qz, bx, word); break;
                }
            }
            qx += Ax;
            qy += Ay;
            qz += Az;
        }
    }
}

// 16 pixels of one 16-byte load in hand-written PTX: per pixel the box word
// address from the three exact coordinates (two multiply-adds and a
// shift-add), the packed entry (one byte permute), one shared reduction, and
// the three 64-bit coordinate steps.  Box-local coordinates, no checks.
#define USV_PIX(W, B)                                                          \
    "mov.b64 {lo, lx}, %0;\n\t"                                                \
    "mov.b64 {lo, ly}, %1;\n\t"                                                \
    "mov.b64 {lo, lz}, %2;\n\t"                                                \
    "mad.lo.u32 t, ly, %10, %12;\n\t"                                          \
    "mad.lo.u32 t, lz, %11, t;\n\t"                                            \
    "shl.b32 ad, lx, 2;\n\t"                                                   \
    "add.u32 ad, ad, t;\n\t"                                                   \
    "prmt.b32 val, " W ", %13, " B ";\n\t"                                     \
    "red.shared.add.u32 [ad], val;\n\t"                                        \
    "add.s64 %0, %0, %3;\n\t"                                                  \
    "add.s64 %1, %1, %4;\n\t"                                                  \
    "add.s64 %2, %2, %5;\n\t"
#define USV_WORD(W) USV_PIX(W, "0x7650") USV_PIX(W, "0x7651") USV_PIX(W, "0x7652") USV_PIX(W, "0x7653")

// The same 16 pixels when the x and z steps are below half a voxel per
// pixel: then each step fits a signed 32-bit word and pixel j's x and z
// coordinates are one exact wide multiply-add from the segment start,
// q(j) = q0 + j*A, instead of a chain of 64-bit adds (half the issue slots,
// and the multiply-adds balance the integer units against the adds of y).
#define USV_PIXW(W, B)                                                         \
    "mov.b64 {lo, lx}, %0;\n\t"                                                \
    "mov.b64 {lo, ly}, %1;\n\t"                                                \
    "mov.b64 {lo, lz}, %2;\n\t"                                                \
    "mad.lo.u32 t, ly, %10, %12;\n\t"                                          \
    "mad.lo.u32 t, lz, %11, t;\n\t"                                            \
    "shl.b32 ad, lx, 2;\n\t"                                                   \
    "add.u32 ad, ad, t;\n\t"                                                   \
    "prmt.b32 val, " W ", %13, " B ";\n\t"                                     \
    "red.shared.add.u32 [ad], val;\n\t"                                        \
    "mad.wide.s32 %0, %3, 1, %0;\n\t"                                          \
    "add.s64 %1, %1, %4;\n\t"                                                  \
    "mad.wide.s32 %2, %5, 1, %2;\n\t"
#define USV_WORDW(W)                                                           \
    USV_PIXW(W, "0x7650") USV_PIXW(W, "0x7651") USV_PIXW(W, "0x7652") USV_PIXW(W, "0x7653")

// (x and z steps as 64-bit adds of a sign-extended 32-bit step: one wide
// multiply-add by 1 each, on the multiply-add units, instead of two adds)
__device__ __forceinline__ void put16_packed_w(long long &qx, long long &qy, long long &qz,
                                               int Ax, long long Ay, int Az, uint4 w,
                                               unsigned ex4, unsigned zs4, unsigned sbase)
{
    asm volatile("{\n\t.reg .u32 lo, lx, ly, lz, t, ad, val;\n\t"
                 USV_WORDW("%6") USV_WORDW("%7") USV_WORDW("%8") USV_WORDW("%9")
                 "}"
                 : "+l"(qx), "+l"(qy), "+l"(qz)
                 : "r"(Ax), "l"(Ay), "r"(Az), "r"(w.x), "r"(w.y), "r"(w.z), "r"(w.w), "r"(ex4),
                   "r"(zs4), "r"(sbase), "r"(1u << kCountShift)
                 : "memory");
}

// 16 pixels of a segment that stays in one y layer: x and z only, the y
// layer's offset (ybase, bytes, with the box base) fixed.
#define USV_PIXF(W, B)                                                         \
    "mov.b64 {lo, lx}, %0;\n\t"                                                \
    "mov.b64 {lo, lz}, %1;\n\t"                                                \
    "mad.lo.u32 t, lz, %8, %9;\n\t"                                            \
    "shl.b32 ad, lx, 2;\n\t"                                                   \
    "add.u32 ad, ad, t;\n\t"                                                   \
    "prmt.b32 val, " W ", %10, " B ";\n\t"                                     \
    "red.shared.add.u32 [ad], val;\n\t"                                        \
    "mad.wide.s32 %0, %2, 1, %0;\n\t"                                          \
    "mad.wide.s32 %1, %3, 1, %1;\n\t"
#define USV_WORDF(W)                                                           \
    USV_PIXF(W, "0x7650") USV_PIXF(W, "0x7651") USV_PIXF(W, "0x7652") USV_PIXF(W, "0x7653")

__device__ __forceinline__ void put16_packed_xz(long long &qx, long long &qz, int Ax, int Az,
                                                uint4 w, unsigned zs4, unsigned ybase)
{
    asm volatile("{\n\t.reg .u32 lo, lx, lz, t, ad, val;\n\t"
                 USV_WORDF("%4") USV_WORDF("%5") USV_WORDF("%6") USV_WORDF("%7")
                 "}"
                 : "+l"(qx), "+l"(qz)
                 : "r"(Ax), "r"(Az), "r"(w.x), "r"(w.y), "r"(w.z), "r"(w.w), "r"(zs4),
                   "r"(ybase), "r"(1u << kCountShift)
                 : "memory");
}

__device__ __forceinline__ void put16_packed(long long &qx, long long &qy, long long &qz,
                                             long long Ax, long long Ay, long long Az, uint4 w,
                                             unsigned ex4, unsigned zs4, unsigned sbase)
{
    asm volatile("{\n\t.reg .u32 lo, lx, ly, lz, t, ad, val;\n\t"
                 USV_WORD("%6") USV_WORD("%7") USV_WORD("%8") USV_WORD("%9")
                 "}"
                 : "+l"(qx), "+l"(qy), "+l"(qz)
                 : "l"(Ax), "l"(Ay), "l"(Az), "r"(w.x), "r"(w.y), "r"(w.z), "r"(w.w), "r"(ex4),
                   "r"(zs4), "r"(sbase), "r"(1u << kCountShift)
                 : "memory");
}

template <bool VEC>
__device__ __forceinline__ void load_segment(const uint8_t *p, int npx, uint4 &w0, uint4 &w1)
{
    if (VEC) {
        w0 = __ldcs(reinterpret_cast<const uint4 *>(p));
        w1 = npx > 16 ? __ldcs(reinterpret_cast<const uint4 *>(p) + 1) : make_uint4(0, 0, 0, 0);
    } else {
        unsigned wd[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int j = 0; j < npx; ++j)
            wd[j >> 2] |= (unsigned)__ldcs(p + j) << (8 * (j & 3));
        w0 = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        w1 = make_uint4(wd[4], wd[5], wd[6], wd[7]);
    }
}

// All of the CTA's segments of the frames f0 + ga .. f0 + gb - 1 (one pass
// of its group; recs, q0 and narrowf are indexed from the group's first
// frame), in one box mode.
template <int TW, bool VEC, bool CHECK, int MODE>
__device__ __forceinline__ void run_tile(const PnnArgs &a, int f0, int ga, int gb, int u0, int u1,
                                         int v0, int v1, const Box &bx, unsigned *box,
                                         unsigned cap, const PnnRec *recs,
                                         const long long (*q0)[TW / kSeg][3],
                                         const unsigned char *narrowf)
{
    constexpr int S = TW / kSeg;                 // segments per tile row
    // a tile cut by the frame's right edge has fewer segments per row: its
    // items pack into fewer warps rather than leave lanes idle in every warp
    const int Se = min(S, (u1 - u0 + kSeg - 1) / kSeg);
    const int nrows = v1 - v0;
    const int q = (nrows + 3) >> 2;              // rows per residue class mod 4
    const int items = Se * 4 * q;
    for (int it = threadIdx.x; it < items; it += kThreads) {
        const int s = Se == S ? it % S : it % Se, rp = Se == S ? it / S : it / Se;
        const int r = 4 * (rp % q) + rp / q;     // consecutive lanes: rows 4 apart
        const int u = u0 + kSeg * s;
        if (r >= nrows || u >= u1)
            continue;
        const int v = v0 + r;
        const int npx = VEC ? (u1 - u >= kSeg ? kSeg : 16) : min(kSeg, u1 - u);
        const uint8_t *row = a.img + (size_t)v * a.W + u;
        const size_t fstride = (size_t)a.H * a.W;
        // the frames of the group whose row v is inserted (valid, below the cut)
        unsigned want = 0u;
        for (int g = ga; g < gb; ++g)
            want |= (recs[g].valid && v >= recs[g].first_row ? 1u : 0u) << g;
        if (!want)
            continue;
        int f = __ffs(want) - 1;
        want &= want - 1u;
        uint4 w0, w1;
        load_segment<VEC>(row + (size_t)(f0 + f) * fstride, npx, w0, w1);
        for (;;) {
            const int fn = want ? __ffs(want) - 1 : -1;
            want &= want - 1u;
            uint4 n0 = make_uint4(0, 0, 0, 0), n1 = n0;
            if (fn >= 0)
                load_segment<VEC>(row + (size_t)(f0 + fn) * fstride, npx, n0, n1);
            const PnnRec *rr = recs + f;
            const long long Ax = rr->q[0], Ay = rr->q[1], Az = rr->q[2];
            const long long qx = mad64((unsigned)r, rr->q[3], q0[f][s][0]);
            const long long qy = mad64((unsigned)r, rr->q[4], q0[f][s][1]);
            const long long qz = mad64((unsigned)r, rr->q[5], q0[f][s][2]);
            bool inside = true;
            if (CHECK) {
                const long long e = npx - 1;
                inside = hi32(qx) < bx.ex && hi32(qy) < bx.ey && hi32(qz) < bx.ez &&
                         hi32(qx + e * Ax) < bx.ex && hi32(qy + e * Ay) < bx.ey &&
                         hi32(qz + e * Az) < bx.ez;
            }
            if (!kChecked && (!CHECK || inside) && VEC && MODE == MODE_PACKED) {
                long long x = qx, y = qy, z = qz;
                const unsigned sbase = (unsigned)__cvta_generic_to_shared(box);
                // steps below half a voxel: the wide multiply-add form
                const bool narrow = narrowf[f] != 0;
                // the segment stays in one y layer (and so, by the vote, does
                // every lane of the warp here): two coordinates per pixel
                const bool yc = hi32(qy) == hi32(qy + (long long)(npx - 1) * Ay);
                if (narrow && __all_sync(__activemask(), yc) && yc) {
                    const unsigned ybase = sbase + 4u * bx.ex4 * hi32(qy);
                    put16_packed_xz(x, z, (int)Ax, (int)Az, w0, 4u * bx.zs, ybase);
                    if (npx == kSeg)
                        put16_packed_xz(x, z, (int)Ax, (int)Az, w1, 4u * bx.zs, ybase);
                } else if (narrow) {
                    put16_packed_w(x, y, z, (int)Ax, Ay, (int)Az, w0, 4u * bx.ex4, 4u * bx.zs,
                                   sbase);
                    if (npx == kSeg)
                        put16_packed_w(x, y, z, (int)Ax, Ay, (int)Az, w1, 4u * bx.ex4,
                                       4u * bx.zs, sbase);
                } else {
                    put16_packed(x, y, z, Ax, Ay, Az, w0, 4u * bx.ex4, 4u * bx.zs, sbase);
                    if (npx == kSeg)
                        put16_packed(x, y, z, Ax, Ay, Az, w1, 4u * bx.ex4, 4u * bx.zs, sbase);
                }
            } else if (!CHECK || inside)
                put_segment<VEC, false, MODE>(box, cap, a.acc, qx, qy, qz, Ax, Ay, Az, bx, w0, w1,
                                              npx);
            else
                put_segment<VEC, true, MODE>(box, cap, a.acc, qx, qy, qz, Ax, Ay, Az, bx, w0, w1,
                                             npx);
            if (fn < 0)
                break;
            f = fn;
            w0 = n0;
            w1 = n1;
        }
    }
}

// The flush of a CTA's box: quad p is row p / qr, quad p % qr of it, the
// row (y, z) = (row % ey, row / ey), both by exact multiply-high division.
// The x padding of a row is never touched, so it is skipped as empty.  The
// whole box of a clipped tile (SPILL) may hold entries outside the grid:
// they are dropped here, by row and by entry.
template <int MODE, bool SPILL>
__device__ __forceinline__ void flush_box(const PnnArgs &a, const unsigned *box, unsigned cap,
                                          const Box &bx, const int *lo)
{
    const unsigned qr = bx.ex4 / 4, nq = qr * bx.ey * bx.ez;
    const unsigned mq = div_magic(qr), my = div_magic(bx.ey);
    const long long gplane = (long long)a.nx * a.ny;
    // signed: a spilled box may start before the grid
    const long long gbase = ((long long)lo[2] * a.ny + lo[1]) * a.nx + lo[0];
    const unsigned long long nvox = (unsigned long long)a.nx * a.ny * a.nz;
    for (unsigned p = threadIdx.x; p < nq; p += kThreads) {
        const unsigned row = div_by(p, qr, mq), qx4 = 4u * (p - row * qr);
        const unsigned lz = div_by(row, bx.ey, my), ly = row - lz * bx.ey;
        const unsigned off = lz * bx.zs + ly * bx.ex4 + qx4;
        const uint4 e = *reinterpret_cast<const uint4 *>(box + off);
        uint4 c4 = e;
        unsigned any = e.x | e.y | e.z | e.w;
        if (MODE == MODE_SPLIT) {
            c4 = *reinterpret_cast<const uint4 *>(box + cap + off);
            any |= c4.x | c4.y | c4.z | c4.w;
        }
        if (any == 0u)
            continue;
        unsigned xin = 0xFu;  // entries of the quad inside the grid
        if (SPILL) {
            if ((unsigned)(lo[1] + (int)ly) >= (unsigned)a.ny ||
                (unsigned)(lo[2] + (int)lz) >= (unsigned)a.nz)
                continue;
            const int gx = lo[0] + (int)qx4;
            xin = 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                xin |= ((unsigned)(gx + k) < (unsigned)a.nx ? 1u : 0u) << k;
        }
        const long long gi = gbase + (long long)lz * gplane + (long long)ly * a.nx + qx4;
        unsigned long long *const g = a.acc + gi;
        const unsigned ev[4] = {e.x, e.y, e.z, e.w}, cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned sv = MODE == MODE_PACKED ? ev[k] & ((1u << kCountShift) - 1) : ev[k];
            const unsigned cn = MODE == MODE_PACKED ? ev[k] >> kCountShift : cv[k];
            if (cn != 0u && (!SPILL || ((xin >> k) & 1u)) && guard(qx4 + k, bx.ex, a.status) &&
                guard((unsigned long long)(gi + k), nvox, a.status))
                atomicAdd(g + k, pack64(sv, cn));
        }
    }
}

// The box plan of a frame range from its voxel bounding box (lo, hi), its
// validity and its bound on pixels per voxel (lane 0 of warp 0).
__device__ __forceinline__ void plan_box(const PnnArgs &a, const int (&lo)[3], const int (&hi)[3],
                                         bool any, unsigned nsum, Plan &p)
{
    // box row stride: ex rounded up to 4; plane stride 4 mod 8
    auto strides = [](const long long (&e)[3], int &r4, long long &z) {
        r4 = (int)((e[0] + 3) & ~3LL);
        z = (long long)r4 * e[1];
        z += (z & 4) ? 0 : 4;
        return z * e[2];
    };
    int mode = MODE_SKIP, check = 0, zs = 0, ex4 = 0, spill = 0;
    if (any) {
        const int n[3] = {a.nx, a.ny, a.nz};
        mode = MODE_PACKED;
        long long ce[3], ue[3];
        int cl[3];
        bool small = true;
        for (int ax = 0; ax < 3; ++ax) {
            const int l = max(lo[ax], 0), h = min(hi[ax], n[ax] - 1);
            if (l > h)
                mode = MODE_SKIP;
            if (l != lo[ax] || h != hi[ax])
                check = 1;
            cl[ax] = l;
            ce[ax] = max(h - l + 1, 0);
            ue[ax] = (long long)hi[ax] - lo[ax] + 1;
            small = small && ue[ax] <= kBoxWords;
        }
        if (mode != MODE_SKIP && check && small && nsum <= kPackedMaxCount) {
            // a tile the grid clips takes its whole box if that fits: every
            // pixel then lands in the box with no bounds check, and the
            // flush drops the entries outside the grid
            int r4;
            long long z;
            if (strides(ue, r4, z) <= kBoxWords) {
                spill = 1;
                check = 0;
                ex4 = r4;
                zs = (int)z;
                for (int ax = 0; ax < 3; ++ax) {
                    p.lo[ax] = lo[ax];
                    p.ext[ax] = (int)ue[ax];
                }
            }
        }
        if (mode != MODE_SKIP && !spill) {
            for (int ax = 0; ax < 3; ++ax) {
                p.lo[ax] = cl[ax];
                p.ext[ax] = (int)ce[ax];
            }
            long long z;
            const long long words = strides(ce, ex4, z);
            zs = (int)min(z, (long long)INT_MAX);
            if (nsum <= kPackedMaxCount && words <= kBoxWords)
                mode = MODE_PACKED;
            else if (words <= kBoxWords / 2)
                mode = MODE_SPLIT;
            else
                mode = MODE_DIRECT;
        }
    }
    p.mode = mode;
    p.check = check;
    p.spill = spill;
    p.zs = zs;
    p.ex4 = ex4;
}

// One CTA's work: tile `tile` of the frame group `group` (frames
// group*fpc ..).  Every thread of the CTA calls it with the same arguments;
// it leaves shared memory to be reused only after a barrier.  A group of
// more than 8 frames whose box does not take the packed one-word entries in
// shared memory is done as two passes of its first 8 and its other frames,
// each with its own box.
template <int TW, bool VEC>
__device__ __forceinline__ void insert_tile(const PnnArgs &a, int tile, int group)
{
    constexpr int S = TW / kSeg;
    constexpr int FPC = TW >= 256 ? kHalfFpc : kMaxFpc;
    extern __shared__ __align__(16) unsigned box[];
    __shared__ Plan s_plan[2];
    __shared__ int s_npass;
    __shared__ PnnRec s_rec[FPC];
    __shared__ long long s_q0[FPC][S][3];
    __shared__ unsigned char s_narrow[FPC];

    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int u0 = tx * TW, v0 = ty * a.th;
    const int u1 = min(a.W, u0 + TW), v1 = min(a.H, v0 + a.th);
    const int f0 = group * a.fpc, f1 = min(a.n, f0 + a.fpc);
    const int nf = f1 - f0;

    // the CTA's frame records (map and flags), copied once into shared memory
    for (int i = threadIdx.x; i < nf * 11; i += kThreads) {
        const int f = i / 11, w = i - 11 * f;
        reinterpret_cast<unsigned long long *>(s_rec + f)[w] =
            reinterpret_cast<const unsigned long long *>(a.rec + f0 + f)[w < 9 ? w : 9 + w];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // lane i: corner i & 3 of frames f0 + (i >> 2) (set A) and
        // f0 + 8 + (i >> 2) (set B)
        const int lane = threadIdx.x;
        int lo[2][3], hi[2][3];
        unsigned cnt[2] = {0u, 0u}, valid[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int f = (lane >> 2) + kHalfFpc * h;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                lo[h][ax] = INT_MAX;
                hi[h][ax] = INT_MIN;
            }
            if (f < nf && s_rec[f].valid) {
                const PnnRec *r = s_rec + f;
                const long long u = (lane & 1) ? u1 - 1 : u0;
                const long long v = (lane & 2) ? v1 - 1 : v0;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    const long long Q = r->q[6 + ax] + u * r->q[ax] + v * r->q[3 + ax];
                    lo[h][ax] = hi[h][ax] = (int)((Q + (1LL << 31)) >> 32);  // arithmetic: floor
                }
                valid[h] = 1u;
                cnt[h] = (lane & 3) == 0 ? (unsigned)r->nmax : 0u;
            }
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                lo[h][ax] = __reduce_min_sync(0xFFFFFFFFu, lo[h][ax]);
                hi[h][ax] = __reduce_max_sync(0xFFFFFFFFu, hi[h][ax]);
            }
            valid[h] = __reduce_or_sync(0xFFFFFFFFu, valid[h]);
            cnt[h] = __reduce_add_sync(0xFFFFFFFFu, cnt[h]);
        }
        if (lane == 0) {
            int npass = 1;
            if (nf <= kHalfFpc) {
                plan_box(a, lo[0], hi[0], valid[0] != 0u, cnt[0], s_plan[0]);
            } else {
                int wl[3], wh[3];
                for (int ax = 0; ax < 3; ++ax) {
                    wl[ax] = min(lo[0][ax], lo[1][ax]);
                    wh[ax] = max(hi[0][ax], hi[1][ax]);
                }
                plan_box(a, wl, wh, (valid[0] | valid[1]) != 0u, cnt[0] + cnt[1], s_plan[0]);
                if (s_plan[0].mode != MODE_PACKED && s_plan[0].mode != MODE_SKIP) {
                    // the group's box is too large for packed entries: two
                    // passes of 8 frames and the rest
                    plan_box(a, lo[0], hi[0], valid[0] != 0u, cnt[0], s_plan[0]);
                    plan_box(a, lo[1], hi[1], valid[1] != 0u, cnt[1], s_plan[1]);
                    npass = 2;
                }
            }
            s_plan[0].fa = 0;
            s_plan[0].fb = npass == 2 ? kHalfFpc : nf;
            s_plan[1].fa = kHalfFpc;
            s_plan[1].fb = nf;
            s_npass = npass;
        }
    }
    // per frame whether the x and z steps are below half a voxel (the wide
    // multiply-add loop)
    if (threadIdx.x < nf) {
        const long long Ax = s_rec[threadIdx.x].q[0], Az = s_rec[threadIdx.x].q[2];
        s_narrow[threadIdx.x] = Ax > -(1LL << 31) && Ax < (1LL << 31) &&
                                Az > -(1LL << 31) && Az < (1LL << 31);
    }
    __syncthreads();
    const int npass = s_npass;
    for (int ps = 0; ps < npass; ++ps) {
        const Plan &P = s_plan[ps];
        const int mode = P.mode, fa = P.fa, fb = P.fb;
        if (mode == MODE_SKIP)
            continue;
        // each frame's Q at each segment's first column (u0 + 32 s) of the
        // tile's first row, box-local (or global for MODE_DIRECT), with the
        // 2^31 of the rounding folded in
        for (int i = threadIdx.x; i < 3 * S * (fb - fa); i += kThreads) {
            const int fi = fa + i / (3 * S), sg = (i / 3) % S, ax = i % 3;
            const PnnRec *r = s_rec + fi;
            const long long off =
                (1LL << 31) - (mode == MODE_DIRECT ? 0LL : (long long)P.lo[ax] * (1LL << 32));
            s_q0[fi][sg][ax] = r->q[6 + ax] + (long long)(u0 + kSeg * sg) * r->q[ax] +
                               (long long)v0 * r->q[3 + ax] + off;
        }
        if (mode == MODE_DIRECT) {
            __syncthreads();
            // keys are global linear indices into the whole grid
            const Box g = {(unsigned)a.nx, (unsigned)a.ny, (unsigned)a.nz,
                           (unsigned)a.nx * (unsigned)a.ny, (unsigned)a.nx,
                           (unsigned long long)a.nx * a.ny * a.nz, a.status};
            run_tile<TW, VEC, true, MODE_DIRECT>(a, f0, fa, fb, u0, u1, v0, v1, g, nullptr, 0,
                                                 s_rec, s_q0, s_narrow);
            if (ps + 1 < npass)
                __syncthreads();
            continue;
        }
        const Box bx = {(unsigned)P.ext[0], (unsigned)P.ext[1], (unsigned)P.ext[2], (unsigned)P.zs,
                        (unsigned)P.ex4, (unsigned long long)(unsigned)P.zs * (unsigned)P.ext[2],
                        a.status};
        const unsigned bwords = bx.zs * bx.ez;
        const unsigned cap = kBoxWords / 2;
        {
            // 16-byte stores (every stride is a multiple of 4 words)
            const unsigned quads = bwords / 4;
            uint4 *b4 = reinterpret_cast<uint4 *>(box);
            for (unsigned i = threadIdx.x; i < quads; i += kThreads) {
                b4[i] = make_uint4(0u, 0u, 0u, 0u);
                if (mode == MODE_SPLIT)
                    b4[cap / 4 + i] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        __syncthreads();
        if (mode == MODE_PACKED) {
            if (P.check)
                run_tile<TW, VEC, true, MODE_PACKED>(a, f0, fa, fb, u0, u1, v0, v1, bx, box,
                                                     0, s_rec, s_q0, s_narrow);
            else
                run_tile<TW, VEC, false, MODE_PACKED>(a, f0, fa, fb, u0, u1, v0, v1, bx, box,
                                                     0, s_rec, s_q0, s_narrow);
        } else {
            if (P.check)
                run_tile<TW, VEC, true, MODE_SPLIT>(a, f0, fa, fb, u0, u1, v0, v1, bx, box,
                                                     cap, s_rec, s_q0, s_narrow);
            else
                run_tile<TW, VEC, false, MODE_SPLIT>(a, f0, fa, fb, u0, u1, v0, v1, bx, box,
                                                     cap, s_rec, s_q0, s_narrow);
        }
        __syncthreads();
        // Flush: the threads take the box's quads (4 consecutive x entries of
        // one (y, z) row) in row order; each touched entry goes to HBM with
        // one packed 64-bit atomic (flush_box).
        if (mode == MODE_PACKED) {
            if (P.spill)
                flush_box<MODE_PACKED, true>(a, box, cap, bx, P.lo);
            else
                flush_box<MODE_PACKED, false>(a, box, cap, bx, P.lo);
        } else {
            flush_box<MODE_SPLIT, false>(a, box, cap, bx, P.lo);
        }
        if (ps + 1 < npass)
            __syncthreads();  // the next pass clears the box
    }
}

template <int TW, bool VEC>
__global__ void __launch_bounds__(kThreads, 4) k_insert_pnn(PnnArgs a)
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

__global__ void __launch_bounds__(kThreads, 4) k_insert_pnn_multi(const __grid_constant__ PnnJobs J)
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
           c.tile_h <= 1024 && c.frames_per_cta >= 1 &&
           c.frames_per_cta <= (c.tile_w == 256 ? kHalfFpc : kMaxFpc);
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
    a.status = v.status;
    a.nx = v.g.nx;
    a.ny = v.g.ny;
    a.nz = v.g.nz;
    a.th = min(cfg.tile_h, H);
    a.tiles_x = (W + cfg.tile_w - 1) / cfg.tile_w;
    a.fpc = cfg.frames_per_cta;
    return a;
}

// 16-byte loads need 16-byte rows and a 16-byte aligned first pixel.
bool vec_ok(const uint8_t *img, int W)
{
    return (W % 16 == 0) && ((reinterpret_cast<uintptr_t>(img) & 15) == 0);
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
    PnnArgs a = make_args(v, img, n, H, W, cfg);
    const int tiles_y = (H + a.th - 1) / a.th;
    // frames_per_cta is an upper bound: a batch too small to fill the GPU's
    // resident blocks (4 per SM at the 52 KB box) takes fewer frames per
    // block, down to one, so that more blocks share it
    const long long resident = (long long)v.num_sms * 4;
    while (a.fpc > 1 && (long long)((n + a.fpc - 1) / a.fpc) * a.tiles_x * tiles_y < resident)
        a.fpc = (a.fpc + 1) / 2;
    const bool vec = vec_ok(img, W);
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
