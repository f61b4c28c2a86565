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
// GB300 design: HBM-bound stencil.  A CTA owns an (x, y) column tile and
// marches along z through a slab of planes, keeping halo'd planes of
// accumulators in a shared-memory ring, so every accumulator is read from
// HBM once (plus a thin halo that neighbouring CTAs share through L2).  The
// has-data mask is one warp ballot per 32 voxels of a row.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

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
    int rx0, ry0, rz0, rz1;  // refreshed region: x from rx0 (a multiple of 32), y from ry0, z in [rz0, rz1)
    unsigned long long *clear;  // PNN, whole grid: accumulators to zero in the same pass, or null
    int withhold = -1;          // test hook: plane (>= 0) whose copy is never issued; -1: none
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

// ---- nearest-neighbour fill ------------------------------------------------
//
// CTA: 32 x 8 threads own a 32 x 32 (x, y) column tile; thread (tx, ty)
// owns column x0 + tx, rows y0 + 4ty .. y0 + 4ty + 3, and the CTA marches z.
// Planes of packed accumulators (tile + 1-voxel halo) stream into a 5-slot
// shared ring two planes ahead of use: one TMA tensor copy per plane
// (cp.async.bulk.tensor, completion on an mbarrier, zero fill outside the
// grid), or, where the grid's row pitch rules TMA out (odd nx), 8-byte
// cp.async copies by all threads.  The pooled sums are separable: per plane
// each thread forms the x-row sums of its 6 rows (y-1 .. y+4) and from them
// the 3x3 plane sums of its 4 voxels (registers, kept for three planes);
// the 3x3x3 sum is the sum of three plane sums, own voxel included (an
// empty voxel adds zero).  An OR of the words a thread sums tells whether
// its window of the plane is all zero (then its voxels take no arithmetic)
// and whether any count reaches 2^16 or any sum 2^24 (then its voxels of
// that output plane take a direct 64-bit path); below those every sum, and
// the mean's 2S + C, is exact in 32 bits.  With tensor copies each thread
// waits for the plane on the mbarrier and decides alone, so the CTA meets
// at one barrier per plane (slot reuse); with per-entry copies the flags
// are the CTA's, after a second barrier.
constexpr int FTX = 32, FTY = 32, FBY = 8, FRW = 4;  // FRW rows per thread
constexpr int FPX = FTX + 2, FPY = FTY + 2, FPLANE = FPX * FPY;
constexpr int FSLOTS = 5;
constexpr unsigned kBig = 1u << 24;
// TMA boxes start at x0 - 2 (the tensor copy's x offset must be a multiple
// of 16 bytes = 2 entries), so a TMA plane is 36 entries wide; slots are
// padded to 128-byte multiples.
constexpr int kTmaW = FTX + 4;
constexpr int kTmaBytes = kTmaW * FPY * 8;
constexpr int kTmaSlot = (kTmaBytes + 127) / 128 * 128 / 8;  // entries per slot
// Clearing with TMA stores a zero tile of 32 x 16 entries, twice per plane.
constexpr int kZeroRows = 16;
constexpr int kZeroBytes = FTX * kZeroRows * 8;
constexpr int kFillSmemCp = FSLOTS * FPLANE * 8;
constexpr int kFillSmemTma = FSLOTS * kTmaSlot * 8 + kZeroBytes;
// Bounded mbarrier waits: about one second by the global nanosecond timer,
// and never more than kSpinCap polls.
constexpr unsigned long long kWaitNs = 1000000000ull;
constexpr unsigned kSpinCap = 1u << 26;

__device__ __forceinline__ void cp_async8(unsigned saddr, const void *gmem, bool valid)
{
    const int n = valid ? 8 : 0;  // 0: zero-fill, nothing read
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(saddr), "l"(gmem), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0u;
}
// true once the phase with this parity has completed; false after the limit
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// true once the phase with this parity has completed; false after the limit
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = global_ns();
    for (unsigned i = 0; i < kSpinCap; ++i) {
        if (mbar_try_wait(bar, parity))
            return true;
        if ((i & 63u) == 63u && global_ns() - t0 > kWaitNs)
            return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, int x, int y,
                                            int z, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int x, int y, int z,
                                             unsigned src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group"
                 " [%0, {%1, %2, %3}], [%4];" ::"l"(reinterpret_cast<unsigned long long>(map)),
                 "r"(x), "r"(y), "r"(z), "r"(src)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// floor(S/C + 1/2) = floor((2S + C) / 2C), clamped to 255, for S < 2^29 and
// 0 < C < 2^29 (so N = 2S + C and D = 2C fit in 31 bits): the FP32 estimate
// of N/D is within one of the true quotient (|error| < 2^-21 relative, the
// quotient is small), and the exact remainder N - q*D corrects it by one
// in either direction.  Branch-free.
__device__ __forceinline__ unsigned mean_round_fast(unsigned S, unsigned C)
{
    const unsigned N = 2u * S + C, D = 2u * C;
    unsigned q = (unsigned)__fdividef(__uint2float_rn(N), __uint2float_rn(D));
    const int r = (int)(N - q * D);
    q = q + (r >= (int)D ? 1u : 0u) - (r < 0 ? 1u : 0u);
    return min(q, 255u);
}

template <bool TMA>
__global__ void __launch_bounds__(FTX *FBY, 4)
    k_fill_pnn(FillArgs a, const __grid_constant__ CUtensorMap map,
               const __grid_constant__ CUtensorMap clear_map)
{
    constexpr int NT = FTX * FBY;
    constexpr int PER = (FPLANE + NT - 1) / NT;  // plane entries per thread (copy / OR pass)
    constexpr int RS = TMA ? kTmaW : FPX;        // ring row stride (entries)
    constexpr int CO = TMA ? 1 : 0;              // ring column of halo column 0
    constexpr int SLOT = TMA ? kTmaSlot : FPLANE;
    extern __shared__ __align__(128) unsigned long long Pring[];  // [FSLOTS][FPY][RS]
    __shared__ unsigned sflag[FSLOTS];
    __shared__ __align__(8) unsigned long long sbar[FSLOTS];
    __shared__ int s_abort;
    const auto *acc = static_cast<const unsigned long long *>(a.acc);
    auto *val = static_cast<uint8_t *>(a.val);
    const int x0 = a.rx0 + blockIdx.x * FTX, y0 = a.ry0 + blockIdx.y * FTY;
    const int z0 = a.rz0 + blockIdx.z * a.zchunk, z1 = min(a.rz1, z0 + a.zchunk);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;
    const int x = x0 + tx, yb = 4 * ty;  // first of this thread's rows (tile-local)
    const size_t plane = (size_t)a.nx * a.ny;
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(Pring);
    const unsigned bbase = (unsigned)__cvta_generic_to_shared(sbar);
    bool saturated = false;
    unsigned phase = 0u;      // TMA: parity of each slot's next completion
    unsigned pending = 0u;    // TMA, thread 0: slots with a copy in flight

    // this thread's entries of the plane for the copy and OR passes
    size_t goff[PER];
    bool gok[PER];
    int soff[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * NT;
        const int ly = i / FPX, lx = i - ly * FPX;
        const int X = x0 - 1 + lx, Y = y0 - 1 + ly;
        gok[k] = i < FPLANE && X >= 0 && X < a.nx && Y >= 0 && Y < a.ny;
        goff[k] = gok[k] ? (size_t)Y * a.nx + X : 0;
        soff[k] = ly * RS + lx + CO;
    }
    auto issue = [&](int pl) {
        if (TMA) {
            // (plane -1 is a real ring entry: the zero plane below the grid)
            if (tid == 0 && pl <= z1 && (a.withhold < 0 || pl != a.withhold)) {
                const int s = (pl + FSLOTS) % FSLOTS;
                mbar_expect_tx(bbase + 8u * s, kTmaBytes);
                // outside the grid (x < 0, y < 0, z < 0, beyond the far
                // faces) the copy writes zeros
                tma_load_3d(sbase + (unsigned)(s * SLOT * 8), &map, x0 - 2, y0 - 1, pl,
                            bbase + 8u * s);
                pending |= 1u << s;
            }
        } else {
            if (pl <= z1) {
                const unsigned dst = sbase + (unsigned)(((pl + FSLOTS) % FSLOTS) * SLOT * 8);
                const bool zok = pl >= 0 && pl < a.nz;
                const unsigned long long *base = acc + (zok ? (size_t)pl * plane : 0);
#pragma unroll
                for (int k = 0; k < PER; ++k)
                    if (tid + k * NT < FPLANE)
                        cp_async8(dst + 8u * soff[k], base + goff[k], zok && gok[k]);
            }
            cp_async_commit();
        }
    };
    // TMA writes whole 128-byte-aligned slots; a ring that is not aligned is
    // refused (reported as a failed wait) before any copy is issued
    if (TMA && (sbase & 127u) != 0u) {
        if (tid == 0)
            atomicOr(a.status, USV_STATUS_TIMEOUT);
        return;
    }
    // the zero tile that TMA stores into the accumulators being cleared
    const unsigned zbase = sbase + (unsigned)(FSLOTS * SLOT * 8);
    if (TMA && a.clear) {
        for (int i = tid; i < kZeroBytes / 16; i += NT)
            reinterpret_cast<uint4 *>(Pring + FSLOTS * SLOT)[i] = make_uint4(0u, 0u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the copies
    }
    if (tid < FSLOTS)
        sflag[tid] = 0u;
    if (tid == 0) {
        s_abort = 0;
        if (TMA) {
            for (int s = 0; s < FSLOTS; ++s)
                mbar_init(bbase + 8u * s, 1u);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
    }
    __syncthreads();

    // 3x3 plane sums (S, C) of this thread's rows; plane p lives in slot p % 3
    // (the 3x3x3 sum adds all three, so the order does not matter)
    uint2 B[3][FRW];
    int nzf[3] = {0, 0, 0}, bigf[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int r = 0; r < FRW; ++r)
            B[k][r] = make_uint2(0, 0);

    // output pointers of this thread's first row, advanced one plane per output
    const bool xin = x < a.nx;
    uint8_t *vout = val + ((size_t)z0 * a.ny + y0 + yb) * a.nx + x;
    uint32_t *mout = a.mask + ((size_t)z0 * a.ny + y0 + yb) * a.nxw + (x0 >> 5);
    const size_t mplane = (size_t)a.ny * a.nxw;
    const int nrows = min(FRW, a.ny - (y0 + yb));  // rows of this thread inside the grid

    // returns false when the CTA gives up (a TMA wait ran out)
    auto step = [&](int pl, int slot, uint2(&Bn)[FRW], int &nzn, int &bign) {
        issue(pl + 2);
        if (TMA) {
            if (!mbar_wait(bbase + 8u * slot, (phase >> slot) & 1u)) {
                s_abort = 1;
                atomicOr(a.status, USV_STATUS_TIMEOUT);
            }
            phase ^= 1u << slot;
            if (tid == 0)
                pending &= ~(1u << slot);
        } else {
            cp_async_wait<2>();
        }
        const unsigned long long *Pp = Pring + slot * SLOT;
#pragma unroll
        for (int r = 0; r < FRW; ++r)
            Bn[r] = make_uint2(0, 0);
        if (TMA) {
            // every thread has seen the copy complete on the mbarrier, so the
            // plane is visible to it; the flags are this thread's own, over
            // the 6 x 3 words it sums, which are all the words its 4 voxels'
            // neighbourhoods in this plane read
            // x-row sums of rows yb-1 .. yb+4 (halo rows yb .. yb+5), two
            // kept at a time, each plane sum formed as soon as its 3 rows are in
            uint2 R0 = make_uint2(0, 0), R1 = make_uint2(0, 0);
            // OR of the packed words: a count at or above 2^16 or a sum at or
            // above 2^24 takes the exact 64-bit path
            unsigned long long orv = 0ull;
#pragma unroll
            for (int k = 0; k < FRW + 2; ++k) {
                const unsigned long long *row = Pp + (yb + k) * RS + tx + CO;
                const unsigned long long p0 = row[0], p1 = row[1], p2 = row[2];
                const unsigned c0 = (unsigned)(p0 >> 32), c1 = (unsigned)(p1 >> 32),
                               c2 = (unsigned)(p2 >> 32);
                const unsigned s0 = (unsigned)p0, s1 = (unsigned)p1, s2 = (unsigned)p2;
                orv |= p0 | p1 | p2;
                const uint2 R2 = make_uint2(s0 + s1 + s2, c0 + c1 + c2);
                if (k >= 2)
                    Bn[k - 2] = make_uint2(R0.x + R1.x + R2.x, R0.y + R1.y + R2.y);
                R0 = R1;
                R1 = R2;
            }
            nzn = orv != 0ull;
            bign = (orv & 0xFFFF0000FF000000ull) != 0ull;
        } else {
            unsigned orv = 0u;
#pragma unroll
            for (int k = 0; k < PER; ++k)
                if (tid + k * NT < FPLANE) {
                    const unsigned long long w = Pp[soff[k]];
                    orv |= (unsigned)w | (unsigned)(w >> 32);
                }
            orv = __reduce_or_sync(0xFFFFFFFFu, orv);
            if (tx == 0 && orv)
                atomicOr(&sflag[slot], orv);
            __syncthreads();  // every thread's copies have landed; flags complete
            const unsigned fl = sflag[slot];
            if (tid == 0)
                sflag[slot == 0 ? FSLOTS - 1 : slot - 1] = 0u;  // read by everyone last step
            nzn = fl != 0u;
            bign = fl >= kBig;
            if (nzn && !bign) {
                uint2 Rw[FRW + 2];
#pragma unroll
                for (int k = 0; k < FRW + 2; ++k) {
                    const unsigned long long *row = Pp + (yb + k) * RS + tx + CO;
                    const unsigned long long p0 = row[0], p1 = row[1], p2 = row[2];
                    Rw[k] = make_uint2((unsigned)p0 + (unsigned)p1 + (unsigned)p2,
                                       (unsigned)(p0 >> 32) + (unsigned)(p1 >> 32) +
                                           (unsigned)(p2 >> 32));
                }
#pragma unroll
                for (int r = 0; r < FRW; ++r)
                    Bn[r] = make_uint2(Rw[r].x + Rw[r + 1].x + Rw[r + 2].x,
                                       Rw[r].y + Rw[r + 1].y + Rw[r + 2].y);
            }
        }
        const int z = pl - 1;
        if (z >= z0 && a.clear) {
            // this tile of plane z in the accumulators being cleared; every
            // voxel of the grid lies in exactly one (tile, plane)
            if (TMA) {
                if (tid == 0 && guard(x0, a.nx, a.status) && guard(y0, a.ny, a.status) &&
                    guard(z, a.nz, a.status)) {
                    tma_store_3d(&clear_map, x0, y0, z, zbase);
                    if (y0 + kZeroRows < a.ny)
                        tma_store_3d(&clear_map, x0, y0 + kZeroRows, z, zbase);
                }
            } else if (xin) {
                unsigned long long *c = a.clear + ((size_t)z * a.ny + y0 + yb) * a.nx + x;
                for (int r = 0; r < nrows; ++r)
                    if (guard((c + (size_t)r * a.nx) - a.clear, plane * a.nz, a.status))
                        c[(size_t)r * a.nx] = 0ull;
            }
        }
        if (z >= z0) {
            const int sz = slot == 0 ? FSLOTS - 1 : slot - 1;  // plane z
            const unsigned long long *Pz = Pring + sz * SLOT;
            const bool any = nzf[0] | nzf[1] | nzf[2];
            const bool big = bigf[0] | bigf[1] | bigf[2];
#pragma unroll
            for (int r = 0; r < FRW; ++r) {
                unsigned v = 0;
                bool has = false;
                if (any && !big) {
                    const unsigned long long own = Pz[(yb + r + 1) * RS + tx + 1 + CO];
                    const unsigned c_own = (unsigned)(own >> 32);
                    // own samples if any, else the pooled neighbours (the own
                    // count is 0 then; its sum is dropped so only neighbours pool)
                    const unsigned S = c_own ? (unsigned)own
                                             : B[0][r].x + B[1][r].x + B[2][r].x - (unsigned)own;
                    const unsigned C = c_own ? c_own : B[0][r].y + B[1][r].y + B[2][r].y;
                    has = C != 0u;
                    v = mean_round_fast(S, has ? C : 1u);
                } else if (any) {
                    const unsigned long long own = Pz[(yb + r + 1) * RS + tx + 1 + CO];
                    unsigned long long S = own & 0xFFFFFFFFull, C = own >> 32;
                    saturated |= C >= (1ull << 24);
                    if (C == 0) {
                        S = 0ull - (own & 0xFFFFFFFFull);  // the centre is not a neighbour
                        for (int dz = 0; dz < 3; ++dz) {
                            const unsigned long long *Pd =
                                Pring + ((sz + FSLOTS - 1 + dz) % FSLOTS) * SLOT;
                            for (int dy = 0; dy < 3; ++dy)
                                for (int dx = 0; dx < 3; ++dx) {
                                    const unsigned long long w =
                                        Pd[(yb + r + dy) * RS + tx + dx + CO];
                                    S += w & 0xFFFFFFFFull;
                                    C += w >> 32;
                                }
                        }
                    }
                    has = C != 0;
                    if (has)
                        v = mean_round_u8(S, C);
                }
                const bool yin = r < nrows;
                if (xin && yin &&
                    guard((vout + (size_t)r * a.nx) - val, plane * a.nz, a.status))
                    vout[(size_t)r * a.nx] = (uint8_t)v;
                const unsigned bits = __ballot_sync(0xFFFFFFFFu, xin && yin && has);
                if (tx == 0 && yin &&
                    guard((mout + (size_t)r * a.nxw) - a.mask,
                          (size_t)a.nxw * a.ny * a.nz, a.status))
                    mout[(size_t)r * a.nxw] = bits;
            }
            vout += plane;
            mout += mplane;
        }
        __syncthreads();  // ring slot reuse
        return !(TMA && s_abort);
    };

    issue(z0 - 1);
    issue(z0);
    int slot = (z0 - 1 + FSLOTS) % FSLOTS;
    bool ok = true;
    // plane p's sums go to B[(p - z0 + 1) % 3]; unrolled by 3 so the slot is static
    for (int pl = z0 - 1; pl <= z1 && ok; pl += 3) {
        ok = step(pl, slot, B[0], nzf[0], bigf[0]);
        slot = slot + 1 == FSLOTS ? 0 : slot + 1;
        if (!ok || pl + 1 > z1)
            break;
        ok = step(pl + 1, slot, B[1], nzf[1], bigf[1]);
        slot = slot + 1 == FSLOTS ? 0 : slot + 1;
        if (!ok || pl + 2 > z1)
            break;
        ok = step(pl + 2, slot, B[2], nzf[2], bigf[2]);
        slot = slot + 1 == FSLOTS ? 0 : slot + 1;
    }
    if (TMA) {
        // after a timeout: wait (bounded) for the copies still in flight, so
        // none lands in shared memory after the CTA has gone
        if (tid == 0)
            for (int s = 0; s < FSLOTS; ++s)
                if (pending & (1u << s))
                    mbar_wait(bbase + 8u * s, (phase >> s) & 1u);
        if (tid == 0 && a.clear)
            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // the zero stores
    } else {
        cp_async_wait<0>();
    }
    if (__syncthreads_or(saturated) && tid == 0)
        atomicOr(a.status, USV_STATUS_SATURATED);
}

// ---- trilinear fill -----------------------------------------------------
//
// The nearest-neighbour fill's tiling and plane ring on (S, W) float pairs:
// a 32 x 32 column tile marched along z by 32 x 8 threads (4 rows each),
// one TMA tensor copy per plane two planes ahead into a 5-slot ring (zero
// fill outside the grid), bounded mbarrier waits.  Per plane each thread
// forms FP32 x-row sums of S and W for its 6 rows and from them the 3x3
// plane sums of its 4 voxels; the 3x3x3 sums add three planes.  A voxel with
// W > 0 takes S/W; an empty one (its own S and W are zero, so they add
// nothing) the pooled sum of S over the pooled sum of W of its neighbours;
// one IEEE division each.  Each thread waits for the plane on the
// mbarrier and needs no flag (the sums of a window without data are zero),
// so the CTA meets at one barrier per plane, for slot reuse.
__global__ void __launch_bounds__(FTX *FBY, 4)
    k_fill_tri(FillArgs a, const __grid_constant__ CUtensorMap map)
{
    constexpr int RS = kTmaW;                    // ring row stride (entries)
    constexpr int CO = 1;                        // ring column of halo column 0
    constexpr int SLOT = kTmaSlot;
    extern __shared__ __align__(128) unsigned long long Pring[];  // [FSLOTS][FPY][RS]
    __shared__ __align__(8) unsigned long long sbar[FSLOTS];
    __shared__ int s_abort;
    auto *val = static_cast<float *>(a.val);
    const int x0 = a.rx0 + blockIdx.x * FTX, y0 = a.ry0 + blockIdx.y * FTY;
    const int z0 = a.rz0 + blockIdx.z * a.zchunk, z1 = min(a.rz1, z0 + a.zchunk);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;
    const int x = x0 + tx, yb = 4 * ty;  // first of this thread's rows (tile-local)
    const size_t plane = (size_t)a.nx * a.ny;
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(Pring);
    const unsigned bbase = (unsigned)__cvta_generic_to_shared(sbar);
    unsigned phase = 0u;    // parity of each slot's next completion
    unsigned pending = 0u;  // thread 0: slots with a copy in flight

    auto issue = [&](int pl) {
        // (plane -1 is a real ring entry: the zero plane below the grid)
        if (tid == 0 && pl <= z1) {
            const int s = (pl + FSLOTS) % FSLOTS;
            mbar_expect_tx(bbase + 8u * s, kTmaBytes);
            tma_load_3d(sbase + (unsigned)(s * SLOT * 8), &map, x0 - 2, y0 - 1, pl,
                        bbase + 8u * s);
            pending |= 1u << s;
        }
    };
    // TMA writes whole 128-byte-aligned slots; a ring that is not aligned is
    // refused (reported as a failed wait) before any copy is issued
    if ((sbase & 127u) != 0u) {
        if (tid == 0)
            atomicOr(a.status, USV_STATUS_TIMEOUT);
        return;
    }
    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < FSLOTS; ++s)
            mbar_init(bbase + 8u * s, 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    // 3x3 plane sums (S, W) of this thread's rows; plane p lives in slot p % 3
    float2 B[3][FRW];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int r = 0; r < FRW; ++r)
            B[k][r] = make_float2(0.0f, 0.0f);

    const bool xin = x < a.nx;
    float *vout = val + ((size_t)z0 * a.ny + y0 + yb) * a.nx + x;
    uint32_t *mout = a.mask + ((size_t)z0 * a.ny + y0 + yb) * a.nxw + (x0 >> 5);
    const size_t mplane = (size_t)a.ny * a.nxw;
    const int nrows = min(FRW, a.ny - (y0 + yb));  // rows of this thread inside the grid

    // returns false when the CTA gives up (a wait ran out)
    auto step = [&](int pl, int slot, float2(&Bn)[FRW]) {
        issue(pl + 2);
        if (!mbar_wait(bbase + 8u * slot, (phase >> slot) & 1u)) {
            s_abort = 1;
            atomicOr(a.status, USV_STATUS_TIMEOUT);
        }
        phase ^= 1u << slot;
        if (tid == 0)
            pending &= ~(1u << slot);
        // every thread has seen the copy complete on the mbarrier, so the
        // plane is visible to it; the sums of a window without data are
        // zero, so no flag is needed
        const float2 *Pp = reinterpret_cast<const float2 *>(Pring + slot * SLOT);
        float2 R0 = make_float2(0.0f, 0.0f), R1 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k < FRW + 2; ++k) {  // rows yb-1 .. yb+4 = halo rows yb .. yb+5
            const float2 *row = Pp + (yb + k) * RS + tx + CO;
            const float2 p0 = row[0], p1 = row[1], p2 = row[2];
            const float2 R2 = make_float2(p0.x + p1.x + p2.x, p0.y + p1.y + p2.y);
            if (k >= 2)
                Bn[k - 2] = make_float2(R0.x + R1.x + R2.x, R0.y + R1.y + R2.y);
            R0 = R1;
            R1 = R2;
        }
        const int z = pl - 1;
        if (z >= z0) {
            const int sz = slot == 0 ? FSLOTS - 1 : slot - 1;  // plane z
            const float2 *Pz = reinterpret_cast<const float2 *>(Pring + sz * SLOT);
#pragma unroll
            for (int r = 0; r < FRW; ++r) {
                float v = 0.0f;
                bool has = false;
                {
                    const float2 own = Pz[(yb + r + 1) * RS + tx + 1 + CO];
                    const float S = own.y > 0.0f ? own.x : B[0][r].x + B[1][r].x + B[2][r].x;
                    const float W = own.y > 0.0f ? own.y : B[0][r].y + B[1][r].y + B[2][r].y;
                    has = W > 0.0f;
                    if (has)
                        v = __fdiv_rn(S, W);
                }
                const bool yin = r < nrows;
                if (xin && yin &&
                    guard((vout + (size_t)r * a.nx) - val, plane * a.nz, a.status))
                    vout[(size_t)r * a.nx] = v;
                const unsigned bits = __ballot_sync(0xFFFFFFFFu, xin && yin && has);
                if (tx == 0 && yin &&
                    guard((mout + (size_t)r * a.nxw) - a.mask,
                          (size_t)a.nxw * a.ny * a.nz, a.status))
                    mout[(size_t)r * a.nxw] = bits;
            }
            vout += plane;
            mout += mplane;
        }
        __syncthreads();  // ring slot reuse
        return !s_abort;
    };

    issue(z0 - 1);
    issue(z0);
    int slot = (z0 - 1 + FSLOTS) % FSLOTS;
    bool ok = true;
    // plane p's sums go to B[(p - z0 + 1) % 3]; unrolled by 3 so the slot is static
    for (int pl = z0 - 1; pl <= z1 && ok; pl += 3) {
        ok = step(pl, slot, B[0]);
        slot = slot + 1 == FSLOTS ? 0 : slot + 1;
        if (!ok || pl + 1 > z1)
            break;
        ok = step(pl + 1, slot, B[1]);
        slot = slot + 1 == FSLOTS ? 0 : slot + 1;
        if (!ok || pl + 2 > z1)
            break;
        ok = step(pl + 2, slot, B[2]);
        slot = slot + 1 == FSLOTS ? 0 : slot + 1;
    }
    // after a timeout: wait (bounded) for the copies still in flight, so none
    // lands in shared memory after the CTA has gone
    if (tid == 0)
        for (int s = 0; s < FSLOTS; ++s)
            if (pending & (1u << s))
                mbar_wait(bbase + 8u * s, (phase >> s) & 1u);
}

// Without TMA (odd nx): one thread per voxel, 32 x 8 tiles, three planes of
// the tile and its halo in shared memory, the 27 neighbours summed in turn.
__global__ void __launch_bounds__(TX *TY) k_fill_f32(FillArgs a)
{
    __shared__ float2 pl[3][PY][PX];
    const auto *acc = static_cast<const float2 *>(a.acc);
    auto *val = static_cast<float *>(a.val);
    const int x0 = a.rx0 + blockIdx.x * TX, y0 = a.ry0 + blockIdx.y * TY;
    const int z0 = a.rz0 + blockIdx.z * a.zchunk, z1 = min(a.rz1, z0 + a.zchunk);
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
        const size_t nvox = (size_t)a.nx * a.ny * a.nz;
        if (inside && guard(i, nvox, a.status))
            val[i] = v;
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, inside && has);
        const size_t mi = ((size_t)z * a.ny + y) * a.nxw + (x0 >> 5);
        if (tx == 0 && y < a.ny && guard(mi, (size_t)a.nxw * a.ny * a.nz, a.status))
            a.mask[mi] = bits;
        __syncthreads();
    }
}

// Region [lo, hi) (already clipped to the grid, lo[0] a multiple of 32)
dim3 fill_grid(FillArgs &a, int tx, int ty, int waves_ctas, const int *lo, const int *hi,
               int num_sms, int min_slab)
{
    const int gx = (hi[0] - lo[0] + tx - 1) / tx, gy = (hi[1] - lo[1] + ty - 1) / ty;
    const int nzr = hi[2] - lo[2];
    const long long want = (long long)num_sms * waves_ctas;
    long long zc = ((long long)gx * gy * nzr + want - 1) / want;
    zc = zc < min_slab ? min_slab : zc;
    zc = zc > nzr ? nzr : zc;
    a.zchunk = (int)(zc < 1 ? 1 : zc);
    a.rx0 = lo[0];
    a.ry0 = lo[1];
    a.rz0 = lo[2];
    a.rz1 = hi[2];
    return dim3(gx, gy, (nzr + a.zchunk - 1) / a.zchunk);
}

}  // namespace

namespace {

// cuTensorMapEncodeTiled from the driver, looked up once
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// Accumulators as a 3D tensor of u64 (x fastest): a 36 x 34 x 1 box to load
// planes, a 32 x 16 x 1 box to clear.  TMA needs 16-byte row and plane
// pitches, i.e. an even nx.
bool acc_tensor_map(const Volume &v, const void *acc, int box_x, int box_y, CUtensorMap *map)
{
    if (v.g.nx % 2 != 0 || (reinterpret_cast<uintptr_t>(acc) & 15) != 0)
        return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
    if (!enc)
        return false;
    const cuuint64_t dim[3] = {(cuuint64_t)v.g.nx, (cuuint64_t)v.g.ny, (cuuint64_t)v.g.nz};
    const cuuint64_t stride[2] = {(cuuint64_t)v.g.nx * 8, (cuuint64_t)v.g.nx * v.g.ny * 8};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1u};
    const cuuint32_t estride[3] = {1u, 1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void *>(acc), dim, stride, box,
               estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_fill_pnn(const Volume &v, const int *lo, const int *hi, cudaStream_t st,
                            void *clear, int withhold)
{
    FillArgs a{v.acc, v.val, v.mask, v.status, v.g.nx, v.g.ny, v.g.nz, v.nxw, 0, 0, 0, 0, 0,
               static_cast<unsigned long long *>(clear), withhold};
    if (clear && (lo[0] != 0 || lo[1] != 0 || lo[2] != 0 || hi[0] != v.g.nx ||
                  hi[1] != v.g.ny || hi[2] != v.g.nz))
        return cudaErrorInvalidValue;  // clearing covers the whole grid only
    // ~6 waves of 4 resident CTAs per SM; slabs of at least 16 planes
    const dim3 grid = fill_grid(a, FTX, FTY, 4 * 6, lo, hi, v.num_sms, 16);
    if (grid.x == 0 || grid.y == 0 || grid.z == 0)
        return cudaSuccess;
    cudaError_t e = prepare_kernel(reinterpret_cast<const void *>(k_fill_pnn<false>), kFillSmemCp);
    if (e == cudaSuccess)
        e = prepare_kernel(reinterpret_cast<const void *>(k_fill_pnn<true>), kFillSmemTma);
    if (e != cudaSuccess)
        return e;
    alignas(64) CUtensorMap map, cmap;
    std::memset(&cmap, 0, sizeof(cmap));
    if (acc_tensor_map(v, v.acc, kTmaW, FPY, &map) &&
        (!clear || acc_tensor_map(v, clear, FTX, kZeroRows, &cmap))) {
        k_fill_pnn<true><<<grid, dim3(FTX, FBY), kFillSmemTma, st>>>(a, map, cmap);
    } else if (withhold >= 0) {
        return cudaErrorNotSupported;  // only the tensor-copy path waits on the device
    } else {
        std::memset(&map, 0, sizeof(map));
        k_fill_pnn<false><<<grid, dim3(FTX, FBY), kFillSmemCp, st>>>(a, map, cmap);
    }
    return cudaGetLastError();
}

cudaError_t launch_fill_trilinear(const Volume &v, const int *lo, const int *hi, cudaStream_t st)
{
    FillArgs a{v.acc, v.val, v.mask, v.status, v.g.nx, v.g.ny, v.g.nz, v.nxw, 0, 0, 0, 0, 0};
    alignas(64) CUtensorMap map;
    if (acc_tensor_map(v, v.acc, kTmaW, FPY, &map)) {
        // ~6 waves of 4 resident CTAs per SM; slabs of at least 16 planes
        const dim3 grid = fill_grid(a, FTX, FTY, 4 * 6, lo, hi, v.num_sms, 16);
        if (grid.x == 0 || grid.y == 0 || grid.z == 0)
            return cudaSuccess;
        const int smem = FSLOTS * kTmaSlot * 8;
        const cudaError_t e = prepare_kernel(reinterpret_cast<const void *>(k_fill_tri), smem);
        if (e != cudaSuccess)
            return e;
        k_fill_tri<<<grid, dim3(FTX, FBY), smem, st>>>(a, map);
        return cudaGetLastError();
    }
    const dim3 grid = fill_grid(a, TX, TY, 8 * 8, lo, hi, v.num_sms, 16);
    if (grid.x == 0 || grid.y == 0 || grid.z == 0)
        return cudaSuccess;
    k_fill_f32<<<grid, dim3(TX, TY), 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace usv
