// usv_insert_pnn_noalloc: nearest-neighbour insertion for callers that must
// not allocate device memory.
//
// Some hosts cannot call cudaMalloc on the path that feeds frames: a
// real-time acquisition loop whose memory is fixed up front (allocation can
// block and synchronise the device, which breaks a 30 fps frame budget), an
// embedded or certified deployment that forbids allocation after start-up,
// or a plugin inside another framework that owns every buffer.  They cannot
// hand the library the volume storage that usv_volume_create() expects,
// because that storage also holds the per-frame set-up scratch.
//
// This entry point takes only the caller's inputs (frames, poses,
// calibration, grid geometry) and output (the packed accumulators) and keeps
// its scratch -- the per-frame map records written by the set-up kernel and
// read by the insertion kernel -- in a fixed array compiled into the
// library.  Every GPU that loads the library holds that array (about 160 KB)
// until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "usv_internal.cuh"

namespace usv {

namespace {

constexpr int kNoAllocFrames = USV_NOALLOC_MAX_FRAMES;

// The scratch.  Shared by every call on a device; no call needs any of it
// to start at zero, because each call writes all the records it reads.
static __device__ __align__(256) FrameRec g_noalloc_rec[kNoAllocFrames];
// Status bits of calls that pass no status word of their own.
static __device__ __align__(256) uint32_t g_noalloc_status[64];

constexpr int kMaxDevices = 64;

// Per device: the scratch's device addresses and the SM count, looked up
// with that device current, and the id of the CUDA context they belong to.
// A context destroyed and created again (cudaDeviceReset) loads the library's
// module anew, so the addresses are looked up again for the new context.
struct DeviceScratch {
    unsigned long long ctx_id;
    FrameRec *rec;
    uint32_t *status;
    int num_sms;
};
std::mutex g_mu;
DeviceScratch g_dev[kMaxDevices];

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// Id of the current context (driver entry points, fetched once); 0 if the
// driver does not provide one, in which case the first lookup is kept (ids
// are unique for the life of the process and never 0).
unsigned long long current_ctx_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0)
        return id;
    return 0;
}

// The scratch of device `dev` (current) in its current context.  In host
// code the symbols are only host-side stand-ins; their device addresses
// must be asked for, once per device and context.
cudaError_t scratch_for(int dev, DeviceScratch *out)
{
    // cudaSetDevice initialises the device's primary context and makes it
    // current, so the context id below is that of the context the next
    // launch uses (also right after a cudaDeviceReset)
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceScratch &d = g_dev[dev];
    const unsigned long long id = current_ctx_id();
    if (!d.rec || id != d.ctx_id) {
        void *r = nullptr, *s = nullptr;
        int sms = 0;
        e = cudaGetSymbolAddress(&r, g_noalloc_rec);
        if (e == cudaSuccess)
            e = cudaGetSymbolAddress(&s, g_noalloc_status);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return e;
        d.rec = static_cast<FrameRec *>(r);
        d.status = static_cast<uint32_t *>(s);
        d.num_sms = sms;
        d.ctx_id = id;
    }
    *out = d;
    return cudaSuccess;
}

}  // namespace

}  // namespace usv

extern "C" int usv_insert_pnn_noalloc(uint64_t *accum_dev, usv_grid grid,
                                      const double spacing_mm[3], const double origin_mm[3],
                                      const void *images_dev, int32_t n, int32_t H, int32_t W,
                                      const double *poses_dev, const usv_calibration *cal,
                                      uint32_t *status_dev, void *stream)
{
    if (!accum_dev || !cal || n < 0)
        return USV_ERR_ARG;
    if (grid.nx < 1 || grid.ny < 1 || grid.nz < 1 ||
        (unsigned long long)grid.nx * grid.ny * grid.nz > 0x7FFFFFFFull)
        return USV_ERR_ARG;
    if (!spacing_mm || !origin_mm)
        return USV_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(spacing_mm[a]) || !(spacing_mm[a] > 0.0) ||
            !std::isfinite(origin_mm[a]))
            return USV_ERR_ARG;
    if (n > usv::kNoAllocFrames)
        return USV_ERR_RANGE;  // more frames than the fixed scratch holds
    if (n == 0)
        return USV_OK;
    if (!images_dev || !poses_dev || (reinterpret_cast<uintptr_t>(poses_dev) & 7) != 0 ||
        (reinterpret_cast<uintptr_t>(accum_dev) & 7) != 0)
        return USV_ERR_ARG;
    if (H < 1 || W < 1)
        return USV_ERR_ARG;
    if (H > usv::kMaxDim || W > usv::kMaxDim)
        return USV_ERR_RANGE;
    if (cal->geom != USV_LINEAR)
        return USV_ERR_UNSUPPORTED;
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(cal->image_to_probe[i]))
            return USV_ERR_ARG;
    if (cal->image_to_probe[12] != 0.0 || cal->image_to_probe[13] != 0.0 ||
        cal->image_to_probe[14] != 0.0 || cal->image_to_probe[15] != 1.0)
        return USV_ERR_ARG;
    if (!(std::isfinite(cal->sx_mm) && std::isfinite(cal->sy_mm) && cal->sx_mm > 0.0 &&
          cal->sy_mm > 0.0))
        return USV_ERR_ARG;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= usv::kMaxDevices)
        return USV_ERR_CUDA;
    usv::DeviceScratch sc;
    if (usv::scratch_for(dev, &sc) != cudaSuccess)
        return USV_ERR_CUDA;

    // A stack-only view of the caller's accumulators for the shared launchers.
    usv::Volume v;
    std::memset(&v, 0, sizeof(v));
    v.g = grid;
    v.mode = USV_PNN;
    v.acc = accum_dev;
    v.rec = sc.rec;
    v.status = status_dev ? status_dev : sc.status;
    v.device = dev;
    v.num_sms = sc.num_sms;  // lets small batches spread over the GPU, as usv_insert_frames
    usv::SetupParams sp;
    std::memcpy(sp.K, cal->image_to_probe, sizeof(sp.K));
    for (int a = 0; a < 3; ++a) {
        sp.s[a] = spacing_mm[a];
        sp.o[a] = origin_mm[a];
    }
    sp.sx = cal->sx_mm;
    sp.sy = cal->sy_mm;
    sp.convex = 0;
    sp.first_rows = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = usv::launch_frame_setup(poses_dev, n, sp, v.rec, v.status, st);
    if (e == cudaSuccess)
        e = usv::launch_insert_pnn(v, static_cast<const uint8_t *>(images_dev), n, H, W, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return USV_ERR_CUDA;
    }
    return USV_OK;
}
