// The C ABI of include/usvol.h: host-side argument checks, the storage
// layout inside caller-provided device memory, and the launches.  Nothing
// here allocates device memory; the only host allocation is the handle.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "usv_internal.cuh"

namespace usv {

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool grid_ok(usv_grid g)
{
    if (g.nx < 1 || g.ny < 1 || g.nz < 1)
        return false;
    const unsigned long long n = (unsigned long long)g.nx * g.ny * g.nz;
    return n <= 0x7FFFFFFFull;
}

bool finite3(const double *v)
{
    return v && std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

bool affine_ok(const double *m)
{
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(m[i]))
            return false;
    return m[12] == 0.0 && m[13] == 0.0 && m[14] == 0.0 && m[15] == 1.0;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev)
            cudaSetDevice(dev);
        else
            prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

thread_local const char *t_last_cuda_error = "no error";

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess)
        return USV_OK;
    t_last_cuda_error = cudaGetErrorString(e);
    cudaGetLastError();  // clear a sticky launch error so later calls are not blamed
    return USV_ERR_CUDA;
}

}  // namespace

// Pinned, device-mapped host memory through which host-side poses reach
// the device: each insertion launch copies its frames' poses (128 B per
// frame) into a region of the ring, and the frame set-up kernel reads them
// from there over the host link.  No copy engine is involved: an
// asynchronous host->device copy on the caller's stream would queue behind
// the caller's own bulk frame copies on the copy engines and hold back the
// insertion.  A region is written again only after the work that read it
// has completed (an event per region), so the host can run several calls
// ahead of the device.
class PoseRing {
public:
    static constexpr size_t kBytes = 2u << 20;  // 2 MB: four full launches of 4096 frames
    static constexpr int kMaxInFlight = 64;

    cudaError_t init()
    {
        cudaError_t e = cudaHostAlloc(reinterpret_cast<void **>(&base_), kBytes,
                                      cudaHostAllocMapped);
        void *dev = nullptr;
        if (e == cudaSuccess)
            e = cudaHostGetDevicePointer(&dev, base_, 0);
        dev_ = static_cast<const char *>(dev);
        for (int i = 0; e == cudaSuccess && i < kMaxInFlight; ++i)
            e = cudaEventCreateWithFlags(&ev_[i], cudaEventDisableTiming);
        return e;
    }
    ~PoseRing()
    {
        // the device may still be reading regions: wait for their readers
        for (; count_ > 0; --count_, first_ = (first_ + 1) % kMaxInFlight)
            cudaEventSynchronize(ev_[first_]);
        for (int i = 0; i < kMaxInFlight; ++i)
            if (ev_[i])
                cudaEventDestroy(ev_[i]);
        if (base_)
            cudaFreeHost(base_);
    }

    // Copy `bytes` (<= kBytes) from `src` into a free region and return its
    // device address in *dev; fence() must follow once its reader is queued.
    cudaError_t put(const void *src, size_t bytes, const void **dev)
    {
        size_t off = head_;
        if (off + bytes > kBytes)
            off = 0;  // wrap: regions never straddle the end
        // wait for the oldest in-flight regions until [off, off + bytes) is free
        while (count_ > 0 && (overlaps(first_, off, bytes) || count_ == kMaxInFlight)) {
            cudaError_t e = cudaEventSynchronize(ev_[first_]);
            if (e != cudaSuccess)
                return e;
            first_ = (first_ + 1) % kMaxInFlight;
            --count_;
        }
        std::memcpy(base_ + off, src, bytes);
        put_off_ = off;
        put_bytes_ = bytes;
        *dev = dev_ + off;
        return cudaSuccess;
    }

    // The region of the last put() stays in use until the work queued on
    // `st` so far has completed.
    cudaError_t fence(cudaStream_t st)
    {
        const int slot = (first_ + count_) % kMaxInFlight;
        cudaError_t e = cudaEventRecord(ev_[slot], st);
        if (e != cudaSuccess)
            return e;
        use_off_[slot] = put_off_;
        use_bytes_[slot] = put_bytes_;
        ++count_;
        head_ = put_off_ + put_bytes_;
        return cudaSuccess;
    }

private:
    bool overlaps(int slot, size_t off, size_t bytes) const
    {
        return use_off_[slot] < off + bytes && off < use_off_[slot] + use_bytes_[slot];
    }

    char *base_ = nullptr;
    const char *dev_ = nullptr;
    size_t head_ = 0, put_off_ = 0, put_bytes_ = 0;
    cudaEvent_t ev_[kMaxInFlight] = {};
    size_t use_off_[kMaxInFlight] = {}, use_bytes_[kMaxInFlight] = {};
    int first_ = 0, count_ = 0;
};

Layout layout_for(usv_grid g, int mode)
{
    Layout L{};
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const size_t nxw = ((size_t)g.nx + 31) / 32;
    size_t off = 0;
    L.acc = off;
    off += align_up(n * 8);
    L.val = off;
    off += align_up(n * ((mode & ~USV_SPARE_ACCUM) == USV_PNN ? 1 : 4));
    L.mask = off;
    off += align_up((size_t)g.nz * g.ny * nxw * 4);
    L.rec = off;
    off += align_up((size_t)kRecCap * sizeof(FrameRec));
    L.beams = off;
    off += align_up((size_t)kBeamCap * sizeof(double2));
    L.status = off;
    off += kAlign;
    L.spare = 0;
    if (mode & USV_SPARE_ACCUM) {
        L.spare = off;
        off += align_up(n * 8);
    }
    L.total = off;
    return L;
}

}  // namespace usv

using usv::Volume;

extern "C" {

int usv_abi_version(void) { return USVOL_ABI_VERSION; }

const char *usv_last_cuda_error(void) { return usv::t_last_cuda_error; }

const char *usv_strerror(int code)
{
    switch (code) {
    case USV_OK: return "ok";
    case USV_ERR_ARG: return "invalid argument";
    case USV_ERR_RANGE: return "argument out of supported range";
    case USV_ERR_CUDA: return "CUDA runtime error";
    case USV_ERR_TIMEOUT: return "bounded device wait timed out";
    case USV_ERR_NOMEM: return "device storage smaller than usv_volume_bytes()";
    case USV_ERR_UNSUPPORTED: return "unsupported mode/geometry/dtype combination";
    default: return "unknown usvol error";
    }
}

size_t usv_volume_bytes(usv_grid grid, int32_t mode)
{
    const int32_t base = mode & ~USV_SPARE_ACCUM;
    if (!usv::grid_ok(grid) || (base != USV_PNN && base != USV_TRILINEAR))
        return 0;
    return usv::layout_for(grid, mode).total;
}

int usv_volume_create(usv_grid grid, const double spacing_mm[3], const double origin_mm[3],
                      int32_t mode, void *device_storage, size_t storage_bytes, usv_volume **out)
{
    if (!out)
        return USV_ERR_ARG;
    *out = nullptr;
    const int32_t base_mode = mode & ~USV_SPARE_ACCUM;
    if (!usv::grid_ok(grid) || (base_mode != USV_PNN && base_mode != USV_TRILINEAR))
        return USV_ERR_ARG;
    if (!usv::finite3(spacing_mm) || !usv::finite3(origin_mm))
        return USV_ERR_ARG;
    if (!(spacing_mm[0] > 0.0 && spacing_mm[1] > 0.0 && spacing_mm[2] > 0.0))
        return USV_ERR_ARG;
    if (!device_storage || (reinterpret_cast<uintptr_t>(device_storage) % usv::kAlign) != 0)
        return USV_ERR_ARG;
    const usv::Layout L = usv::layout_for(grid, mode);
    if (storage_bytes < L.total)
        return USV_ERR_NOMEM;
    cudaPointerAttributes attr;
    if (int rc = usv::cuda_rc(cudaPointerGetAttributes(&attr, device_storage)))
        return rc;
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return USV_ERR_ARG;
    int sms = 0;
    if (int rc = usv::cuda_rc(
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, attr.device)))
        return rc;
    Volume *v = new (std::nothrow) Volume();
    if (!v)
        return USV_ERR_NOMEM;
    v->g = grid;
    for (int a = 0; a < 3; ++a) {
        v->spacing[a] = spacing_mm[a];
        v->origin[a] = origin_mm[a];
    }
    v->mode = base_mode;
    v->base = static_cast<char *>(device_storage);
    v->bytes = storage_bytes;
    v->acc = v->base + L.acc;
    v->spare = L.spare ? v->base + L.spare : nullptr;
    v->val = v->base + L.val;
    v->mask = reinterpret_cast<uint32_t *>(v->base + L.mask);
    v->nxw = (grid.nx + 31) / 32;
    v->rec = reinterpret_cast<usv::FrameRec *>(v->base + L.rec);
    v->beams = reinterpret_cast<double2 *>(v->base + L.beams);
    v->status = reinterpret_cast<uint32_t *>(v->base + L.status);
    v->num_sms = sms;
    v->device = attr.device;
    v->ring = new (std::nothrow) usv::PoseRing();
    if (!v->ring) {
        delete v;
        return USV_ERR_NOMEM;
    }
    {
        usv::DeviceGuard g(attr.device);
        if (int rc = usv::cuda_rc(v->ring->init())) {
            delete v->ring;
            delete v;
            return rc;
        }
    }
    *out = reinterpret_cast<usv_volume *>(v);
    return USV_OK;
}

int usv_volume_destroy(usv_volume *vol)
{
    if (!vol)
        return USV_ERR_ARG;
    Volume *v = reinterpret_cast<Volume *>(vol);
    {
        usv::DeviceGuard g(v->device);
        delete v->ring;  // waits for the set-up kernels that read the ring, then frees it
    }
    delete v;
    return USV_OK;
}

int usv_volume_reset(usv_volume *vol, void *stream)
{
    if (!vol)
        return USV_ERR_ARG;
    Volume &v = *reinterpret_cast<Volume *>(vol);
    usv::DeviceGuard g(v.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const usv::Layout L = usv::layout_for(v.g, v.mode);
    cudaError_t e = usv::launch_zero(v.acc, L.val - L.acc, v.num_sms, st);  // = the spare's size
    if (e == cudaSuccess)
        e = usv::launch_zero(v.status, usv::kAlign, v.num_sms, st);
    return usv::cuda_rc(e);
}

namespace usv {
// acc_override / cfg_override: insert into other accumulators with a given
// tile shape (the autotuner); null = the volume's own, tile_for().
// poses_on_host: `poses` is host memory, staged launch by launch through the
// volume's pinned ring, which the set-up kernel reads in place.
int insert_impl(usv_volume *vol, const void *images_dev, int32_t n, int32_t H, int32_t W,
                int32_t dtype, const double *poses, const usv_calibration *cal,
                const int32_t *first_rows_dev, void *stream, void *acc_override = nullptr,
                const TileCfg *cfg_override = nullptr, int tri_min_rows = 8,
                bool tri_carry = true, bool poses_on_host = false);
}

int usv_insert_frames(usv_volume *vol, const void *images_dev, int32_t n, int32_t H, int32_t W,
                      int32_t dtype, const double *poses_host, const usv_calibration *cal,
                      void *stream)
{
    return usv::insert_impl(vol, images_dev, n, H, W, dtype, poses_host, cal, nullptr, stream,
                            nullptr, nullptr, 8, true, true);
}

int usv_insert_frames_dev(usv_volume *vol, const void *images_dev, int32_t n, int32_t H,
                          int32_t W, int32_t dtype, const double *poses_dev,
                          const usv_calibration *cal, void *stream)
{
    return usv::insert_impl(vol, images_dev, n, H, W, dtype, poses_dev, cal, nullptr, stream);
}

int usv_frames_voxel_box(usv_grid grid, const double spacing_mm[3], const double origin_mm[3],
                         const double *poses_host, int32_t n, int32_t H, int32_t W,
                         const usv_calibration *cal, int32_t margin, int32_t lo[3], int32_t hi[3])
{
    if (!cal || !lo || !hi || n < 0 || H < 1 || W < 1 || margin < 0)
        return USV_ERR_ARG;
    if (!usv::grid_ok(grid) || !usv::finite3(spacing_mm) || !usv::finite3(origin_mm) ||
        !(spacing_mm[0] > 0.0 && spacing_mm[1] > 0.0 && spacing_mm[2] > 0.0))
        return USV_ERR_ARG;
    if (n > 0 && !poses_host)
        return USV_ERR_ARG;
    if (!usv::affine_ok(cal->image_to_probe))
        return USV_ERR_ARG;
    // the frame's in-plane extent (x, z in mm of the image frame): a
    // rectangle for a linear probe; for a convex one the sector's bounding
    // rectangle (x = r sin theta, z = r cos theta - r0)
    double x0, x1, z0, z1;
    if (cal->geom == USV_CONVEX) {
        if (!(std::isfinite(cal->r0_mm) && std::isfinite(cal->dr_mm) &&
              std::isfinite(cal->sector_deg) && cal->r0_mm >= 0.0 && cal->dr_mm > 0.0 &&
              cal->sector_deg > 0.0 && cal->sector_deg < 180.0))
            return USV_ERR_ARG;
        const double half = cal->sector_deg * 3.14159265358979323846 / 360.0;
        const double R = cal->r0_mm + (double)(H - 1) * cal->dr_mm;
        x0 = -R * std::sin(half);
        x1 = R * std::sin(half);
        z0 = cal->r0_mm * std::cos(half) - cal->r0_mm;
        z1 = R - cal->r0_mm;
    } else if (cal->geom == USV_LINEAR) {
        if (!(std::isfinite(cal->sx_mm) && std::isfinite(cal->sy_mm) && cal->sx_mm > 0.0 &&
              cal->sy_mm > 0.0))
            return USV_ERR_ARG;
        x0 = 0.0;
        x1 = (double)(W - 1) * cal->sx_mm;
        z0 = 0.0;
        z1 = (double)(H - 1) * cal->sy_mm;
    } else {
        return USV_ERR_ARG;
    }
    const double *K = cal->image_to_probe;
    double qlo[3] = {INFINITY, INFINITY, INFINITY}, qhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int f = 0; f < n; ++f) {
        const double *P = poses_host + (size_t)f * 16;
        if (!usv::affine_ok(P))
            continue;  // skipped by the insertion too
        for (int c = 0; c < 4; ++c) {
            const double pt[4] = {(c & 1) ? x1 : x0, 0.0, (c & 2) ? z1 : z0, 1.0};
            double kp[4];
            for (int i = 0; i < 4; ++i)
                kp[i] = K[4 * i] * pt[0] + K[4 * i + 1] * pt[1] + K[4 * i + 2] * pt[2] +
                        K[4 * i + 3] * pt[3];
            for (int a = 0; a < 3; ++a) {
                const double w = P[4 * a] * kp[0] + P[4 * a + 1] * kp[1] + P[4 * a + 2] * kp[2] +
                                 P[4 * a + 3] * kp[3];
                const double q = (w - origin_mm[a]) / spacing_mm[a];
                qlo[a] = std::min(qlo[a], q);
                qhi[a] = std::max(qhi[a], q);
            }
        }
    }
    const int gn[3] = {grid.nx, grid.ny, grid.nz};
    for (int a = 0; a < 3; ++a) {
        if (!(qlo[a] <= qhi[a]) || !std::isfinite(qlo[a]) || !std::isfinite(qhi[a])) {
            lo[0] = lo[1] = lo[2] = hi[0] = hi[1] = hi[2] = 0;  // no valid frame: empty
            return USV_OK;
        }
    }
    for (int a = 0; a < 3; ++a) {
        // voxels written: nearest (floor(q + 1/2)) or trilinear corners
        // (floor(q), floor(q) + 1); one more voxel each side absorbs the
        // rounding of this FP64 evaluation against the exact insertion map
        const double l = std::floor(qlo[a]) - 1.0 - margin, h = std::floor(qhi[a]) + 3.0 + margin;
        lo[a] = (int32_t)std::max(0.0, std::min((double)gn[a], l));
        hi[a] = (int32_t)std::max(0.0, std::min((double)gn[a], h));
    }
    return USV_OK;
}

int usv_insert_frames_cut(usv_volume *vol, const void *images_dev, int32_t n, int32_t H,
                          int32_t W, int32_t dtype, const double *poses_dev,
                          const usv_calibration *cal, const int32_t *first_row_dev, void *stream)
{
    if (!first_row_dev && n > 0)
        return USV_ERR_ARG;
    return usv::insert_impl(vol, images_dev, n, H, W, dtype, poses_dev, cal, first_row_dev,
                            stream);
}

int usv_cut_rows_alg1(const double *poses_dev, int32_t n, int32_t H, const usv_calibration *cal,
                      const usv_alg1_params *p, int32_t *first_row_dev, void *stream)
{
    if (!cal || !p || n < 0 || H < 1)
        return USV_ERR_ARG;
    if (n == 0)
        return USV_OK;
    if (!poses_dev || !first_row_dev || (reinterpret_cast<uintptr_t>(poses_dev) & 7) != 0)
        return USV_ERR_ARG;
    if (!usv::affine_ok(cal->image_to_probe))
        return USV_ERR_ARG;
    const double row_mm = cal->geom == USV_CONVEX ? cal->dr_mm : cal->sy_mm;
    if (!(std::isfinite(row_mm) && row_mm > 0.0))
        return USV_ERR_ARG;
    const double vals[] = {p->K, p->D_mm, p->L_mm, p->spine_dir[0], p->spine_dir[1],
                           p->spine_dir[2], p->p1_mm[0], p->p1_mm[1], p->p1_mm[2]};
    for (double v : vals)
        if (!std::isfinite(v))
            return USV_ERR_ARG;
    usv::Alg1Params ap;
    std::memcpy(ap.K, cal->image_to_probe, sizeof(ap.K));
    ap.k = p->K;
    ap.d_mm = p->D_mm;
    ap.half_l_mm = p->L_mm * 0.5;
    for (int a = 0; a < 3; ++a) {
        ap.dir[a] = p->spine_dir[a];
        ap.p1[a] = p->p1_mm[a];
    }
    ap.row_mm = row_mm;
    return usv::cuda_rc(usv::launch_cut_rows_alg1(poses_dev, n, H, ap, first_row_dev,
                                                  static_cast<cudaStream_t>(stream)));
}

int usv_bone_rows_alg2(const uint8_t *images_dev, int32_t n, int32_t H, int32_t W,
                       const usv_alg2_params *p, int32_t *bone_row_dev, int32_t *first_row_dev,
                       void *stream)
{
    if (!p || n < 0 || H < 1 || W < 1)
        return USV_ERR_ARG;
    if (n == 0)
        return USV_OK;
    if (!images_dev || !bone_row_dev || !first_row_dev)
        return USV_ERR_ARG;
    if (H > USV_ALG2_MAX_ROWS || W > usv::kMaxDim)
        return USV_ERR_RANGE;
    if (p->search_from_row < 0 || p->search_from_row >= H || p->drop_rows < 1 ||
        p->window < 1 || (p->window & 1) == 0 || p->margin_rows < 0)
        return USV_ERR_ARG;
    return usv::cuda_rc(usv::launch_bone_rows_alg2(images_dev, n, H, W, p->search_from_row,
                                                   p->drop_rows, p->window, p->margin_rows,
                                                   bone_row_dev, first_row_dev,
                                                   static_cast<cudaStream_t>(stream)));
}

int usv_pose_loss_grad(usv_volume *vol, const void *images_dev, int32_t n, int32_t H, int32_t W,
                       int32_t dtype, const double *poses_dev, const usv_calibration *cal,
                       int32_t z_lo, int32_t z_hi, float eps, const float *target_dev,
                       float *proj_dev, float *adj_scratch_dev, double *loss_dev,
                       double *grad_dev, void *stream)
{
    if (!vol || !cal || !target_dev || !proj_dev || !adj_scratch_dev || !loss_dev || !grad_dev)
        return USV_ERR_ARG;
    Volume &v = *reinterpret_cast<Volume *>(vol);
    if (v.mode != USV_TRILINEAR || cal->geom != USV_LINEAR)
        return USV_ERR_UNSUPPORTED;
    if (n < 1 || n > usv::kRecCap)
        return USV_ERR_RANGE;
    if (z_lo < 0 || z_hi > v.g.nz || z_lo >= z_hi)
        return USV_ERR_RANGE;
    if (!(std::isfinite(eps) && eps > 0.0f))
        return USV_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(adj_scratch_dev) & 7) != 0)
        return USV_ERR_ARG;
    usv::DeviceGuard g(v.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the gradient kernel recomputes every sample on 64-row tiles, so the
    // forward splat keeps 64-row tiles (same column anchors, same cells);
    // without the corner carry, which costs more than it saves on the
    // smaller volumes of pose refinement (their atomics stay in L2)
    int rc = usv_volume_reset(vol, stream);
    if (rc == USV_OK)
        rc = usv::insert_impl(vol, images_dev, n, H, W, dtype, poses_dev, cal, nullptr, stream,
                              nullptr, &usv::kTriTileDefault, usv::kTriTileDefault.tile_h,
                              false);
    if (rc != USV_OK)
        return rc;
    cudaError_t e = usv::launch_zero_f64(loss_dev, 1, st);
    if (e == cudaSuccess)
        e = usv::launch_zero_f64(grad_dev, 6 * n, st);
    if (e == cudaSuccess)
        e = usv::launch_soft_project_adjoint(v, z_lo, z_hi, eps, target_dev, proj_dev,
                                             reinterpret_cast<float2 *>(adj_scratch_dev),
                                             loss_dev, st);
    if (e == cudaSuccess)
        e = usv::launch_pose_grad(v, images_dev, dtype == USV_F32, n, H, W, z_lo, z_hi,
                                  reinterpret_cast<const float2 *>(adj_scratch_dev), grad_dev,
                                  st);
    return usv::cuda_rc(e);
}

int usv_apply_pose_delta(const double *poses_dev, const double *delta_dev, int32_t n, int32_t H,
                         int32_t W, const usv_calibration *cal, double *poses_out_dev,
                         void *stream)
{
    if (!cal || n < 0 || H < 1 || W < 1)
        return USV_ERR_ARG;
    if (n == 0)
        return USV_OK;
    if (!poses_dev || !delta_dev || !poses_out_dev || poses_out_dev == poses_dev)
        return USV_ERR_ARG;
    if (cal->geom != USV_LINEAR)
        return USV_ERR_UNSUPPORTED;
    if (!usv::affine_ok(cal->image_to_probe))
        return USV_ERR_ARG;
    const double cx = 0.5 * (double)(W - 1) * cal->sx_mm, cz = 0.5 * (double)(H - 1) * cal->sy_mm;
    return usv::cuda_rc(usv::launch_apply_pose_delta(poses_dev, delta_dev, n, cx, cz,
                                                     cal->image_to_probe, poses_out_dev,
                                                     static_cast<cudaStream_t>(stream)));
}

int usv::insert_impl(usv_volume *vol, const void *images_dev, int32_t n, int32_t H, int32_t W,
                     int32_t dtype, const double *poses, const usv_calibration *cal,
                     const int32_t *first_rows_dev, void *stream, void *acc_override,
                     const TileCfg *cfg_override, int tri_min_rows, bool tri_carry,
                     bool poses_on_host)
{
    if (!vol || !cal || n < 0)
        return USV_ERR_ARG;
    if (n == 0)
        return USV_OK;
    if (!images_dev || !poses)
        return USV_ERR_ARG;
    if (!poses_on_host && (reinterpret_cast<uintptr_t>(poses) & 7) != 0)
        return USV_ERR_ARG;
    if (H < 1 || W < 1)
        return USV_ERR_ARG;
    if (H > usv::kMaxDim || W > usv::kMaxDim)
        return USV_ERR_RANGE;
    if (dtype != USV_U8 && dtype != USV_F32)
        return USV_ERR_ARG;
    if (cal->geom != USV_LINEAR && cal->geom != USV_CONVEX)
        return USV_ERR_ARG;
    if (!usv::affine_ok(cal->image_to_probe))
        return USV_ERR_ARG;
    Volume v = *reinterpret_cast<Volume *>(vol);  // a view: acc may be redirected
    if (acc_override)
        v.acc = acc_override;
    const usv::TileCfg cfg = cfg_override ? *cfg_override : usv::tile_for(v, H, W);
    usv::SetupParams sp;
    std::memcpy(sp.K, cal->image_to_probe, sizeof(sp.K));
    for (int a = 0; a < 3; ++a) {
        sp.s[a] = v.spacing[a];
        sp.o[a] = v.origin[a];
    }
    const bool convex = cal->geom == USV_CONVEX;
    sp.convex = convex ? 1 : 0;
    sp.first_rows = nullptr;
    if (convex) {
        if (!(std::isfinite(cal->r0_mm) && std::isfinite(cal->dr_mm) &&
              std::isfinite(cal->sector_deg)))
            return USV_ERR_ARG;
        if (!(cal->r0_mm >= 0.0 && cal->dr_mm > 0.0 && cal->sector_deg > 0.0 &&
              cal->sector_deg < 180.0) || W < 2)
            return USV_ERR_ARG;
        if (cal->r0_mm + (H - 1) * cal->dr_mm > 16384.0)
            return USV_ERR_RANGE;
        sp.sx = 1.0;
        sp.sy = 1.0;
    } else {
        if (!(std::isfinite(cal->sx_mm) && std::isfinite(cal->sy_mm) && cal->sx_mm > 0.0 &&
              cal->sy_mm > 0.0))
            return USV_ERR_ARG;
        sp.sx = cal->sx_mm;
        sp.sy = cal->sy_mm;
    }
    if (v.mode == USV_PNN && (dtype != USV_U8 || convex))
        return USV_ERR_UNSUPPORTED;

    usv::DeviceGuard g(v.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (poses_on_host) {
        // the staging ring's host-side waits and copies from host memory
        // have no place in a captured graph: capture the device-pose form
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (int rc = usv::cuda_rc(cudaStreamIsCapturing(st, &cs)))
            return rc;
        if (cs != cudaStreamCaptureStatusNone)
            return USV_ERR_UNSUPPORTED;
    }
    const size_t elt = dtype == USV_U8 ? 1 : 4;
    const size_t frame_bytes = (size_t)H * W * elt;
    cudaError_t e = cudaSuccess;
    if (convex)
        e = usv::launch_beam_setup(v.beams, W, cal->sector_deg, st);
    for (int c0 = 0; c0 < n && e == cudaSuccess; c0 += usv::kRecCap) {
        const int nc = n - c0 < usv::kRecCap ? n - c0 : usv::kRecCap;
        sp.first_rows = first_rows_dev ? first_rows_dev + c0 : nullptr;
        const double *pc = poses + (size_t)c0 * 16;
        if (poses_on_host) {
            const void *mapped = nullptr;
            e = v.ring->put(pc, (size_t)nc * 16 * sizeof(double), &mapped);
            if (e != cudaSuccess)
                break;
            pc = static_cast<const double *>(mapped);
        }
        e = usv::launch_frame_setup(pc, nc, sp, v.rec, v.status, st);
        if (e == cudaSuccess && poses_on_host)
            e = v.ring->fence(st);  // the set-up kernel is the region's only reader
        if (e != cudaSuccess)
            break;
        const char *img = static_cast<const char *>(images_dev) + (size_t)c0 * frame_bytes;
        if (v.mode == USV_PNN)
            e = usv::launch_insert_pnn(v, reinterpret_cast<const uint8_t *>(img), nc, H, W, st,
                                       cfg);
        else
            e = usv::launch_insert_trilinear(v, img, dtype == USV_F32, nc, H, W, sp.convex,
                                             cal->r0_mm, cal->dr_mm, st, cfg, tri_min_rows,
                                             tri_carry);
    }
    if (e == cudaErrorNotSupported)
        return USV_ERR_UNSUPPORTED;
    return usv::cuda_rc(e);
}

int usv_fill_holes(usv_volume *vol, int32_t radius, void *stream)
{
    if (!vol)
        return USV_ERR_ARG;
    const Volume &v = *reinterpret_cast<Volume *>(vol);
    const int32_t lo[3] = {0, 0, 0}, hi[3] = {v.g.nx, v.g.ny, v.g.nz};
    return usv_fill_holes_region(vol, lo, hi, radius, stream);
}

int usv_fill_holes_and_clear(usv_volume *vol, int32_t radius, void *stream)
{
    if (!vol)
        return USV_ERR_ARG;
    if (radius != 1)
        return USV_ERR_UNSUPPORTED;
    Volume &v = *reinterpret_cast<Volume *>(vol);
    if (v.mode != USV_PNN || !v.spare) {
        const int rc = usv_fill_holes(vol, radius, stream);
        return rc != USV_OK ? rc : usv_volume_reset(vol, stream);
    }
    const int lo[3] = {0, 0, 0}, hi[3] = {v.g.nx, v.g.ny, v.g.nz};
    usv::DeviceGuard g(v.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the fill reads every accumulator of `acc` and writes a zero into every
    // one of `spare`; later work on the stream sees the zeroed set
    const int rc = usv::cuda_rc(usv::launch_fill_pnn(v, lo, hi, st, v.spare));
    if (rc == USV_OK)
        std::swap(v.acc, v.spare);
    return rc;
}

int usv_fill_holes_region(usv_volume *vol, const int32_t lo[3], const int32_t hi[3],
                          int32_t radius, void *stream)
{
    if (!vol || !lo || !hi)
        return USV_ERR_ARG;
    if (radius != 1)
        return USV_ERR_UNSUPPORTED;
    Volume &v = *reinterpret_cast<Volume *>(vol);
    const int n[3] = {v.g.nx, v.g.ny, v.g.nz};
    int l[3], h[3];
    for (int a = 0; a < 3; ++a) {
        l[a] = lo[a] < 0 ? 0 : lo[a];
        h[a] = hi[a] > n[a] ? n[a] : hi[a];
        if (l[a] >= h[a])
            return USV_OK;  // empty region
    }
    l[0] &= ~31;  // mask words cover 32 columns
    usv::DeviceGuard g(v.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return usv::cuda_rc(v.mode == USV_PNN ? usv::launch_fill_pnn(v, l, h, st)
                                          : usv::launch_fill_trilinear(v, l, h, st));
}

int usv_project_depth_band(usv_volume *vol, int32_t z_lo, int32_t z_hi, float *out_dev,
                           uint16_t *count_dev, void *stream)
{
    if (!vol)
        return USV_ERR_ARG;
    const Volume &v = *reinterpret_cast<Volume *>(vol);
    const int32_t lo[2] = {0, 0}, hi[2] = {v.g.nx, v.g.ny};
    return usv_project_depth_band_region(vol, z_lo, z_hi, lo, hi, out_dev, count_dev, stream);
}

int usv_project_depth_band_region(usv_volume *vol, int32_t z_lo, int32_t z_hi,
                                  const int32_t xy_lo[2], const int32_t xy_hi[2], float *out_dev,
                                  uint16_t *count_dev, void *stream)
{
    if (!vol || !out_dev || !xy_lo || !xy_hi)
        return USV_ERR_ARG;
    Volume &v = *reinterpret_cast<Volume *>(vol);
    if (z_lo < 0 || z_hi > v.g.nz || z_lo >= z_hi)
        return USV_ERR_RANGE;
    if (z_hi - z_lo > 65535)
        return USV_ERR_RANGE;
    const int n[2] = {v.g.nx, v.g.ny};
    int l[2], h[2];
    for (int a = 0; a < 2; ++a) {
        l[a] = xy_lo[a] < 0 ? 0 : xy_lo[a];
        h[a] = xy_hi[a] > n[a] ? n[a] : xy_hi[a];
        if (l[a] >= h[a])
            return USV_OK;
    }
    usv::DeviceGuard g(v.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return usv::cuda_rc(v.mode == USV_PNN
                            ? usv::launch_project_u8(v, z_lo, z_hi, l, h, out_dev, count_dev, st)
                            : usv::launch_project_f32(v, z_lo, z_hi, l, h, out_dev, count_dev,
                                                      st));
}

int usv_volume_read(usv_volume *vol, int32_t what, void *dst_dev, void *stream)
{
    if (!vol || !dst_dev)
        return USV_ERR_ARG;
    Volume &v = *reinterpret_cast<Volume *>(vol);
    usv::DeviceGuard g(v.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)v.g.nx * v.g.ny * v.g.nz;
    switch (what) {
    case USV_READ_ACCUM:
        return usv::cuda_rc(cudaMemcpyAsync(dst_dev, v.acc, n * 8, cudaMemcpyDeviceToDevice, st));
    case USV_READ_VALUES:
        return usv::cuda_rc(cudaMemcpyAsync(dst_dev, v.val, n * (v.mode == USV_PNN ? 1 : 4),
                                            cudaMemcpyDeviceToDevice, st));
    case USV_READ_MASK:
        return usv::cuda_rc(usv::launch_unpack_mask(v, static_cast<uint8_t *>(dst_dev), st));
    default:
        return USV_ERR_ARG;
    }
}

int usv_volume_write_accum(usv_volume *vol, const void *src_dev, void *stream)
{
    if (!vol || !src_dev)
        return USV_ERR_ARG;
    Volume &v = *reinterpret_cast<Volume *>(vol);
    usv::DeviceGuard g(v.device);
    const size_t n = (size_t)v.g.nx * v.g.ny * v.g.nz;
    return usv::cuda_rc(cudaMemcpyAsync(v.acc, src_dev, n * 8, cudaMemcpyDeviceToDevice,
                                        static_cast<cudaStream_t>(stream)));
}

int usv_status(usv_volume *vol, void *stream)
{
    if (!vol)
        return USV_ERR_ARG;
    Volume &v = *reinterpret_cast<Volume *>(vol);
    usv::DeviceGuard g(v.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t bits = 0;
    int rc = usv::cuda_rc(cudaStreamSynchronize(st));
    if (rc == USV_OK)
        rc = usv::cuda_rc(cudaMemcpy(&bits, v.status, sizeof(bits), cudaMemcpyDeviceToHost));
    if (rc == USV_OK && bits != 0)
        rc = usv::cuda_rc(cudaMemset(v.status, 0, sizeof(bits)));
    if (rc != USV_OK)
        return rc;
    return (int)(bits & 0x7FFFFFFFu);
}

}  // extern "C"

// ---- tile shapes and the insertion autotuner ----

namespace usv {

TileCfg tile_for(const Volume &v, int H, int W)
{
    for (int i = 0; i < v.ntuned; ++i)
        if (v.tuned[i].H == H && v.tuned[i].W == W)
            return v.tuned[i].cfg;
    return v.mode == USV_PNN ? kPnnTileDefault : kTriTileDefault;
}

namespace {

int find_tuned(const Volume &v, int H, int W)
{
    for (int i = 0; i < v.ntuned; ++i)
        if (v.tuned[i].H == H && v.tuned[i].W == W)
            return i;
    return -1;
}

int store_tuned(Volume &v, int H, int W, const TileCfg &cfg)
{
    int i = find_tuned(v, H, W);
    if (i < 0) {
        if (v.ntuned == kTunedCap)
            return USV_ERR_RANGE;
        i = v.ntuned++;
    }
    v.tuned[i] = TunedTile{H, W, cfg};
    return USV_OK;
}

// The shapes the autotuner tries, in order (the default first).
int tune_candidates(int mode, TileCfg *out)
{
    int k = 0;
    if (mode == USV_PNN) {
        out[k++] = kPnnTileDefault;
        const int tw[3] = {64, 128, 256}, th[5] = {32, 48, 64, 96, 128}, fpc[4] = {4, 8, 12, 16};
        for (int a : tw)
            for (int b : th)
                for (int c : fpc) {
                    const TileCfg t{a, b, c};
                    if (pnn_tile_ok(t) &&
                        !(a == kPnnTileDefault.tile_w && b == kPnnTileDefault.tile_h &&
                          c == kPnnTileDefault.frames_per_cta))
                        out[k++] = t;
                }
    } else {
        out[k++] = kTriTileDefault;
        const int th[4] = {16, 32, 64, 128}, fpc[3] = {2, 4, 8};
        for (int b : th)
            for (int c : fpc) {
                const TileCfg t{256, b, c};
                if (!(b == kTriTileDefault.tile_h && c == kTriTileDefault.frames_per_cta))
                    out[k++] = t;
            }
    }
    return k;
}

}  // namespace

}  // namespace usv

int usv_set_tile_config(usv_volume *vol, int32_t H, int32_t W, const usv_tile_config *cfg)
{
    if (!vol || H < 1 || W < 1)
        return USV_ERR_ARG;
    Volume &v = *reinterpret_cast<Volume *>(vol);
    const int i = usv::find_tuned(v, H, W);
    if (!cfg) {
        if (i >= 0)
            v.tuned[i] = v.tuned[--v.ntuned];
        return USV_OK;
    }
    if (!(v.mode == USV_PNN ? usv::pnn_tile_ok(*cfg) : usv::tri_tile_ok(*cfg)))
        return USV_ERR_RANGE;
    return usv::store_tuned(v, H, W, *cfg);
}

int usv_get_tile_config(usv_volume *vol, int32_t H, int32_t W, usv_tile_config *out)
{
    if (!vol || !out || H < 1 || W < 1)
        return USV_ERR_ARG;
    *out = usv::tile_for(*reinterpret_cast<Volume *>(vol), H, W);
    return USV_OK;
}

int usv_tune_insert(usv_volume *vol, const void *images_dev, int32_t n, int32_t H, int32_t W,
                    int32_t dtype, const double *poses_dev, const usv_calibration *cal,
                    void *scratch_dev, size_t scratch_bytes, usv_tile_config *best_out,
                    float *best_ms_out, void *stream)
{
    if (!vol || !scratch_dev || n < 1 || (reinterpret_cast<uintptr_t>(scratch_dev) & 15) != 0)
        return USV_ERR_ARG;
    Volume &v = *reinterpret_cast<Volume *>(vol);
    const size_t acc_bytes = (size_t)v.g.nx * v.g.ny * v.g.nz * 8;
    if (scratch_bytes < acc_bytes)
        return USV_ERR_NOMEM;
    const int nt = n < 4096 ? n : 4096;
    usv::TileCfg cand[64];
    const int ncand = usv::tune_candidates(v.mode, cand);
    usv::DeviceGuard g(v.device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (int rc = usv::cuda_rc(cudaEventCreate(&e0)))
        return rc;
    if (int rc = usv::cuda_rc(cudaEventCreate(&e1))) {
        cudaEventDestroy(e0);
        return rc;
    }
    int rc = USV_OK;
    usv::TileCfg best = cand[0];
    float best_ms = 0.0f;
    bool have = false;
    for (int c = 0; c < ncand && rc == USV_OK; ++c) {
        float t[3];
        for (int rep = 0; rep < 4 && rc == USV_OK; ++rep) {  // rep 0 warms up
            rc = usv::cuda_rc(usv::launch_zero(scratch_dev, acc_bytes, v.num_sms, st));
            if (rc == USV_OK)
                rc = usv::cuda_rc(cudaEventRecord(e0, st));
            if (rc == USV_OK)
                rc = usv::insert_impl(vol, images_dev, nt, H, W, dtype, poses_dev, cal, nullptr,
                                      stream, scratch_dev, &cand[c]);
            if (rc == USV_OK)
                rc = usv::cuda_rc(cudaEventRecord(e1, st));
            if (rc == USV_OK)
                rc = usv::cuda_rc(cudaEventSynchronize(e1));
            float ms = 0.0f;
            if (rc == USV_OK)
                rc = usv::cuda_rc(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0)
                t[rep - 1] = ms;
        }
        if (rc != USV_OK)
            break;
        const float med = std::max(std::min(t[0], t[1]), std::min(std::max(t[0], t[1]), t[2]));
        if (!have || med < best_ms) {
            best = cand[c];
            best_ms = med;
            have = true;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != USV_OK)
        return rc;
    rc = usv::store_tuned(v, H, W, best);
    if (rc != USV_OK)
        return rc;
    if (best_out)
        *best_out = best;
    if (best_ms_out)
        *best_ms_out = best_ms;
    return USV_OK;
}

// ---- several (volume, frames) jobs in one launch pair ----

int usv_insert_frames_multi(const usv_insert_job *jobs, int32_t njobs, void *stream)
{
    if (njobs < 0 || (njobs > 0 && !jobs))
        return USV_ERR_ARG;
    if (njobs > usv::kMaxJobs)
        return USV_ERR_RANGE;
    usv::SetupJobs sj;
    usv::InsertJob ij[usv::kMaxJobs];
    const Volume *vols[usv::kMaxJobs];
    int m = 0, device = -1, num_sms = 0;
    sj.begin[0] = 0;
    for (int j = 0; j < njobs; ++j) {
        const usv_insert_job &b = jobs[j];
        if (!b.vol || !b.cal || b.n < 0)
            return USV_ERR_ARG;
        const Volume &v = *reinterpret_cast<const Volume *>(b.vol);
        for (int k = 0; k < m; ++k)
            if (vols[k] == &v)
                return USV_ERR_ARG;  // one job per volume (its set-up scratch)
        if (device >= 0 && v.device != device)
            return USV_ERR_ARG;
        if (v.mode != USV_PNN || b.dtype != USV_U8 || b.cal->geom != USV_LINEAR)
            return b.dtype != USV_U8 && b.dtype != USV_F32 ? USV_ERR_ARG : USV_ERR_UNSUPPORTED;
        if (b.n > usv::kRecCap)
            return USV_ERR_RANGE;
        if (b.n == 0)
            continue;
        if (!b.images_dev || !b.poses_dev || (reinterpret_cast<uintptr_t>(b.poses_dev) & 7) != 0)
            return USV_ERR_ARG;
        if (b.H < 1 || b.W < 1)
            return USV_ERR_ARG;
        if (b.H > usv::kMaxDim || b.W > usv::kMaxDim)
            return USV_ERR_RANGE;
        if (!usv::affine_ok(b.cal->image_to_probe))
            return USV_ERR_ARG;
        if (!(std::isfinite(b.cal->sx_mm) && std::isfinite(b.cal->sy_mm) && b.cal->sx_mm > 0.0 &&
              b.cal->sy_mm > 0.0))
            return USV_ERR_ARG;
        device = v.device;
        num_sms = v.num_sms;
        usv::SetupJob &s = sj.job[m];
        s.poses = b.poses_dev;
        std::memcpy(s.sp.K, b.cal->image_to_probe, sizeof(s.sp.K));
        for (int a = 0; a < 3; ++a) {
            s.sp.s[a] = v.spacing[a];
            s.sp.o[a] = v.origin[a];
        }
        s.sp.sx = b.cal->sx_mm;
        s.sp.sy = b.cal->sy_mm;
        s.sp.convex = 0;
        s.sp.first_rows = b.first_rows_dev;
        s.rec = v.rec;
        s.status = v.status;
        sj.begin[m + 1] = sj.begin[m] + b.n;
        usv::TileCfg cfg = usv::tile_for(v, b.H, b.W);
        if (cfg.tile_w != 128)
            cfg = usv::kPnnTileDefault;
        ij[m] = usv::InsertJob{&v, static_cast<const uint8_t *>(b.images_dev), b.n, b.H, b.W, cfg};
        vols[m++] = &v;
    }
    sj.njobs = m;
    if (m == 0)
        return USV_OK;
    usv::DeviceGuard g(device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = usv::launch_frame_setup_multi(sj, st);
    if (e == cudaSuccess)
        e = usv::launch_insert_pnn_multi(ij, m, num_sms, st);
    return usv::cuda_rc(e);
}

// ---- per-(kernel, device) launch preparation ----

cudaError_t usv::prepare_kernel(const void *func, int dyn_smem, int threads, int *blocks_per_sm)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> done;  // -> blocks per SM (0: not asked)
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(func, dev);
    auto it = done.find(key);
    if (it == done.end()) {
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem);
        if (e != cudaSuccess)
            return e;
        it = done.emplace(key, 0).first;
    }
    if (blocks_per_sm) {
        if (it->second == 0) {
            int b = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, func, threads, dyn_smem);
            if (e != cudaSuccess)
                return e;
            it->second = b < 1 ? 1 : b;
        }
        *blocks_per_sm = it->second;
    }
    return cudaSuccess;
}

// ---- test hook for the device-side failure path ----

int usv_test_fill_wait_timeout(usv_volume *vol, int32_t plane, void *stream)
{
    if (!vol)
        return USV_ERR_ARG;
    Volume &v = *reinterpret_cast<Volume *>(vol);
    if (plane < 0 || plane >= v.g.nz)
        return USV_ERR_ARG;
    if (v.mode != USV_PNN || v.g.nx % 2 != 0)
        return USV_ERR_UNSUPPORTED;
    const int lo[3] = {0, 0, 0}, hi[3] = {v.g.nx, v.g.ny, v.g.nz};
    usv::DeviceGuard g(v.device);
    const cudaError_t e =
        usv::launch_fill_pnn(v, lo, hi, static_cast<cudaStream_t>(stream), nullptr, plane);
    return e == cudaErrorNotSupported ? USV_ERR_UNSUPPORTED : usv::cuda_rc(e);
}

int usv_test_insert_trilinear_carry(usv_volume *vol, const void *images_dev, int32_t n,
                                    int32_t H, int32_t W, int32_t dtype, const double *poses_dev,
                                    const usv_calibration *cal, int32_t carry, void *stream)
{
    if (!vol)
        return USV_ERR_ARG;
    if (reinterpret_cast<Volume *>(vol)->mode != USV_TRILINEAR)
        return USV_ERR_UNSUPPORTED;
    return usv::insert_impl(vol, images_dev, n, H, W, dtype, poses_dev, cal, nullptr, stream,
                            nullptr, nullptr, 8, carry != 0);
}

int usv_probe_red_f2(void *buf_dev, size_t bytes, int32_t reds_per_thread, void *stream)
{
    if (!buf_dev || (reinterpret_cast<uintptr_t>(buf_dev) & 7) != 0 || bytes < sizeof(float2) ||
        reds_per_thread < 1)
        return USV_ERR_ARG;
    int dev = 0, sms = 0;
    if (int rc = usv::cuda_rc(cudaGetDevice(&dev)))
        return rc;
    if (int rc = usv::cuda_rc(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
        return rc;
    return usv::cuda_rc(usv::launch_red_f2_probe(buf_dev, bytes, reds_per_thread, sms,
                                                 static_cast<cudaStream_t>(stream)));
}
