"""Thin ctypes binding to libusvol.so (include/usvol.h).

Argument marshalling only: every step of the path runs in the library's
CUDA kernels.  PyTorch supplies device memory (the volume storage, frames,
poses, outputs) and the CUDA stream.  There is no CPU fallback: if the
library is missing this module raises.

The functions keep the C names without the ``usv_`` prefix
(``volume_bytes``, ``volume_create``, ``insert_frames``, ``fill_holes``,
``project_depth_band``, ``volume_read``, ``status``); ``Volume`` bundles
them with torch-owned storage.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
# USV_CHECKED=1 in the environment loads the bounds-checked build, in which
# every kernel write tests its index (an out-of-range one sets STATUS_OOB)
CHECKED = os.environ.get("USV_CHECKED", "") == "1"
LIB_PATH = os.path.join(_PKG, "libusvol_checked.so" if CHECKED else "libusvol.so")

OK, ERR_ARG, ERR_RANGE, ERR_CUDA, ERR_TIMEOUT, ERR_NOMEM, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
STATUS_BAD_POSE, STATUS_SATURATED, STATUS_TIMEOUT, STATUS_OOB = 0x1, 0x2, 0x4, 0x8
PNN, TRILINEAR = 0, 1
SPARE_ACCUM = 0x100
LINEAR, CONVEX = 0, 1
U8, F32 = 0, 1
READ_ACCUM, READ_VALUES, READ_MASK = 0, 1, 2

# every symbol declared in include/usvol.h
EXPORTS = ("usv_volume_bytes", "usv_volume_create", "usv_volume_destroy", "usv_volume_reset",
           "usv_insert_frames", "usv_fill_holes", "usv_project_depth_band", "usv_volume_read",
           "usv_volume_write_accum", "usv_status", "usv_strerror", "usv_last_cuda_error",
           "usv_abi_version", "usv_insert_pnn_noalloc", "usv_fill_holes_region",
           "usv_project_depth_band_region", "usv_insert_frames_cut", "usv_cut_rows_alg1",
           "usv_bone_rows_alg2", "usv_pose_loss_grad", "usv_apply_pose_delta",
           "usv_fill_holes_and_clear", "usv_tune_insert", "usv_set_tile_config",
           "usv_get_tile_config", "usv_insert_frames_multi", "usv_test_fill_wait_timeout",
           "usv_insert_frames_dev", "usv_frames_voxel_box", "usv_test_insert_trilinear_carry",
           "usv_probe_red_f2")


class UsvError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {strerror(code)} ({code})"
        if code == ERR_CUDA:
            msg += f": {lib().usv_last_cuda_error().decode()}"
        super().__init__(msg)


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class TileConfig(ctypes.Structure):
    """Insertion tile shape (usv_tile_config)."""
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("frames_per_cta", ctypes.c_int32)]

    def as_tuple(self):
        return (self.tile_w, self.tile_h, self.frames_per_cta)


class InsertJob(ctypes.Structure):
    """One (volume, batch of frames) job of usv_insert_frames_multi."""
    _fields_ = [("vol", ctypes.c_void_p), ("images_dev", ctypes.c_void_p),
                ("n", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("poses_dev", ctypes.c_void_p),
                ("cal", ctypes.c_void_p), ("first_rows_dev", ctypes.c_void_p)]


class Calibration(ctypes.Structure):
    _fields_ = [("image_to_probe", ctypes.c_double * 16), ("geom", ctypes.c_int32),
                ("sx_mm", ctypes.c_double), ("sy_mm", ctypes.c_double),
                ("r0_mm", ctypes.c_double), ("dr_mm", ctypes.c_double),
                ("sector_deg", ctypes.c_double)]


class Alg1Params(ctypes.Structure):
    """Algorithm 1 constants: Cut_n = K |P_c1.x - P_cn.x - L/2| + D."""
    _fields_ = [("K", ctypes.c_double), ("D_mm", ctypes.c_double), ("L_mm", ctypes.c_double),
                ("spine_dir", ctypes.c_double * 3), ("p1_mm", ctypes.c_double * 3)]


class Alg2Params(ctypes.Structure):
    """Algorithm 2 settings (bone contour search and temporal median)."""
    _fields_ = [("search_from_row", ctypes.c_int32), ("drop_rows", ctypes.c_int32),
                ("window", ctypes.c_int32), ("margin_rows", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libusvol.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            P, I, Z = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
            D3 = ctypes.POINTER(ctypes.c_double)
            L.usv_volume_bytes.argtypes = [Grid, I]
            L.usv_volume_bytes.restype = Z
            L.usv_volume_create.argtypes = [Grid, D3, D3, I, P, Z, ctypes.POINTER(P)]
            L.usv_volume_create.restype = ctypes.c_int
            L.usv_volume_destroy.argtypes = [P]
            L.usv_volume_destroy.restype = ctypes.c_int
            L.usv_volume_reset.argtypes = [P, P]
            L.usv_volume_reset.restype = ctypes.c_int
            L.usv_insert_frames.argtypes = [P, P, I, I, I, I, P, ctypes.POINTER(Calibration), P]
            L.usv_insert_frames.restype = ctypes.c_int
            L.usv_insert_frames_dev.argtypes = [P, P, I, I, I, I, P, ctypes.POINTER(Calibration),
                                                 P]
            L.usv_insert_frames_dev.restype = ctypes.c_int
            I3o = ctypes.POINTER(ctypes.c_int32)
            L.usv_frames_voxel_box.argtypes = [Grid, D3, D3, P, I, I, I,
                                               ctypes.POINTER(Calibration), I, I3o, I3o]
            L.usv_frames_voxel_box.restype = ctypes.c_int
            L.usv_test_insert_trilinear_carry.argtypes = [P, P, I, I, I, I, P,
                                                          ctypes.POINTER(Calibration), I, P]
            L.usv_test_insert_trilinear_carry.restype = ctypes.c_int
            L.usv_probe_red_f2.argtypes = [P, Z, I, P]
            L.usv_probe_red_f2.restype = ctypes.c_int
            L.usv_fill_holes.argtypes = [P, I, P]
            L.usv_fill_holes.restype = ctypes.c_int
            L.usv_project_depth_band.argtypes = [P, I, I, P, P, P]
            L.usv_project_depth_band.restype = ctypes.c_int
            I3 = ctypes.POINTER(ctypes.c_int32)
            L.usv_fill_holes_region.argtypes = [P, I3, I3, I, P]
            L.usv_fill_holes_region.restype = ctypes.c_int
            L.usv_project_depth_band_region.argtypes = [P, I, I, I3, I3, P, P, P]
            L.usv_project_depth_band_region.restype = ctypes.c_int
            L.usv_volume_read.argtypes = [P, I, P, P]
            L.usv_volume_read.restype = ctypes.c_int
            L.usv_volume_write_accum.argtypes = [P, P, P]
            L.usv_volume_write_accum.restype = ctypes.c_int
            L.usv_status.argtypes = [P, P]
            L.usv_status.restype = ctypes.c_int
            L.usv_strerror.argtypes = [ctypes.c_int]
            L.usv_strerror.restype = ctypes.c_char_p
            L.usv_insert_frames_cut.argtypes = [P, P, I, I, I, I, P,
                                                ctypes.POINTER(Calibration), P, P]
            L.usv_insert_frames_cut.restype = ctypes.c_int
            L.usv_cut_rows_alg1.argtypes = [P, I, I, ctypes.POINTER(Calibration),
                                            ctypes.POINTER(Alg1Params), P, P]
            L.usv_cut_rows_alg1.restype = ctypes.c_int
            L.usv_bone_rows_alg2.argtypes = [P, I, I, I, ctypes.POINTER(Alg2Params), P, P, P]
            L.usv_bone_rows_alg2.restype = ctypes.c_int
            L.usv_pose_loss_grad.argtypes = [P, P, I, I, I, I, P, ctypes.POINTER(Calibration), I,
                                             I, ctypes.c_float, P, P, P, P, P, P]
            L.usv_pose_loss_grad.restype = ctypes.c_int
            L.usv_apply_pose_delta.argtypes = [P, P, I, I, I, ctypes.POINTER(Calibration), P, P]
            L.usv_apply_pose_delta.restype = ctypes.c_int
            L.usv_last_cuda_error.argtypes = []
            L.usv_last_cuda_error.restype = ctypes.c_char_p
            L.usv_abi_version.argtypes = []
            L.usv_abi_version.restype = ctypes.c_int
            _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().usv_strerror(int(code)).decode()


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise UsvError(rc, what)
    return rc


def _d3(v) -> ctypes.Array:
    return (ctypes.c_double * 3)(*[float(x) for x in v])


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def make_calibration(image_to_probe, geom="linear", sx=0.0, sy=0.0, r0=0.0, dr=0.0,
                     sector_deg=0.0) -> Calibration:
    m = np.ascontiguousarray(np.asarray(image_to_probe, dtype=np.float64).reshape(16))
    return Calibration((ctypes.c_double * 16)(*m.tolist()), CONVEX if geom == "convex" else LINEAR,
                       float(sx), float(sy), float(r0), float(dr), float(sector_deg))


def _mode(mode) -> int:
    return {"pnn": PNN, "trilinear": TRILINEAR}.get(mode, mode)


# ---------------------------------------------------------------- C-named calls

def volume_bytes(grid, mode) -> int:
    return int(lib().usv_volume_bytes(Grid(*grid), _mode(mode)))


def volume_create(grid, spacing, origin, mode, storage_ptr: int, storage_bytes: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().usv_volume_create(Grid(*grid), _d3(spacing), _d3(origin), _mode(mode),
                                   ctypes.c_void_p(storage_ptr), storage_bytes, ctypes.byref(h)),
           "usv_volume_create")
    return h.value


def volume_destroy(handle: int) -> None:
    _check(lib().usv_volume_destroy(ctypes.c_void_p(handle)), "usv_volume_destroy")


def volume_reset(handle: int, stream=None) -> None:
    _check(lib().usv_volume_reset(ctypes.c_void_p(handle), ctypes.c_void_p(_stream_ptr(stream))),
           "usv_volume_reset")


def insert_frames(handle: int, images_ptr: int, n: int, H: int, W: int, dtype: int,
                  poses_host_ptr: int, cal: Calibration, stream=None) -> None:
    """Poses in host memory (staged by the library)."""
    _check(lib().usv_insert_frames(ctypes.c_void_p(handle), ctypes.c_void_p(images_ptr), n, H, W,
                                   dtype, ctypes.c_void_p(poses_host_ptr), ctypes.byref(cal),
                                   ctypes.c_void_p(_stream_ptr(stream))), "usv_insert_frames")


def insert_frames_dev(handle: int, images_ptr: int, n: int, H: int, W: int, dtype: int,
                      poses_dev_ptr: int, cal: Calibration, stream=None) -> None:
    """Poses in device memory."""
    _check(lib().usv_insert_frames_dev(ctypes.c_void_p(handle), ctypes.c_void_p(images_ptr), n, H,
                                       W, dtype, ctypes.c_void_p(poses_dev_ptr),
                                       ctypes.byref(cal), ctypes.c_void_p(_stream_ptr(stream))),
           "usv_insert_frames_dev")


def frames_voxel_box(grid, spacing, origin, poses_host_ptr: int, n: int, H: int, W: int,
                     cal: Calibration, margin: int = 0):
    """(lo, hi): the half-open voxel box the frames can write, widened by margin."""
    lo = (ctypes.c_int32 * 3)()
    hi = (ctypes.c_int32 * 3)()
    _check(lib().usv_frames_voxel_box(Grid(*grid), _d3(spacing), _d3(origin),
                                      ctypes.c_void_p(poses_host_ptr), n, H, W, ctypes.byref(cal),
                                      int(margin), lo, hi), "usv_frames_voxel_box")
    return tuple(lo), tuple(hi)


def insert_trilinear_carry(handle: int, images_ptr: int, n: int, H: int, W: int, dtype: int,
                           poses_dev_ptr: int, cal: Calibration, carry: bool,
                           stream=None) -> None:
    """Test hook: trilinear insertion with the corner carry on or off."""
    _check(lib().usv_test_insert_trilinear_carry(ctypes.c_void_p(handle),
                                                 ctypes.c_void_p(images_ptr), n, H, W, dtype,
                                                 ctypes.c_void_p(poses_dev_ptr), ctypes.byref(cal),
                                                 1 if carry else 0,
                                                 ctypes.c_void_p(_stream_ptr(stream))),
           "usv_test_insert_trilinear_carry")


def insert_frames_cut(handle: int, images_ptr: int, n: int, H: int, W: int, dtype: int,
                      poses_ptr: int, cal: Calibration, first_rows_ptr: int, stream=None) -> None:
    _check(lib().usv_insert_frames_cut(ctypes.c_void_p(handle), ctypes.c_void_p(images_ptr), n, H,
                                       W, dtype, ctypes.c_void_p(poses_ptr), ctypes.byref(cal),
                                       ctypes.c_void_p(first_rows_ptr),
                                       ctypes.c_void_p(_stream_ptr(stream))),
           "usv_insert_frames_cut")


def cut_rows_alg1(poses_ptr: int, n: int, H: int, cal: Calibration, prm: Alg1Params,
                  first_rows_ptr: int, stream=None) -> None:
    _check(lib().usv_cut_rows_alg1(ctypes.c_void_p(poses_ptr), n, H, ctypes.byref(cal),
                                   ctypes.byref(prm), ctypes.c_void_p(first_rows_ptr),
                                   ctypes.c_void_p(_stream_ptr(stream))), "usv_cut_rows_alg1")


def bone_rows_alg2(images_ptr: int, n: int, H: int, W: int, prm: Alg2Params, bone_rows_ptr: int,
                   first_rows_ptr: int, stream=None) -> None:
    _check(lib().usv_bone_rows_alg2(ctypes.c_void_p(images_ptr), n, H, W, ctypes.byref(prm),
                                    ctypes.c_void_p(bone_rows_ptr),
                                    ctypes.c_void_p(first_rows_ptr),
                                    ctypes.c_void_p(_stream_ptr(stream))), "usv_bone_rows_alg2")


def pose_loss_grad(handle: int, images_ptr: int, n: int, H: int, W: int, dtype: int,
                   poses_ptr: int, cal: Calibration, z_lo: int, z_hi: int, eps: float,
                   target_ptr: int, proj_ptr: int, adj_ptr: int, loss_ptr: int, grad_ptr: int,
                   stream=None) -> None:
    _check(lib().usv_pose_loss_grad(ctypes.c_void_p(handle), ctypes.c_void_p(images_ptr), n, H, W,
                                    dtype, ctypes.c_void_p(poses_ptr), ctypes.byref(cal), z_lo,
                                    z_hi, float(eps), ctypes.c_void_p(target_ptr),
                                    ctypes.c_void_p(proj_ptr), ctypes.c_void_p(adj_ptr),
                                    ctypes.c_void_p(loss_ptr), ctypes.c_void_p(grad_ptr),
                                    ctypes.c_void_p(_stream_ptr(stream))), "usv_pose_loss_grad")


def apply_pose_delta(poses_ptr: int, delta_ptr: int, n: int, H: int, W: int, cal: Calibration,
                     out_ptr: int, stream=None) -> None:
    _check(lib().usv_apply_pose_delta(ctypes.c_void_p(poses_ptr), ctypes.c_void_p(delta_ptr), n, H,
                                      W, ctypes.byref(cal), ctypes.c_void_p(out_ptr),
                                      ctypes.c_void_p(_stream_ptr(stream))),
           "usv_apply_pose_delta")


def probe_red_f2(buf_ptr: int, nbytes: int, reds_per_thread: int, stream=None) -> None:
    """Measurement utility: the float2 vector-atomic rate probe."""
    _check(lib().usv_probe_red_f2(ctypes.c_void_p(buf_ptr), ctypes.c_size_t(nbytes),
                                  int(reds_per_thread), ctypes.c_void_p(_stream_ptr(stream))),
           "usv_probe_red_f2")


def fill_holes(handle: int, radius: int = 1, stream=None) -> None:
    _check(lib().usv_fill_holes(ctypes.c_void_p(handle), radius,
                                ctypes.c_void_p(_stream_ptr(stream))), "usv_fill_holes")


def insert_frames_multi(jobs, stream=None) -> None:
    """jobs: sequence of (Volume, images [n,H,W] u8, poses [n,4,4] f64, Calibration)
    or (..., first_rows [n] int32 on the device) for tissue-segmented frames."""
    arr = (InsertJob * max(len(jobs), 1))()
    keep = []
    for k, job in enumerate(jobs):
        vol, images, poses, cal = job[:4]
        rows = job[4] if len(job) > 4 else None
        assert images.is_cuda and poses.is_cuda and images.is_contiguous() and poses.is_contiguous()
        if rows is not None:
            assert rows.is_cuda and rows.dtype == torch.int32 and rows.is_contiguous()
        n, H, W = images.shape
        keep.append(cal)
        arr[k] = InsertJob(vol.handle, images.data_ptr(), n, H, W, U8, poses.data_ptr(),
                           ctypes.cast(ctypes.pointer(cal), ctypes.c_void_p),
                           rows.data_ptr() if rows is not None else None)
    _check(lib().usv_insert_frames_multi(arr, len(jobs), ctypes.c_void_p(_stream_ptr(stream))),
           "usv_insert_frames_multi")


def tune_insert(handle: int, images_ptr: int, n: int, H: int, W: int, dtype: int,
                poses_ptr: int, cal: Calibration, scratch_ptr: int, scratch_bytes: int,
                stream=None):
    """Run the insertion autotuner; returns (TileConfig, ms)."""
    best = TileConfig()
    ms = ctypes.c_float()
    _check(lib().usv_tune_insert(ctypes.c_void_p(handle), ctypes.c_void_p(images_ptr), n, H, W,
                                 dtype, ctypes.c_void_p(poses_ptr), ctypes.byref(cal),
                                 ctypes.c_void_p(scratch_ptr), ctypes.c_size_t(scratch_bytes),
                                 ctypes.byref(best), ctypes.byref(ms),
                                 ctypes.c_void_p(_stream_ptr(stream))), "usv_tune_insert")
    return best, ms.value


def set_tile_config(handle: int, H: int, W: int, cfg) -> None:
    c = None if cfg is None else TileConfig(*cfg)
    _check(lib().usv_set_tile_config(ctypes.c_void_p(handle), H, W,
                                     ctypes.byref(c) if c is not None else None),
           "usv_set_tile_config")


def get_tile_config(handle: int, H: int, W: int) -> tuple:
    out = TileConfig()
    _check(lib().usv_get_tile_config(ctypes.c_void_p(handle), H, W, ctypes.byref(out)),
           "usv_get_tile_config")
    return out.as_tuple()


def fill_with_withheld_copy(handle: int, plane: int, stream=None) -> None:
    """Test hook: the fill with one plane copy withheld (its wait runs out)."""
    _check(lib().usv_test_fill_wait_timeout(ctypes.c_void_p(handle), plane,
                                            ctypes.c_void_p(_stream_ptr(stream))),
           "usv_test_fill_wait_timeout")


def fill_holes_and_clear(handle: int, radius: int = 1, stream=None) -> None:
    _check(lib().usv_fill_holes_and_clear(ctypes.c_void_p(handle), radius,
                                          ctypes.c_void_p(_stream_ptr(stream))),
           "usv_fill_holes_and_clear")


def project_depth_band(handle: int, z_lo: int, z_hi: int, out_ptr: int, count_ptr: int | None,
                       stream=None) -> None:
    _check(lib().usv_project_depth_band(ctypes.c_void_p(handle), z_lo, z_hi,
                                        ctypes.c_void_p(out_ptr), ctypes.c_void_p(count_ptr or 0),
                                        ctypes.c_void_p(_stream_ptr(stream))),
           "usv_project_depth_band")


def _i32(v) -> ctypes.Array:
    return (ctypes.c_int32 * len(v))(*[int(x) for x in v])


def fill_holes_region(handle: int, lo, hi, radius: int = 1, stream=None) -> None:
    _check(lib().usv_fill_holes_region(ctypes.c_void_p(handle), _i32(lo), _i32(hi), radius,
                                       ctypes.c_void_p(_stream_ptr(stream))),
           "usv_fill_holes_region")


def project_depth_band_region(handle: int, z_lo: int, z_hi: int, xy_lo, xy_hi, out_ptr: int,
                              count_ptr: int | None, stream=None) -> None:
    _check(lib().usv_project_depth_band_region(ctypes.c_void_p(handle), z_lo, z_hi, _i32(xy_lo),
                                               _i32(xy_hi), ctypes.c_void_p(out_ptr),
                                               ctypes.c_void_p(count_ptr or 0),
                                               ctypes.c_void_p(_stream_ptr(stream))),
           "usv_project_depth_band_region")


def volume_read(handle: int, what: int, dst_ptr: int, stream=None) -> None:
    _check(lib().usv_volume_read(ctypes.c_void_p(handle), what, ctypes.c_void_p(dst_ptr),
                                 ctypes.c_void_p(_stream_ptr(stream))), "usv_volume_read")


def volume_write_accum(handle: int, src_ptr: int, stream=None) -> None:
    _check(lib().usv_volume_write_accum(ctypes.c_void_p(handle), ctypes.c_void_p(src_ptr),
                                        ctypes.c_void_p(_stream_ptr(stream))),
           "usv_volume_write_accum")


def status(handle: int, stream=None) -> int:
    bits = _check(lib().usv_status(ctypes.c_void_p(handle), ctypes.c_void_p(_stream_ptr(stream))),
                  "usv_status")
    if bits & STATUS_OOB:
        raise RuntimeError("the checked build caught a kernel write outside its buffer "
                           f"(status {bits:#x})")
    return bits


# ---------------------------------------------------------------- convenience

class Volume:
    """A reconstruction volume in torch-owned device storage."""

    def __init__(self, grid, spacing, origin=(0.0, 0.0, 0.0), mode="pnn", device="cuda",
                 spare=False):
        """spare=True adds a second accumulator set (USV_SPARE_ACCUM), so that
        fill_and_clear() clears the accumulators inside the fill pass."""
        self.grid = tuple(int(g) for g in grid)
        self.mode = _mode(mode)
        self.spacing = tuple(float(s) for s in spacing)
        self.origin = tuple(float(o) for o in origin)
        flags = self.mode | (SPARE_ACCUM if spare else 0)
        nbytes = volume_bytes(self.grid, flags)
        if nbytes == 0:
            raise UsvError(ERR_ARG, f"invalid grid {self.grid}")
        self.storage = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.handle = volume_create(self.grid, self.spacing, self.origin, flags,
                                    self.storage.data_ptr(), nbytes)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                volume_destroy(h)
            except Exception:
                pass
            self.handle = None

    @property
    def shape(self):
        nx, ny, nz = self.grid
        return (nz, ny, nx)

    def reset(self, stream=None):
        volume_reset(self.handle, stream)

    def insert(self, images: torch.Tensor, poses, cal: Calibration, stream=None):
        """Insert frames (device tensor [n, H, W]); poses [n, 4, 4] float64 on
        the device (usv_insert_frames_dev) or on the host -- a CPU tensor or
        a numpy array -- (usv_insert_frames, staged by the library)."""
        assert images.is_cuda and images.is_contiguous()
        n, H, W = images.shape
        dt = U8 if images.dtype == torch.uint8 else F32
        if dt == F32:
            assert images.dtype == torch.float32
        if isinstance(poses, np.ndarray):
            poses = torch.from_numpy(np.ascontiguousarray(poses, dtype=np.float64))
        assert poses.dtype == torch.float64 and poses.is_contiguous()
        if poses.is_cuda:
            insert_frames_dev(self.handle, images.data_ptr(), n, H, W, dt, poses.data_ptr(), cal,
                              stream)
        else:
            insert_frames(self.handle, images.data_ptr(), n, H, W, dt, poses.data_ptr(), cal,
                          stream)

    def voxel_box(self, poses, H: int, W: int, cal: Calibration, margin: int = 0):
        """usv_frames_voxel_box for host poses [n, 4, 4] (numpy or CPU tensor)."""
        p = np.ascontiguousarray(poses.numpy() if isinstance(poses, torch.Tensor) else poses,
                                 dtype=np.float64)
        return frames_voxel_box(self.grid, self.spacing, self.origin, p.ctypes.data, p.shape[0],
                                H, W, cal, margin)

    def tune(self, images: torch.Tensor, poses: torch.Tensor, cal: Calibration, stream=None):
        """Autotune the insertion tile shape for these frames (scratch
        accumulators from torch); the choice is kept for their frame size.
        Returns ((tile_w, tile_h, frames_per_cta), ms)."""
        n, H, W = images.shape
        dt = U8 if images.dtype == torch.uint8 else F32
        nx, ny, nz = self.grid
        scratch = torch.empty(nx * ny * nz, dtype=torch.int64, device=self.storage.device)
        best, ms = tune_insert(self.handle, images.data_ptr(), n, H, W, dt, poses.data_ptr(), cal,
                               scratch.data_ptr(), scratch.numel() * 8, stream)
        return best.as_tuple(), ms

    def set_tile(self, H: int, W: int, cfg) -> None:
        set_tile_config(self.handle, H, W, cfg)

    def get_tile(self, H: int, W: int) -> tuple:
        return get_tile_config(self.handle, H, W)

    def fill(self, stream=None):
        fill_holes(self.handle, 1, stream)

    def fill_and_clear(self, stream=None):
        """fill(), then the accumulators read as zero (end of a sweep)."""
        fill_holes_and_clear(self.handle, 1, stream)

    def project(self, z_lo, z_hi, out=None, count=None, stream=None):
        nz, ny, nx = self.shape
        dev = self.storage.device
        if out is None:
            out = torch.empty((ny, nx), dtype=torch.float32, device=dev)
        if count is None:
            count = torch.empty((ny, nx), dtype=torch.int16, device=dev)
        project_depth_band(self.handle, z_lo, z_hi, out.data_ptr(),
                           count.data_ptr() if count is not False else None, stream)
        return out, count

    def read(self, what, stream=None) -> torch.Tensor:
        dev = self.storage.device
        if what == READ_ACCUM:
            dst = torch.empty(self.shape + ((2,) if self.mode == TRILINEAR else ()),
                              dtype=torch.float32 if self.mode == TRILINEAR else torch.int64,
                              device=dev)
        elif what == READ_VALUES:
            dst = torch.empty(self.shape, dtype=torch.uint8 if self.mode == PNN else torch.float32,
                              device=dev)
        else:
            dst = torch.empty(self.shape, dtype=torch.uint8, device=dev)
        volume_read(self.handle, what, dst.data_ptr(), stream)
        return dst

    def status(self, stream=None) -> int:
        return status(self.handle, stream)

    def save(self, path, stream=None) -> None:
        """Write the accumulators (the raw integer sum/count pairs of PNN, the
        FP32 (S, W) pairs of trilinear) and the geometry to `path`, so that a
        scan can be resumed bit-exactly with Volume.load (the paper stores
        its volume at the end of a scan, Sec. II.C)."""
        acc = self.read(READ_ACCUM, stream).cpu().numpy()
        write_volume_file(path, dict(grid=list(self.grid), spacing=list(self.spacing),
                                     origin=list(self.origin), mode=_MODE_NAMES[self.mode]), acc)

    @classmethod
    def load(cls, path, device="cuda", spare=False, stream=None) -> "Volume":
        """A volume with the geometry and accumulators saved by Volume.save;
        its filled values are not restored (run fill() again)."""
        meta, acc = read_volume_file(path)
        vol = cls(meta["grid"], meta["spacing"], meta["origin"], meta["mode"], device=device,
                  spare=spare)
        src = torch.from_numpy(acc).to(vol.storage.device)
        volume_write_accum(vol.handle, src.data_ptr(), stream)
        # the host copy must stay alive until the stream-ordered write is done
        (torch.cuda.current_stream(vol.storage.device) if stream is None else stream).synchronize()
        return vol

    def save_slices(self, directory, stream=None) -> list:
        """Write the filled volume as one 8-bit greyscale image per slice along
        the spine axis (y), depth down and lateral across, as binary PGM files
        (the paper's end-of-scan output, Sec. II.C).  Trilinear values are
        rounded and clamped to [0, 255].  Returns the file names."""
        vals = self.read(READ_VALUES, stream).cpu().numpy()          # [nz, ny, nx]
        if vals.dtype != np.uint8:
            vals = np.clip(np.rint(vals), 0, 255).astype(np.uint8)
        os.makedirs(directory, exist_ok=True)
        nz, ny, nx = vals.shape
        names = []
        for y in range(ny):
            name = os.path.join(directory, f"slice_{y:05d}.pgm")
            with open(name, "wb") as f:
                f.write(b"P5\n%d %d\n255\n" % (nx, nz))
                f.write(np.ascontiguousarray(vals[:, y, :]).tobytes())
            names.append(name)
        return names


_MODE_NAMES = {PNN: "pnn", TRILINEAR: "trilinear"}
_FILE_MAGIC = b"USVOLACC"


def write_volume_file(path, meta: dict, acc: np.ndarray) -> None:
    """The saved-volume format: 8 magic bytes, a 4-byte little-endian header
    length, a UTF-8 JSON header (geometry, mode, dtype, shape) and the raw
    accumulator array in C order."""
    import json
    head = dict(meta, dtype=str(acc.dtype), shape=list(acc.shape), version=1)
    hb = json.dumps(head, sort_keys=True).encode()
    with open(path, "wb") as f:
        f.write(_FILE_MAGIC)
        f.write(len(hb).to_bytes(4, "little"))
        f.write(hb)
        f.write(np.ascontiguousarray(acc).tobytes())


def read_volume_file(path):
    """(header dict, accumulator array) of a file written by write_volume_file;
    raises ValueError on a foreign, truncated or inconsistent file."""
    import json
    with open(path, "rb") as f:
        if f.read(8) != _FILE_MAGIC:
            raise ValueError(f"{path}: not a saved volume")
        n = int.from_bytes(f.read(4), "little")
        head = json.loads(f.read(n).decode())
        data = f.read()
    if head.get("version") != 1 or head.get("mode") not in ("pnn", "trilinear"):
        raise ValueError(f"{path}: unsupported header {head}")
    nx, ny, nz = head["grid"]
    want = [nz, ny, nx] + ([2] if head["mode"] == "trilinear" else [])
    dt = np.dtype(head["dtype"])
    if head["shape"] != want or dt != (np.int64 if head["mode"] == "pnn" else np.float32):
        raise ValueError(f"{path}: accumulator shape/dtype do not match the grid")
    if len(data) != int(np.prod(want)) * dt.itemsize:
        raise ValueError(f"{path}: truncated accumulators")
    return head, np.frombuffer(data, dtype=dt).reshape(want).copy()


def calibration_of(w) -> Calibration:
    """Calibration struct for a synth.Workload (or any object with the same fields)."""
    return make_calibration(w.calib, w.geom, w.sx, w.sy, w.r0, w.dr, w.sector_deg)
