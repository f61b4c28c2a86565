"""CPU oracle for the free-hand ultrasound volume path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and the ``--impl reference`` arm) may import this
package.  The product path (``paper_2412_00058_gb300``) never imports it and
shares no code with it; both sides only share the seeded input generators of
``paper_2412_00058_gb300.synth``, which hold none of the method's arithmetic.

The arithmetic lives in plain C (``usv_oracle.c``, FP64 / exact integers,
compiled with gcc ``-O2 -ffp-contract=off``); this module builds it on demand
and wraps it with numpy.  ``brute.py`` holds independent numpy restatements
used to pin the C code on tiny inputs.

Parity status: the nearest-neighbour path (insert, fill, project) and the
trilinear splat are pinned by the invariants in tests/test_oracle_pins.py;
the image-level output on the synthetic sweeps has no printed value in the
paper to pin against beyond those invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "usv_oracle.c")
_HDR = os.path.join(_HERE, "usv_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so (if stale), with
    OpenMP for its multi-core forms where the compiler has it (without it
    they run on one thread)."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        r = subprocess.run(["gcc", *CFLAGS, "-fopenmp", _SRC, "-o", tmp, "-lm"],
                           capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Geometry(ctypes.Structure):
    _fields_ = [("convex", ctypes.c_int), ("sx", ctypes.c_double), ("sy", ctypes.c_double),
                ("r0", ctypes.c_double), ("dr", ctypes.c_double),
                ("sector_deg", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.ora_set_threads.argtypes = [I]
            lib.ora_set_threads.restype = I
            lib.ora_insert_pnn_rows_mt.argtypes = [P, P, I, I, I, P, I, I, I, P, P, D, D, P, P, P]
            lib.ora_insert_pnn_rows_mt.restype = ctypes.c_int64
            lib.ora_round_half_away.argtypes = [D]
            lib.ora_round_half_away.restype = ctypes.c_int64
            lib.ora_frame_affine_q32.argtypes = [P, P, D, D, P, P, P]
            lib.ora_frame_affine_q32.restype = I
            lib.ora_insert_pnn.argtypes = [P, P, I, I, I, P, I, I, I, P, P, D, D, P, P]
            lib.ora_insert_pnn.restype = ctypes.c_int64
            lib.ora_fill_pnn.argtypes = [P, P, I, I, I, P, P]
            lib.ora_fill_pnn.restype = None
            lib.ora_project_u8.argtypes = [P, P, I, I, I, I, I, P, P]
            lib.ora_project_u8.restype = None
            lib.ora_insert_trilinear.argtypes = [P, P, I, I, I, P, I, I, I, I, P, P,
                                                 ctypes.POINTER(_Geometry), P, P]
            lib.ora_insert_trilinear.restype = ctypes.c_int64
            lib.ora_fill_trilinear.argtypes = [P, P, I, I, I, P, P]
            lib.ora_fill_trilinear.restype = None
            lib.ora_project_f64.argtypes = [P, P, I, I, I, I, I, P, P]
            lib.ora_project_f64.restype = None
            lib.ora_insert_pnn_rows.argtypes = [P, P, I, I, I, P, I, I, I, P, P, D, D, P, P, P]
            lib.ora_insert_pnn_rows.restype = ctypes.c_int64
            lib.ora_insert_trilinear_rows.argtypes = [P, P, I, I, I, P, I, I, I, I, P, P,
                                                      ctypes.POINTER(_Geometry), P, P, P]
            lib.ora_insert_trilinear_rows.restype = ctypes.c_int64
            lib.ora_cut_rows_alg1.argtypes = [P, I, I, P, D, D, D, P, P, D, P, P]
            lib.ora_cut_rows_alg1.restype = None
            lib.ora_bone_rows_alg2.argtypes = [P, I, I, I, I, I, I, I, P, P]
            lib.ora_bone_rows_alg2.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


_threads = 1


def set_threads(n: int) -> int:
    """Host threads for the nearest-neighbour insertion, fill and projection
    (1: the plain single-thread loops).  Returns the count in effect (1 if
    the oracle was built without OpenMP)."""
    global _threads
    _threads = int(_load().ora_set_threads(int(n)))
    return _threads


def round_half_away(x: float) -> int:
    return int(_load().ora_round_half_away(float(x)))


def frame_affine_q32(pose, calib, sx, sy, spacing, origin):
    """(coef int64[9] = A(3), B(3), C(3) in Q31.32, valid flag)."""
    out = np.zeros(9, dtype=np.int64)
    ok = _load().ora_frame_affine_q32(_ptr(_f64(pose, 16)), _ptr(_f64(calib, 16)), float(sx),
                                      float(sy), _ptr(_f64(spacing, 3)), _ptr(_f64(origin, 3)),
                                      _ptr(out))
    return out, bool(ok)


def insert_pnn(grid, images, poses, calib, sx, sy, spacing, origin, sum_=None, cnt=None,
               first_rows=None):
    """Nearest-neighbour insertion; returns (sum u64[nz,ny,nx], cnt u32[...],
    frames skipped).  Pass sum_/cnt to continue an existing scan;
    first_rows[f] cuts away the rows above it (depth of cut)."""
    nx, ny, nz = (int(g) for g in grid)
    images = np.ascontiguousarray(images, dtype=np.uint8)
    n, H, W = images.shape
    if sum_ is None:
        sum_ = np.zeros((nz, ny, nx), dtype=np.uint64)
        cnt = np.zeros((nz, ny, nx), dtype=np.uint32)
    poses = _f64(poses, (n, 16))
    fr = None if first_rows is None else np.ascontiguousarray(first_rows, dtype=np.int32)
    fn = _load().ora_insert_pnn_rows_mt if _threads > 1 else _load().ora_insert_pnn_rows
    sk = fn(_ptr(sum_), _ptr(cnt), nx, ny, nz, _ptr(images), n, H, W, _ptr(poses),
            _ptr(_f64(calib, 16)), float(sx), float(sy), _ptr(_f64(spacing, 3)),
            _ptr(_f64(origin, 3)), _ptr(fr) if fr is not None else None)
    return sum_, cnt, int(sk)


def fill_pnn(sum_, cnt):
    """(val u8, has u8) after normalisation and the 3x3x3 hole fill."""
    nz, ny, nx = sum_.shape
    val = np.empty((nz, ny, nx), dtype=np.uint8)
    has = np.empty((nz, ny, nx), dtype=np.uint8)
    _load().ora_fill_pnn(_ptr(sum_), _ptr(cnt), nx, ny, nz, _ptr(val), _ptr(has))
    return val, has


def project_u8(val, has, lo, hi):
    """(mean f32[ny,nx], count u16[ny,nx]) over the band z in [lo, hi)."""
    nz, ny, nx = val.shape
    out = np.empty((ny, nx), dtype=np.float32)
    c = np.empty((ny, nx), dtype=np.uint16)
    _load().ora_project_u8(_ptr(val), _ptr(has), nx, ny, nz, int(lo), int(hi), _ptr(out),
                           _ptr(c))
    return out, c


def _geometry(cal: dict) -> _Geometry:
    return _Geometry(1 if cal.get("geom", "linear") == "convex" else 0,
                     float(cal.get("sx", 0.0)), float(cal.get("sy", 0.0)),
                     float(cal.get("r0", 0.0)), float(cal.get("dr", 0.0)),
                     float(cal.get("sector_deg", 0.0)))


def insert_trilinear(grid, images, poses, cal: dict, spacing, origin, S=None, Wt=None,
                     first_rows=None):
    """Trilinear splat in FP64; returns (S, Wt, frames skipped).  ``cal`` is
    the dict of Workload.calibration()."""
    nx, ny, nz = (int(g) for g in grid)
    images = np.ascontiguousarray(images)
    is_f32 = images.dtype == np.float32
    if not is_f32:
        images = images.astype(np.uint8, copy=False)
    n, H, W = images.shape
    if S is None:
        S = np.zeros((nz, ny, nx), dtype=np.float64)
        Wt = np.zeros((nz, ny, nx), dtype=np.float64)
    g = _geometry(cal)
    fr = None if first_rows is None else np.ascontiguousarray(first_rows, dtype=np.int32)
    sk = _load().ora_insert_trilinear_rows(_ptr(S), _ptr(Wt), nx, ny, nz, _ptr(images),
                                           1 if is_f32 else 0, n, H, W,
                                           _ptr(_f64(poses, (n, 16))),
                                           _ptr(_f64(cal["image_to_probe"], 16)),
                                           ctypes.byref(g), _ptr(_f64(spacing, 3)),
                                           _ptr(_f64(origin, 3)),
                                           _ptr(fr) if fr is not None else None)
    return S, Wt, int(sk)


def fill_trilinear(S, Wt):
    nz, ny, nx = S.shape
    val = np.empty((nz, ny, nx), dtype=np.float64)
    has = np.empty((nz, ny, nx), dtype=np.uint8)
    _load().ora_fill_trilinear(_ptr(S), _ptr(Wt), nx, ny, nz, _ptr(val), _ptr(has))
    return val, has


def project_f64(val, has, lo, hi):
    nz, ny, nx = val.shape
    out = np.empty((ny, nx), dtype=np.float64)
    c = np.empty((ny, nx), dtype=np.uint16)
    _load().ora_project_f64(_ptr(val), _ptr(has), nx, ny, nz, int(lo), int(hi), _ptr(out),
                            _ptr(c))
    return out, c


def cut_rows_alg1(poses, H, calib, k, d_mm, l_mm, spine_dir, p1, row_mm):
    """Algorithm 1 depth of cut: (first rows int32[n], cut depth mm f64[n])."""
    poses = np.asarray(poses, np.float64)
    n = poses.shape[0]
    rows = np.empty(n, np.int32)
    cut = np.empty(n, np.float64)
    _load().ora_cut_rows_alg1(_ptr(_f64(poses, (n, 16))), n, int(H), _ptr(_f64(calib, 16)),
                              float(k), float(d_mm), float(l_mm), _ptr(_f64(spine_dir, 3)),
                              _ptr(_f64(p1, 3)), float(row_mm), _ptr(rows), _ptr(cut))
    return rows, cut


def bone_rows_alg2(images, from_row, drop, window, margin):
    """Algorithm 2: (per-frame bone row int32[n], first rows int32[n])."""
    images = np.ascontiguousarray(images, dtype=np.uint8)
    n, H, W = images.shape
    bone = np.empty(n, np.int32)
    rows = np.empty(n, np.int32)
    _load().ora_bone_rows_alg2(_ptr(images), n, H, W, int(from_row), int(drop), int(window),
                               int(margin), _ptr(bone), _ptr(rows))
    return bone, rows
