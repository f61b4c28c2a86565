"""The library used from plain C (tests/c/usvol_c_example.c): the program
includes only usvol.h and the CUDA runtime, takes device memory from
cudaMalloc, passes the poses from host memory (the library stages them,
usv_insert_frames as the C ABI defines it), and its projection equals the
CPU oracle's bit for bit.  The header alone is also compiled as C99 on the
CPU."""
import os
import subprocess

import numpy as np
import pytest

from helpers import build_library, oracle_run

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "usvol_c_example.c")


def _compile(out_path):
    from paper_2412_00058_gb300 import build as B
    cuda_lib = B.cuda_lib_dir()
    cuda_inc = os.path.join(os.path.dirname(cuda_lib), "include")
    pkg = os.path.join(ROOT, "paper_2412_00058_gb300")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-O2", SRC,
           "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, "-L", pkg, "-lusvol",
           "-L", cuda_lib, "-lcudart", f"-Wl,-rpath,{pkg}", f"-Wl,-rpath,{cuda_lib}",
           "-o", out_path]
    subprocess.run(cmd, check=True, capture_output=True, text=True)


def test_header_compiles_as_c99(tmp_path):
    src = tmp_path / "h.c"
    src.write_text('#include "usvol.h"\nint main(void) { return usv_abi_version() == 2 ? 0 : 1; }\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-c",
                    str(src), "-I", os.path.join(ROOT, "include"), "-o",
                    str(tmp_path / "h.o")], check=True, capture_output=True, text=True)


@pytest.mark.gpu
def test_c_program_matches_the_oracle(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    build_library()
    from paper_2412_00058_gb300 import synth
    w = synth.whole_spine(n=21, grid=(270, 60, 200), y_start_mm=3.0, y_span_mm=8.0)
    n, H, W = w.images.shape
    nx, ny, nz = w.grid
    inp = tmp_path / "in.bin"
    with open(inp, "wb") as f:
        f.write(np.array([n, H, W, nx, ny, nz, w.band[0], w.band[1]], "<i4").tobytes())
        f.write(np.array(list(w.spacing) + list(w.origin) + [w.sx, w.sy], "<f8").tobytes())
        f.write(np.asarray(w.calib, "<f8").reshape(16).tobytes())
        f.write(np.ascontiguousarray(w.poses, "<f8").tobytes())
        f.write(np.ascontiguousarray(w.images, np.uint8).tobytes())
    exe = str(tmp_path / "usvol_c_example")
    _compile(exe)
    outp = tmp_path / "out.bin"
    r = subprocess.run([exe, str(inp), str(outp)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    raw = outp.read_bytes()
    proj = np.frombuffer(raw[:ny * nx * 4], "<f4").reshape(ny, nx)
    cnt = np.frombuffer(raw[ny * nx * 4:], "<u2").reshape(ny, nx)
    o = oracle_run(w)
    assert np.array_equal(proj, o["proj"]) and np.array_equal(cnt, o["pcnt"])
    assert cnt.sum() > 0
