"""C-ABI checks that need no GPU: the library builds, exports every entry
point declared in include/*.h, and the Python binding's ctypes structures
have the C layout (checked against a gcc-compiled probe of the header)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2605_13855_gb300 import _lib
from paper_2605_13855_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    return pkg_build.build()


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(sparseoit_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_header_declares_the_binding_entry_points():
    declared = _declared_functions()
    assert declared, "no declarations found"
    assert declared == set(_lib.EXPORTED)


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sparseoit_\w+)", out))
    assert _declared_functions() <= exported


def test_version_without_gpu(libpath):
    lib = _lib.load(libpath)
    assert lib.sparseoit_version() == 1


PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "sparseoit.h"
#define F(T, m) printf(#T "." #m " %zu\n", offsetof(T, m));
int main(void) {
  printf("camera %zu\nsplats %zu\ngrads %zu\nconfig %zu\nktime %zu\n", sizeof(sparseoit_camera),
         sizeof(sparseoit_splats), sizeof(sparseoit_grads), sizeof(sparseoit_config), sizeof(sparseoit_kernel_time));
  printf("rows %zu\nadam %zu\n", sizeof(sparseoit_rows), sizeof(sparseoit_adam));
  F(sparseoit_camera, fx) F(sparseoit_camera, width) F(sparseoit_camera, height)
  F(sparseoit_splats, sh_color) F(sparseoit_splats, sh_dtype) F(sparseoit_splats, sigma) F(sparseoit_splats, bg)
  F(sparseoit_splats, n) F(sparseoit_splats, rows)
  F(sparseoit_grads, sigma) F(sparseoit_grads, rows_by_splat) F(sparseoit_grads, accumulate)
  F(sparseoit_config, max_pairs) F(sparseoit_config, fwd_pixels_per_thread)
  F(sparseoit_config, proj_lanes_per_splat) F(sparseoit_config, bwd_walk) F(sparseoit_config, raster_tile_order) F(sparseoit_config, bwd_parallel)
  F(sparseoit_config, raster_persistent)
  F(sparseoit_kernel_time, launches) F(sparseoit_kernel_time, total_ms)
  F(sparseoit_tuning, n_candidates) F(sparseoit_tuning, candidates) F(sparseoit_tuning, ms)
  F(sparseoit_tuning, fwd_persistent) F(sparseoit_tuning, fwd_persistent_ms) F(sparseoit_tuning, bwd_walk)
  F(sparseoit_tuning, bwd_persistent) F(sparseoit_tuning, bwd_ms)
  F(sparseoit_rows, sh_weight) F(sparseoit_rows, sigma)
  F(sparseoit_adam, beta1) F(sparseoit_adam, eps) F(sparseoit_adam, step) F(sparseoit_adam, rows)
  return 0;
}
"""


def test_ctypes_structs_match_header(tmp_path):
    src = tmp_path / "probe.c"
    src.write_text(PROBE)
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                              check=True).stdout.strip().splitlines())
    got = {k: int(v) for k, v in got.items()}
    assert got["camera"] == ctypes.sizeof(_lib.Camera)
    assert got["splats"] == ctypes.sizeof(_lib.Splats)
    assert got["grads"] == ctypes.sizeof(_lib.Grads)
    assert got["config"] == ctypes.sizeof(_lib.Config)
    assert got["ktime"] == ctypes.sizeof(_lib.KernelTime)
    assert got["rows"] == ctypes.sizeof(_lib.Rows)
    assert got["adam"] == ctypes.sizeof(_lib.Adam)
    pairs = {"sparseoit_camera": _lib.Camera, "sparseoit_splats": _lib.Splats, "sparseoit_grads": _lib.Grads,
             "sparseoit_config": _lib.Config, "sparseoit_kernel_time": _lib.KernelTime,
             "sparseoit_tuning": _lib.Tuning, "sparseoit_rows": _lib.Rows, "sparseoit_adam": _lib.Adam}
    for key, off in got.items():
        if "." not in key:
            continue
        t, m = key.split(".")
        assert getattr(pairs[t], m).offset == off, key


def test_binding_fails_loudly_without_library(tmp_path):
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved


def test_renderer_refuses_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2605_13855_gb300.renderer import Renderer
    with pytest.raises(RuntimeError, match="CUDA"):
        Renderer(16, [(16, 16)])
