"""Host-side checks of the C ABI that need no GPU: the library builds and loads, exports every
function the header declares, the Python struct matches the C struct, and invalid arguments
are rejected on the host with LBMHD_ERR_INVALID before any CUDA call."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1705_09807_gb300 import build as libbuild
from paper_1705_09807_gb300 import lbmhd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return lbmhd.load_library()


def test_exports_every_header_function(lib):
    names = lbmhd.header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_params_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "lbmhd.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(lbmhd_params),"
        " offsetof(lbmhd_params, s), offsetof(lbmhd_params, s_m), offsetof(lbmhd_params, delta),"
        " offsetof(lbmhd_params, precision), offsetof(lbmhd_params, grad_stencil),"
        " offsetof(lbmhd_params, cuda_stream));return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    P = lbmhd.LbmhdParams
    want = [ctypes.sizeof(P), P.s.offset, P.s_m.offset, P.delta.offset, P.precision.offset,
            P.grad_stencil.offset, P.cuda_stream.offset]
    assert got == want


def test_params_srt_maps_viscosity_to_rates(lib):
    p = lbmhd.lbmhd_params_srt(64, 32, 0.002, 0.004, 2.0, lbmhd.LBMHD_FP32)
    assert (p.nx, p.ny, p.precision, p.grad_stencil) == (64, 32, 1, 0)
    s = 1 / (3 * 0.002 + 0.5)
    assert all(abs(p.s[j] - s) < 1e-15 for j in range(9))
    assert abs(p.s_m - 1 / (3 * 0.004 + 0.5)) < 1e-15
    assert p.delta == 2.0 and p.cuda_stream is None
    with pytest.raises(lbmhd.LbmhdError) as e:
        lbmhd.lbmhd_params_srt(8, 8, -1.0, 0.1, 0.0)
    assert e.value.code == lbmhd.LBMHD_ERR_INVALID


def _fields(nx, ny):
    z = np.zeros((ny, nx))
    return (1 + z, z, z, z, z)


@pytest.mark.parametrize("mutate,needle", [
    (lambda p: setattr(p, "nx", 2), "grid"),
    (lambda p: setattr(p, "ny", 0), "grid"),
    (lambda p: (setattr(p, "nx", 2**30), setattr(p, "ny", 3)), "2^31 cells"),
    (lambda p: (setattr(p, "nx", 79_536_383), setattr(p, "ny", 3)), "width"),
    (lambda p: p.s.__setitem__(4, 2.0), "s[4]"),
    (lambda p: p.s.__setitem__(7, 0.0), "s[7]"),
    (lambda p: setattr(p, "s_m", -0.5), "s_m"),
    (lambda p: setattr(p, "delta", -1.0), "delta"),
    (lambda p: setattr(p, "delta", float("nan")), "delta"),
    (lambda p: setattr(p, "precision", 7), "precision"),
    (lambda p: setattr(p, "grad_stencil", 3), "grad_stencil"),
])
def test_invalid_params_rejected_on_host(lib, mutate, needle):
    p = lbmhd.lbmhd_params_srt(8, 8, 0.01, 0.01, 1.0)
    mutate(p)
    h = ctypes.c_void_p()
    arrs = [np.ascontiguousarray(a) for a in _fields(8, 8)]
    D = ctypes.POINTER(ctypes.c_double)
    rc = lib.lbmhd_init(ctypes.byref(h), ctypes.byref(p), *(a.ctypes.data_as(D) for a in arrs))
    assert rc == lbmhd.LBMHD_ERR_INVALID
    assert not h.value
    assert needle in lbmhd.lbmhd_last_error(None)


def test_null_arguments_rejected(lib):
    D = ctypes.POINTER(ctypes.c_double)
    p = lbmhd.lbmhd_params_srt(8, 8, 0.01, 0.01, 1.0)
    h = ctypes.c_void_p()
    assert lib.lbmhd_init(ctypes.byref(h), ctypes.byref(p), None, None, None, None, None) == -1
    assert lib.lbmhd_init(None, ctypes.byref(p), *([np.zeros(64).ctypes.data_as(D)] * 5)) == -1
    assert lib.lbmhd_step(None, 1) == -1
    assert lib.lbmhd_diagnostics(None, None) == -1
    assert lib.lbmhd_state_bytes(None) == 0
    assert lib.lbmhd_launch_count(None) == 0
    lib.lbmhd_free(None)  # no-op
    assert "handle is NULL" in lbmhd.lbmhd_last_error(None)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(lbmhd, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        lbmhd.load_library(str(tmp_path / "nope.so"))


@pytest.mark.slow
def test_bounds_checking_variant_builds_and_exports_the_same_functions():
    path = libbuild.build_checked()
    chk = ctypes.CDLL(path)
    for n in lbmhd.header_functions():
        assert hasattr(chk, n), n


def test_relative_binary16_form_host_checks(lib):
    """LBMHD_FP16_REL stores two more planes per row, so its width limit is lower (a row of all
    29 planes must stay below 2^31 elements), and ensembles refuse it; both are host checks."""
    D = ctypes.POINTER(ctypes.c_double)
    arrs = [np.ascontiguousarray(a) for a in _fields(8, 8)]
    p = lbmhd.lbmhd_params_srt(8, 8, 0.01, 0.01, 1.0, lbmhd.LBMHD_FP16_REL)
    p.nx, p.ny = 74_051_103, 3
    h = ctypes.c_void_p()
    rc = lib.lbmhd_init(ctypes.byref(h), ctypes.byref(p), *(a.ctypes.data_as(D) for a in arrs))
    assert rc == lbmhd.LBMHD_ERR_INVALID and "29 planes" in lbmhd.lbmhd_last_error(None)
    p = lbmhd.lbmhd_params_srt(8, 8, 0.01, 0.01, 1.0, lbmhd.LBMHD_FP16_REL)
    fields = (D * 5)(*(a.ctypes.data_as(D) for a in arrs))
    e = ctypes.c_void_p()
    rc = lib.lbmhd_ensemble_create(ctypes.byref(e), 1, ctypes.byref(p), fields, None)
    assert rc == lbmhd.LBMHD_ERR_INVALID and not e.value
    assert "ensembles take" in lib.lbmhd_ensemble_last_error(None).decode()
