"""GPU test of lbmhd_diagnostics_fields_noalloc, the diagnostics entry point for callers that
cannot allocate device memory (code that must draw every byte from another framework's pool, or
that runs under a fixed memory budget).  It is called through the C ABI on moment fields the
handle wrote into caller tensors, twice in a row, and compared with lbmhd_diagnostics, which
uses the handle's own scratch buffers.

The file name sorts last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

import oracle
from paper_1705_09807_gb300 import lbmhd
from paper_1705_09807_gb300.inputs import kh_jet

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1705_09807_gb300 import build
    build.build()
    lbmhd.load_library()


def _compare(got, ref):
    # sums (0..6): same values summed in another grouping -> relative 1e-13 of their scale
    # maxima (7..9): order-independent -> identical
    scale = np.array([ref[0], abs(ref[0]) * 0.05, abs(ref[0]) * 0.05, abs(ref[0]) * 0.02,
                      abs(ref[0]) * 0.02, max(ref[5], 1e-30), max(ref[6], 1e-30)])
    assert np.all(np.abs(got[:7] - ref[:7]) <= 1e-13 * scale)
    assert np.array_equal(got[7:10], ref[7:10])


@pytest.mark.parametrize("nx,ny,precision", [(200, 150, lbmhd.LBMHD_FP64),
                                             (1024, 1024, lbmhd.LBMHD_FP32),
                                             (3, 5, lbmhd.LBMHD_FP64)])
def test_noalloc_diagnostics_match_handle_diagnostics(nx, ny, precision):
    import torch
    fields = kh_jet(nx, ny=ny, seed=3)
    s, sm = oracle.srt_rates(0.002), oracle.rate_from_diffusivity(0.002)
    p = lbmhd.make_params(nx, ny, s, sm, 2.0, precision)
    dev = [torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(5)]
    out = torch.full((lbmhd.LBMHD_NDIAG + 1,), -1.0, dtype=torch.float64, device="cuda")
    with lbmhd.Lbmhd(p, *fields) as sim:
        sim.step(30)
        ref = sim.diagnostics()
        sim.moments_device(dev)
        torch.cuda.synchronize()
        results = []
        for _ in range(2):  # two calls in a row share the library's scratch array
            out.fill_(-1.0)
            lbmhd.lbmhd_diagnostics_fields_noalloc(dev, out)
            torch.cuda.synchronize()
            results.append(out.cpu().numpy().copy())
    for r in results:
        _compare(r[:lbmhd.LBMHD_NDIAG], ref)
        assert r[lbmhd.LBMHD_NDIAG] == 0.0
    assert np.array_equal(results[0], results[1])


def test_noalloc_flags_unstable_and_rejects_oversize():
    import torch
    n = 64
    dev = [torch.zeros((n, n), dtype=torch.float64, device="cuda") for _ in range(5)]
    dev[0].fill_(1.0)
    dev[1][3, 4] = 0.5  # |u| > 0.4 in one cell
    out = torch.zeros(lbmhd.LBMHD_NDIAG + 1, dtype=torch.float64, device="cuda")
    lbmhd.lbmhd_diagnostics_fields_noalloc(dev, out)
    torch.cuda.synchronize()
    assert out[lbmhd.LBMHD_NDIAG].item() == 1.0
    assert out[0].item() == n * n
    # larger than the fixed scratch allows: rejected on the host before any GPU work
    lib = lbmhd.load_library()
    ptrs = [t.data_ptr() for t in dev]
    rc = lib.lbmhd_diagnostics_fields_noalloc(*ptrs, 8192, 4096, out.data_ptr(), None)
    assert rc == lbmhd.LBMHD_ERR_INVALID
    assert "at most" in lbmhd.lbmhd_last_error(None)
    rc = lib.lbmhd_diagnostics_fields_noalloc(*ptrs, 2, 64, out.data_ptr(), None)
    assert rc == lbmhd.LBMHD_ERR_INVALID
