"""GPU box filter and energy spectra against the oracle (oracle/spectrum.py)."""
import numpy as np
import pytest

from oracle import spectrum as osp
from paper_1705_09807_gb300 import lbmhd
from paper_1705_09807_gb300.inputs import kh_jet, smooth_random_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1705_09807_gb300 import build
    build.build()
    lbmhd.load_library()


@pytest.mark.parametrize("nx,ny,r", [(64, 32, 8), (300, 70, 10), (2048, 2048, 8)])
def test_block_mean(nx, ny, r):
    import torch
    a = np.random.default_rng(nx).normal(size=(ny, nx))
    t = torch.tensor(a, device="cuda")
    out = torch.empty((ny // r, nx // r), dtype=torch.float64, device="cuda")
    lbmhd.lbmhd_block_mean_device(t, r, out)
    torch.cuda.synchronize()
    ref = a.reshape(ny // r, r, nx // r, r).sum(axis=(1, 3)) / (r * r)
    if nx <= 300:
        ref = osp.block_mean(a, r)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("n,nbins", [(64, 32), (96, 60), (256, 129), (17, 9)])
def test_spectrum_matches_oracle(n, nbins):
    import torch
    f = smooth_random_fields(n, n, seed=n, amp_u=0.05, amp_b=0.04, kmax=6)
    f = [a + 1e-3 * np.random.default_rng(n + i).normal(size=(n, n)) for i, a in enumerate(f)]
    dev = [torch.tensor(a, device="cuda") for a in f[1:]]
    ek = torch.empty(nbins, dtype=torch.float64, device="cuda")
    em = torch.empty(nbins, dtype=torch.float64, device="cuda")
    work = torch.empty(lbmhd.lbmhd_energy_spectrum_work_bytes(n), dtype=torch.uint8, device="cuda")
    lbmhd.lbmhd_energy_spectrum_device(*dev, nbins, ek, em, work)
    torch.cuda.synchronize()
    rk, rm = osp.energy_spectrum(*f[1:], nbins=nbins)
    np.testing.assert_allclose(ek.cpu().numpy(), rk, rtol=1e-11, atol=1e-20)
    np.testing.assert_allclose(em.cpu().numpy(), rm, rtol=1e-11, atol=1e-20)
    # bitwise reproducible
    ek2 = torch.empty_like(ek)
    em2 = torch.empty_like(em)
    lbmhd.lbmhd_energy_spectrum_device(*dev, nbins, ek2, em2, work)
    torch.cuda.synchronize()
    assert torch.equal(ek, ek2) and torch.equal(em, em2)


def test_handle_spectrum_is_the_spectrum_of_its_moments():
    n = 128
    fields = kh_jet(n, seed=2)
    p = lbmhd.lbmhd_params_srt(n, n, 2e-3, 2e-3, 2.0, lbmhd.LBMHD_FP64)
    with lbmhd.Lbmhd(p, *fields) as sim:
        sim.step(40)
        ek, em = sim.spectrum(65)
        m = sim.moments()
    rk, rm = osp.energy_spectrum(m[1], m[2], m[3], m[4], nbins=65)
    np.testing.assert_allclose(ek, rk, rtol=1e-11, atol=1e-20)
    np.testing.assert_allclose(em, rm, rtol=1e-11, atol=1e-20)


def test_invalid_arguments():
    import torch
    t = torch.zeros((10, 12), dtype=torch.float64, device="cuda")
    out = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    lib = lbmhd.load_library()
    assert lib.lbmhd_block_mean_device(t.data_ptr(), 12, 10, 4, out.data_ptr(), None) == lbmhd.LBMHD_ERR_INVALID
    assert lib.lbmhd_energy_spectrum_device(t.data_ptr(), t.data_ptr(), t.data_ptr(), t.data_ptr(), 8, 4,
                                            out.data_ptr(), out.data_ptr(), t.data_ptr(), 8, None) \
        == lbmhd.LBMHD_ERR_INVALID


def test_les_dns_pipeline_small():
    """The LES-vs-DNS driver at a small size: all numbers finite, energies of the coarse runs
    close to the filtered DNS, the spectra non-negative."""
    from paper_1705_09807_gb300 import les_dns
    out = les_dns.run_experiment(n=256, r=4, nu_dns=8e-3, fine_steps=400, checkpoints=(200, 400),
                                 deltas=(2.0, 0.0), precision=lbmhd.LBMHD_FP64, ic="kh")
    assert out["n_coarse"] == 64 and out["nu_coarse"] == 2e-3
    assert [c["fine_step"] for c in out["checkpoints"]] == [200, 400]
    for c in out["checkpoints"]:
        ref = c["filtered_dns"]
        assert np.isfinite(ref["energy"]) and min(ref["spectrum"]) >= 0
        for name in ("delta2", "delta0"):
            e = c[name]
            assert np.isfinite(e["rel_l2_vs_filtered_dns"]) and np.isfinite(e["slope"])
            assert abs(e["energy"] / ref["energy"] - 1) < 0.05
