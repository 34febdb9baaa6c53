"""Ensembles: many runs of different sizes advanced by one launch per step.  Every member must
equal the same run made alone, under every schedule, through the captured-graph path and after
autotuning: bitwise with the central stencil (the tiling does not change any cell's
arithmetic); with the isotropic stencil the ensemble kernel is a separate instantiation whose
floating-point contractions the compiler may choose differently, which was measured at one
unit in the last place (binary64 5.6e-17, binary32 2.1e-8, binary16 1.5e-5 after 9 steps)."""
import numpy as np
import pytest

import oracle
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


def _members(precision, stencil=0):
    specs = [(64, 64, 0.002, 2.0), (300, 70, 0.01, 1.0), (129, 40, 0.005, 0.0), (33, 17, 0.02, 3.0),
             (256, 256, 0.003, 2.0)]
    out = []
    for i, (nx, ny, nu, delta) in enumerate(specs):
        s = oracle.srt_rates(nu)
        if i == 1:
            s[5], s[6], s[7], s[8] = 1.35, 1.2, 1.45, 1.1
        p = lbmhd.make_params(nx, ny, s, oracle.rate_from_diffusivity(1.5 * nu), delta, precision, stencil)
        f = smooth_random_fields(nx, ny, seed=40 + i, amp_u=0.05, amp_b=0.04, amp_rho=0.02)
        out.append((p, f))
    return out


def _alone(members, nsteps):
    res = []
    for p, f in members:
        with lbmhd.Lbmhd(p, *f) as sim:
            sim.step(nsteps)
            res.append(sim.populations())
    return res


@pytest.mark.parametrize("precision,stencil", [(lbmhd.LBMHD_FP64, 0), (lbmhd.LBMHD_FP32, 1),
                                               (lbmhd.LBMHD_FP16, 0)])
@pytest.mark.parametrize("rows,persistent", [(0, False), (0, True), (8, False), (16, True),
                                             (256, False)])
def test_members_equal_runs_made_alone(precision, stencil, rows, persistent):
    mem = _members(precision, stencil)
    ref = _alone(mem, 9)
    with lbmhd.Ensemble(mem) as ens:
        ens.set_schedule(rows, persistent)
        ens.step(9)
        ens.sync()
        tol = 0.0 if stencil == 0 else {lbmhd.LBMHD_FP64: 1e-15, lbmhd.LBMHD_FP32: 1e-7,
                                         lbmhd.LBMHD_FP16: 4e-5}[precision]
        for i in range(len(mem)):
            assert np.max(np.abs(ens.populations(i) - ref[i])) <= tol, i
        assert ens.launches == 9


def test_graph_path_autotune_and_oracle():
    mem = _members(lbmhd.LBMHD_FP64)
    ref = _alone(mem, 75)
    with lbmhd.Ensemble(mem) as ens:
        ens.step(5)
        before = [ens.populations(i) for i in range(len(mem))]
        ms = ens.autotune(trial_steps=4)
        assert ms > 0
        sch = ens.schedule()
        assert sch["tiles"] > 0 and sch["blocks"] > 0
        for i in range(len(mem)):  # autotuning leaves the states untouched
            assert np.array_equal(ens.populations(i), before[i])
        ens.step(70)  # two captured 32-step graphs and 6 single launches
        ens.sync()
        for i in range(len(mem)):
            assert np.array_equal(ens.populations(i), ref[i]), i
    # one member against the oracle
    p, f = mem[1]
    fo, go = oracle.init(*f)
    s = np.array(list(p.s))
    fo, go = oracle.step(fo, go, s, p.s_m, p.delta, 75)
    assert np.max(np.abs(ref[1] - np.concatenate([fo, go.reshape(18, p.ny, p.nx)]))) < 1e-13


def test_member_handles_are_read_only():
    mem = _members(lbmhd.LBMHD_FP32)[:2]
    with lbmhd.Ensemble(mem) as ens:
        h = ens.member(0)
        with pytest.raises(lbmhd.LbmhdError) as e:
            lbmhd.lbmhd_step(h, 1)
        assert e.value.code == lbmhd.LBMHD_ERR_INVALID
        lbmhd.lbmhd_free(h)  # a no-op for members
        ens.step(3)
        d = lbmhd.lbmhd_diagnostics(ens.member(1))
        assert np.isfinite(d).all()


@pytest.mark.slow
def test_full_size_48_run_ensemble_sampled():
    """The 48-run ensemble of the benchmark (16 each of 128^2, 512^2, 1024^2, binary32,
    Delta = 2) in its autotuned launch configuration, through the graph path: one more
    ensemble step must equal the oracle's single-cell collision of each sampled member's own
    state at sampled cells (f_i(x + c_i) after the step = f*_i(x) before it), to 1e-7 as for
    the single 2048^2 grid."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    mem = bench.ensemble_members()
    picks = (0, 15, 16, 31, 32, 47)
    rng = np.random.default_rng(11)
    with lbmhd.Ensemble(mem) as ens:
        ens.step(4)
        ens.autotune(trial_steps=4)
        ens.step(36)  # one captured 32-step graph and 4 single launches
        before = {i: ens.populations(i) for i in picks}
        ens.step(1)
        after = {i: ens.populations(i) for i in picks}
    worst = 0.0
    for i in picks:
        p, _ = mem[i]
        n = p.nx
        s = np.array(list(p.s))
        f, g = before[i][:9], before[i][9:].reshape(2, 9, n, n)
        pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0), (127, 5), (min(128, n - 1), n // 2),
               (n // 2, 0)]
        pts += [tuple(int(v) for v in rng.integers(0, n, 2)) for _ in range(25)]
        for (x, y) in pts:
            fs, gs = oracle.collide_cell(f, g, s, p.s_m, p.delta, x, y)
            for q in range(9):
                xd, yd = (x + cx[q]) % n, (y + cy[q]) % n
                worst = max(worst, abs(after[i][q, yd, xd] - fs[q]), abs(after[i][9 + q, yd, xd] - gs[0, q]),
                            abs(after[i][18 + q, yd, xd] - gs[1, q]))
    assert worst < 1e-7, worst
