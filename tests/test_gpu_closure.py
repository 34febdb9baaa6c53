"""The learned closure on the GPU against the FP64 oracle (oracle/closure.py): back-propagation,
the binary32 and bf16 tensor-core forward passes, features and training targets from a fine
state, the correction inside the fused step (against the oracle's corrected step), and the
closure-in-the-loop step against the same correction supplied statically."""
import numpy as np
import pytest

import oracle
from oracle import closure as oc
from paper_1705_09807_gb300 import lbmhd
from paper_1705_09807_gb300.inputs import kh_jet, smooth_random_fields, splitmix64_uniform

pytestmark = pytest.mark.gpu
IN_SCALE = np.array([0.05, 0.05, 0.03, 0.03] + [0.005] * 8, dtype=np.float32)
OUT_SCALE = np.array([1e-6, 1e-6, 1e-6, 1e-6], dtype=np.float32)


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1705_09807_gb300 import build
    build.build()
    lbmhd.load_library()


def _params(seed=3):
    u = splitmix64_uniform(seed, oc.num_params())
    theta = oc.init_params(seed) + 0.02 * (2 * u - 1)
    return theta


def _batch(b=2, h=12, w=20, seed=5):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(b, 12, h, w)), 0.3 * rng.normal(size=(b, 4, h, w))


def test_gradient_matches_oracle():
    import torch
    theta = _params()
    x, t = _batch()
    with lbmhd.Closure(theta, IN_SCALE, OUT_SCALE) as cl:
        loss, g = cl.gradient(torch.tensor(x, dtype=torch.float32, device="cuda"),
                              torch.tensor(t, dtype=torch.float32, device="cuda"))
    th32 = theta.astype(np.float32).astype(np.float64)
    L, gref = oc.gradient(th32, x.astype(np.float32).astype(np.float64),
                          t.astype(np.float32).astype(np.float64))
    assert abs(loss - L) < 1e-5 * L
    err = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    assert err < 1e-5, err


def test_forward_binary32_and_tensor_cores():
    import torch
    theta = _params(7)
    x, _ = _batch(b=3, h=16, w=37, seed=9)  # width not a multiple of 16: ragged 16 x 16 tiles
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    ref = oc.forward(theta.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64))[-1]
    with lbmhd.Closure(theta, IN_SCALE, OUT_SCALE) as cl:
        out32 = torch.empty((3, 4, 16, 37), dtype=torch.float32, device="cuda")
        cl.forward(xt, out32, tensor_cores=False)
        out16 = torch.empty_like(out32)
        cl.forward(xt, out16, tensor_cores=True)
    o32, o16 = out32.cpu().numpy(), out16.cpu().numpy()
    scale = np.sqrt(np.mean(ref ** 2))
    assert np.max(np.abs(o32 - ref)) < 1e-5 * max(1.0, np.max(np.abs(ref)))
    # bf16 operands (8-bit significand), binary32 accumulation over up to 288 terms
    assert np.sqrt(np.mean((o16 - ref) ** 2)) < 2e-2 * scale


def test_training_pair_and_features_match_oracle():
    import torch
    n, r, delta = 64, 4, 2.0
    f = smooth_random_fields(n, n, seed=21, amp_u=0.05, amp_b=0.04, amp_rho=0.02, kmax=8)
    fine = torch.tensor(np.stack(f), device="cuda")
    m = n // r
    x = torch.empty((12, m, m), dtype=torch.float32, device="cuda")
    t = torch.empty((4, m, m), dtype=torch.float32, device="cuda")
    work = torch.empty(9 * m * m, dtype=torch.float64, device="cuda")
    with lbmhd.Closure(_params(), IN_SCALE, OUT_SCALE) as cl:
        cl.training_pair(fine, r, delta, x, t, work)
        xr, tr = oc.training_pair(*f, r, delta, IN_SCALE, OUT_SCALE)
        np.testing.assert_allclose(x.cpu().numpy(), xr, rtol=2e-6, atol=1e-6)
        np.testing.assert_allclose(t.cpu().numpy(), tr, rtol=1e-4, atol=1e-4 * np.max(np.abs(tr)))
        # features of a coarse state given as rho, u, B planes
        st = [oc.box(a, r) for a in (f[0], f[0] * f[1], f[0] * f[2], f[3], f[4])]
        R = st[0]
        state = torch.tensor(np.stack([R, st[1] / R, st[2] / R, st[3], st[4]]), device="cuda")
        x2 = torch.empty_like(x)
        an = torch.empty((4, m, m), dtype=torch.float32, device="cuda")
        cl.features(state, delta, x2, an)
        np.testing.assert_allclose(x2.cpu().numpy(), xr, rtol=2e-6, atol=1e-6)
        ar = oc.analytic(R, st[1], st[2], st[3], st[4], delta)
        np.testing.assert_allclose(an.cpu().numpy(), ar, rtol=1e-5, atol=1e-6 * np.max(np.abs(ar)))


def test_tensor_core_forward_with_more_tiles_than_resident_ctas():
    """2 x 13 x 19 = 494 ragged 16 x 16 tiles, more than the 2 x 152 CTAs the tensor-core kernel
    keeps resident, so CTAs take several tiles in turn (the mbarrier phases and the TMEM
    accumulators carry over from tile to tile); checked against the binary32 forward pass."""
    import torch
    theta = _params(11)
    rng = np.random.default_rng(12)
    x = torch.tensor(rng.normal(size=(2, 12, 200, 300)), dtype=torch.float32, device="cuda")
    with lbmhd.Closure(theta, IN_SCALE, OUT_SCALE) as cl:
        o32 = torch.empty((2, 4, 200, 300), dtype=torch.float32, device="cuda")
        cl.forward(x, o32, tensor_cores=False)
        o16 = torch.empty_like(o32)
        cl.forward(x, o16, tensor_cores=True)
        o16b = torch.empty_like(o32)
        cl.forward(x, o16b, tensor_cores=True)
    a, b = o32.cpu().numpy(), o16.cpu().numpy()
    assert np.isfinite(b).all()
    assert np.array_equal(b, o16b.cpu().numpy())  # deterministic
    scale = np.sqrt(np.mean(a ** 2))
    assert np.sqrt(np.mean((b - a) ** 2)) < 2e-2 * scale
    # every tile is written: the worst tile's error is of the same order as the mean
    err = np.abs(b - a).reshape(2, 4, 200, 300)
    worst = max(err[:, :, y:y + 16, x0:x0 + 16].mean() for y in range(0, 200, 16) for x0 in range(0, 300, 16))
    assert worst < 10 * err.mean() + 1e-3 * scale


def test_tensor_core_wait_timeout_reported_and_closure_usable():
    """Failure detection without a fault: the hook leaves out the first layer's MMAs, so the
    kernel's time-bounded completion wait runs out; the call reports LBMHD_ERR_TIMEOUT, and
    the next call (hook off) gives the normal result."""
    import time
    import torch
    theta = _params(13)
    rng = np.random.default_rng(14)
    x = torch.tensor(rng.normal(size=(1, 12, 40, 40)), dtype=torch.float32, device="cuda")
    with lbmhd.Closure(theta, IN_SCALE, OUT_SCALE) as cl:
        ref = torch.empty((1, 4, 40, 40), dtype=torch.float32, device="cuda")
        cl.forward(x, ref, tensor_cores=True)
        cl.test_skip_mma(True)
        out = torch.empty_like(ref)
        t0 = time.perf_counter()
        with pytest.raises(lbmhd.LbmhdError) as e:
            cl.forward(x, out, tensor_cores=True)
        assert e.value.code == lbmhd.LBMHD_ERR_TIMEOUT
        assert time.perf_counter() - t0 > 1.5  # the wait limit, not an early exit
        cl.test_skip_mma(False)
        again = torch.empty_like(ref)
        cl.forward(x, again, tensor_cores=True)
        assert torch.equal(again, ref)


@pytest.mark.parametrize("precision,tol", [(lbmhd.LBMHD_FP64, 1e-13), (lbmhd.LBMHD_FP32, 2e-7)])
def test_static_correction_matches_oracle(precision, tol):
    import torch
    nx, ny = 96, 40
    f = smooth_random_fields(nx, ny, seed=2, amp_u=0.05, amp_b=0.04, amp_rho=0.02)
    corr = (1e-4 * np.random.default_rng(3).normal(size=(4, ny, nx))).astype(np.float32)
    s, sm = oracle.srt_rates(0.01), oracle.rate_from_diffusivity(0.01)
    fo, go = oracle.init(*f)
    fo, go = oracle.step_corrected(fo, go, s, sm, 2.0, 7, corr.astype(np.float64))
    ref = np.concatenate([fo, go.reshape(18, ny, nx)])
    ct = torch.tensor(corr, device="cuda")
    with lbmhd.Lbmhd(lbmhd.make_params(nx, ny, s, sm, 2.0, precision), *f) as sim:
        lbmhd.lbmhd_set_correction_device(sim.h, ct)
        sim.step(7)
        pops = sim.populations()
    assert np.max(np.abs(pops - ref)) < tol
    # and the correction really acts
    fp, gp = oracle.step(*oracle.init(*f), s, sm, 2.0, 7)
    assert np.max(np.abs(np.concatenate([fp, gp.reshape(18, ny, nx)]) - ref)) > 1e-6


@pytest.mark.parametrize("n", [64, 256])  # 256: the learned-closure LES grid (256 tiles)
@pytest.mark.parametrize("precision", [lbmhd.LBMHD_FP64, lbmhd.LBMHD_FP32])
def test_closure_in_the_loop_matches_its_static_correction(precision, n):
    """The attached closure forms u, B and the features from the populations in binary32 inside
    its one fused network launch; the same correction by hand goes through the binary64 moments,
    the features entry point and the forward pass.  They differ only by the rounding of the
    features (and so, rarely, of their bf16 copies), so the corrected steps agree to a small
    fraction of the correction's own effect on the populations."""
    import torch
    f = kh_jet(n, seed=5)
    s, sm = oracle.srt_rates(0.002), oracle.rate_from_diffusivity(0.002)
    p = lbmhd.make_params(n, n, s, sm, 2.0, precision)
    with lbmhd.Closure(_params(), IN_SCALE, OUT_SCALE) as cl, lbmhd.Lbmhd(p, *f) as a, \
            lbmhd.Lbmhd(p, *f) as b, lbmhd.Lbmhd(p, *f) as plain:
        cl.attach(a.h)
        launches = a.launches
        a.step(1)
        assert a.launches == launches + 2  # network + corrected step
        # the same correction by hand: moments -> features -> tensor-core network -> scale
        st = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(5)]
        b.moments_device(st)
        torch.cuda.synchronize()
        x = torch.empty((1, 12, n, n), dtype=torch.float32, device="cuda")
        cl.features(torch.stack(st), 0.0, x.view(12, n, n))
        out = torch.empty((1, 4, n, n), dtype=torch.float32, device="cuda")
        cl.forward(x, out, tensor_cores=True)
        corr = (out[0] * torch.tensor(OUT_SCALE, device="cuda")[:, None, None]).contiguous()
        lbmhd.lbmhd_set_correction_device(b.h, corr)
        b.step(1)
        plain.step(1)
        pa, pb, pp = a.populations(), b.populations(), plain.populations()
        effect = pb - pp
        assert np.max(np.abs(effect)) > 0
        assert np.max(np.abs(pa - pb)) < 5e-2 * np.max(np.abs(effect))
        assert np.sqrt(np.mean((pa - pb) ** 2)) < 1e-2 * np.sqrt(np.mean(effect ** 2))
        lbmhd.lbmhd_detach_closure(a.h)
        a.step(2)  # back to the analytic closure alone


def test_training_lowers_the_loss():
    import torch
    x, t = _batch(b=2, h=16, w=16, seed=12)
    t = 0.5 * np.tanh(x[:, :4])  # a learnable map
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    with lbmhd.Closure(_params(), IN_SCALE, OUT_SCALE) as cl:
        l0 = cl.train_step(xt, tt, 3e-3)
        for _ in range(150):
            l1 = cl.train_step(xt, tt, 3e-3)
    assert l1 < 0.3 * l0


def test_trained_network_beats_the_analytic_closure_a_priori():
    """What the network gains, a priori and a posteriori.  Trained on box-filtered fine runs
    (256^2 -> 64^2, three seeded jets), it must reduce the held-out error of the subgrid terms
    far below the analytic closure's (measured ratio |T - net(X)| / |T| of 0.15 / 0.19 / 0.19 /
    0.19 on the four channels of an unseen run; asserted < 0.4).

    A posteriori (the 64^2 LES run from the filtered initial fields against the filtered DNS,
    relative L2 of the total-energy spectra at DNS step 400) the gain is almost nothing: measured
    2.0544e-3 with the network against 2.0597e-3 with the analytic closure alone (0.26% lower)
    and 2.0597e-3 with no closure at all (the analytic terms change it by 1e-8 relative: in this
    resolved, low-Re run the subgrid terms barely move the flow).  The assertions record that
    result: the network lowers the error by between 0.05% and 1%, and the analytic closure and
    no closure agree to 1e-5."""
    from paper_1705_09807_gb300 import learned_closure as lc
    res = lc.run(n=256, r=4, nu_dns=8e-3, delta=2.0, train_seeds=range(3), test_seed=100,
                 snapshots=(200, 400, 600, 800), iters=400, batch=4, lr=2e-3)
    assert res["loss_last"] < 0.5 * res["loss_first"]
    ratio = res["a_priori_test"]["ratio"]
    assert max(ratio) < 0.4, ratio
    assert len(res["a_posteriori_test"]) >= 1
    for rec in res["a_posteriori_test"]:
        a, net, none = rec["analytic"], rec["analytic_plus_network"], rec["no_closure"]
        assert 1e-3 < a < 5e-3, rec  # the coarse run tracks the filtered DNS to ~0.2%
        assert 0.99 < net / a < 0.9995, rec
        assert abs(a / none - 1.0) < 1e-5, rec


def _identity_paths(feats):
    """Network parameters whose output channel o is tanh(tanh(x[feats[o]])) at every cell: the
    centre tap of layer 1 routes feature feats[o] to hidden channel o, layers 2 and 3 pass hidden
    channel o on (centre taps of weight 1), every other weight and every bias is zero."""
    (W1, b1), (W2, b2), (W3, b3) = oc.unpack(np.zeros(oc.num_params()))
    W1, W2, W3 = W1.copy(), W2.copy(), W3.copy()
    for o, k in enumerate(feats):
        W1[o, k, 1, 1] = 1.0
        W2[o, o, 1, 1] = 1.0
        W3[o, o, 1, 1] = 1.0
    return np.concatenate([W1.ravel(), np.zeros(32), W2.ravel(), np.zeros(32), W3.ravel(), np.zeros(4)])


@pytest.mark.parametrize("precision", [lbmhd.LBMHD_FP64, lbmhd.LBMHD_FP32])
def test_fused_network_features_match_the_oracle_per_channel(precision):
    """The attached closure's kernel forms its 12 input features itself, in binary32, from the
    pulled populations (u = J / rho, B and their central differences, over in_scale).  With a
    network that passes feature k to an output unchanged but for tanh(tanh(.)) and bf16
    rounding, its correction planes show those features cell by cell: they must equal the
    oracle's features of the same state (binary64 moments of the GPU's own populations) to bf16
    accuracy -- three passes of four channels cover all twelve."""
    import torch
    n = 64
    fields = kh_jet(n, u0=0.05, delta_frac=1 / 16, b0=0.02, pert=2e-2, seed=8)
    s, sm = oracle.srt_rates(0.002), oracle.rate_from_diffusivity(0.002)
    p = lbmhd.make_params(n, n, s, sm, 2.0, precision)
    with lbmhd.Lbmhd(p, *fields) as sim:
        sim.step(60)
        pops = sim.populations()
        f, g = pops[:9], pops[9:].reshape(2, 9, n, n)
        rho, ux, uy, bx, by = oracle.moments(f, g)
        raw = oc.features(rho, ux, uy, bx, by, np.ones(12))
        # scale every channel to a largest magnitude of 0.5 (the nonlinearity matters)
        top = np.abs(raw).max(axis=(1, 2))
        assert np.all(top > 0), top  # every channel carries a signal in this state
        in_scale = (top / 0.5).astype(np.float32)
        feats = raw / in_scale.astype(np.float64)[:, None, None]
        out_scale = np.array([1.0, 2.0, 3.0, 4.0], dtype=np.float32)
        corr = torch.empty((4, n, n), dtype=torch.float32, device="cuda")
        for group in ((0, 1, 2, 3), (4, 5, 6, 7), (8, 9, 10, 11)):
            theta = _identity_paths(group)
            with lbmhd.Closure(theta, in_scale, out_scale) as cl:
                cl.attach(sim.h)
                lbmhd.lbmhd_closure_correction_device(sim.h, corr)
                got = corr.cpu().numpy().astype(np.float64)
                lbmhd.lbmhd_detach_closure(sim.h)
            for o, k in enumerate(group):
                want = out_scale[o] * np.tanh(np.tanh(feats[k]))
                err = np.abs(got[o] - want)
                # bf16 rounding of the feature and of two hidden activations (2^-9 relative
                # each), the tanh.approx instruction: below 1.5% of the channel's range
                assert err.max() < 1.5e-2 * np.abs(want).max(), (k, err.max(), np.abs(want).max())
                assert np.sqrt(np.mean(err ** 2)) < 5e-3 * np.abs(want).max(), k
