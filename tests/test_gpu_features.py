"""GPU checks of the rest of the C ABI: checkpoint/resume, determinism, the device-pointer
entry points on a caller's stream, diagnostics (conservation, div B, instability status),
launch accounting and argument errors after a handle exists."""
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


def _params(n, precision=lbmhd.LBMHD_FP64, delta=2.0, stream=None, stencil=0):
    s, sm = oracle.srt_rates(0.002), oracle.rate_from_diffusivity(0.002)
    return lbmhd.make_params(n, n, s, sm, delta, precision, stencil, stream)


@pytest.mark.parametrize("precision", [lbmhd.LBMHD_FP64, lbmhd.LBMHD_FP32, lbmhd.LBMHD_FP16,
                                       lbmhd.LBMHD_FP16_REL])
def test_checkpoint_resume_bitwise(precision):
    fields = kh_jet(96, seed=4)
    with lbmhd.Lbmhd(_params(96, precision), *fields) as sim:
        sim.step(37)
        ck = sim.get_state()
        assert ck.nbytes == lbmhd.lbmhd_state_bytes(sim.h)
        sim.step(45)
        a = sim.populations()
        sim.set_state(ck)
        assert sim.steps == 0
        sim.step(45)
        b = sim.populations()
    assert np.array_equal(a, b)
    # restoring into a fresh handle continues the same run
    with lbmhd.Lbmhd(_params(96, precision), *kh_jet(96, seed=9)) as other:
        other.set_state(ck)
        other.step(45)
        assert np.array_equal(other.populations(), a)


@pytest.mark.parametrize("shape", [(96, 80), (3, 3), (261, 7), (300, 70)])
@pytest.mark.parametrize("precision", [lbmhd.LBMHD_FP64, lbmhd.LBMHD_FP32, lbmhd.LBMHD_FP16,
                                       lbmhd.LBMHD_FP16_REL])
def test_page_locked_host_arrays_give_the_same_bits(precision, shape):
    """Page-locked initial fields (read by the initialisation kernel directly) and page-locked
    outputs (written by the read-out kernel directly) give the same state and moments as pageable
    ones, also for output arrays at offsets inside one page-locked block; ragged grids cover
    partial column strips and row bands of the initialisation.  The row padding of the state is
    zero."""
    import torch
    nx, ny = shape
    fields = smooth_random_fields(nx, ny, seed=12, amp_u=0.04, amp_b=0.03, amp_rho=0.01)
    pin_in = torch.empty((5, ny, nx), dtype=torch.float64, pin_memory=True).numpy()
    pin_in[...] = np.stack(fields)
    block = torch.empty((6, ny, nx), dtype=torch.float64, pin_memory=True).numpy()
    s, sm = oracle.srt_rates(0.002), oracle.rate_from_diffusivity(0.002)
    p = lbmhd.make_params(nx, ny, s, sm, 2.0, precision)
    with lbmhd.Lbmhd(p, *fields) as a, lbmhd.Lbmhd(p, *pin_in) as b:
        a.step(23)
        b.step(23)
        assert np.array_equal(a.populations(), b.populations())
        state = b.get_state()
        assert np.array_equal(a.get_state(), state)
        # state rows: [ny][planes][plane] elements; columns [0, 30) and [nx + 34, plane) are pad
        elem = {lbmhd.LBMHD_FP64: 8, lbmhd.LBMHD_FP32: 4}.get(precision, 2)
        planes = 29 if precision == lbmhd.LBMHD_FP16_REL else 27
        plane = (nx + 34 + 31) // 32 * 32
        rows = state.view(np.dtype(f"u{elem}")).reshape(ny, planes, plane)
        assert not rows[:, :, :30].any() and not rows[:, :, nx + 34:].any()
        want = a.moments()
        launches = b.launches
        got = b.moments(out=[block[k + 1] for k in range(5)])
        assert b.launches == launches + 1
        assert all(g.ctypes.data == block[k + 1].ctypes.data for k, g in enumerate(got))
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", [lbmhd.LBMHD_FP32, lbmhd.LBMHD_FP16])
def test_binary32_read_out_matches_binary64_moments_of_the_state(precision):
    """The binary32 and binary16 forms read the moments out with binary32 pair sums (each
    addition's rounding error kept): rho, bx and by equal the binary64 moments of the same stored
    populations to binary64 rounding; u takes one binary32 division (four binary32 roundings)."""
    nx, ny = 96, 80
    fields = smooth_random_fields(nx, ny, seed=13, amp_u=0.05, amp_b=0.03, amp_rho=0.02)
    s, sm = oracle.srt_rates(0.002), oracle.rate_from_diffusivity(0.002)
    with lbmhd.Lbmhd(lbmhd.make_params(nx, ny, s, sm, 2.0, precision), *fields) as sim:
        sim.step(31)
        pops = sim.populations()
        got = sim.moments()
    ref = oracle.moments(pops[:9], pops[9:].reshape(2, 9, ny, nx))
    for k in (0, 3, 4):
        assert np.max(np.abs(got[k] - ref[k])) < 4e-15
    for k in (1, 2):
        assert np.all(np.abs(got[k] - ref[k]) <= 2.5e-7 * np.abs(ref[k]) + 1e-15)
    assert np.max(np.abs(ref[1])) > 0.01


def test_runs_are_deterministic_and_graph_free_path_agrees():
    import torch
    fields = kh_jet(160, seed=5)
    with lbmhd.Lbmhd(_params(160), *fields) as s1:
        s1.step(70)  # own stream: two captured graphs + 6 launches
        a = s1.populations()
    with lbmhd.Lbmhd(_params(160), *fields) as s2:
        s2.step(70)
        b = s2.populations()
    st = torch.cuda.Stream()
    with lbmhd.Lbmhd(_params(160, stream=st.cuda_stream), *fields) as s3:
        s3.step(70)  # caller's stream: plain launches
        c = s3.populations()
    # consecutive step kernels may start while their predecessor drains (programmatic dependent
    # launch); fully serialised steps, each synchronised before the next, give the same state
    with lbmhd.Lbmhd(_params(160), *fields) as s4:
        for _ in range(70):
            s4.step(1)
            s4.moments()
        d = s4.populations()
    assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, d)


def test_device_entry_points_with_torch_tensors():
    import torch
    n = 72
    fields = smooth_random_fields(n, n, seed=8, amp_u=0.04, amp_b=0.03, amp_rho=0.01)
    dev = [torch.tensor(a, device="cuda") for a in fields]
    outs = [torch.empty(n, n, dtype=torch.float64, device="cuda") for _ in range(5)]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        p = _params(n, stream=torch.cuda.current_stream().cuda_stream)
        with lbmhd.Lbmhd(p, *dev, device=True) as sim:
            sim.step(10)
            sim.moments_device(outs)
            host = sim.moments()
    st.synchronize()
    for o, h in zip(outs, host):
        assert np.array_equal(o.cpu().numpy(), h)
    # default stream (handle owns a stream; ordering with the legacy stream is automatic)
    with lbmhd.Lbmhd(_params(n), *dev, device=True) as sim:
        sim.step(10)
        sim.moments_device(outs)
        torch.cuda.synchronize()
        for o, h in zip(outs, host):
            assert np.array_equal(o.cpu().numpy(), h)
    f, g = oracle.init(*fields)
    fo, go = oracle.step(f, g, oracle.srt_rates(0.002), oracle.rate_from_diffusivity(0.002), 2.0, 10)
    for a, b in zip(host, oracle.moments(fo, go)):
        assert np.max(np.abs(a - b)) < 1e-13


@pytest.mark.parametrize("precision,tol", [(lbmhd.LBMHD_FP64, 1e-13), (lbmhd.LBMHD_FP32, 2e-6)])
def test_diagnostics_conservation(precision, tol):
    n = 128
    fields = kh_jet(n, seed=6)
    with lbmhd.Lbmhd(_params(n, precision), *fields) as sim:
        d0 = sim.diagnostics()
        sim.step(600)
        d1 = sim.diagnostics()
    assert abs(d0[0] - n * n) < 1e-9 * n * n
    assert abs(d1[0] - d0[0]) < tol * n * n                 # mass
    assert abs(d1[1] - d0[1]) < tol * n * n * 0.05          # momentum
    assert abs(d1[2] - d0[2]) < tol * n * n * 0.05
    assert abs(d1[3] - d0[3]) < tol * n * n * 0.02          # magnetic flux
    assert abs(d1[4] - d0[4]) < tol * n * n * 0.02
    assert d1[5] < d0[5]                                    # viscous decay of kinetic energy
    # diagnostics are bitwise reproducible
    with lbmhd.Lbmhd(_params(n, precision), *fields) as sim:
        sim.step(600)
        assert np.array_equal(sim.diagnostics(), d1)


def test_one_step_keeps_isotropic_div_b_at_roundoff():
    """GPU counterpart of the oracle pin: from an equilibrium with a discretely solenoidal B,
    one step keeps the isotropic divergence at roundoff."""
    n = 64
    W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])

    def iso_d(a, c):
        return sum(3 * W[i] * c[i] * np.roll(a, (-CY[i], -CX[i]), axis=(0, 1)) for i in range(1, 9))

    rho, ux, uy, _, _ = smooth_random_fields(n, n, seed=5, amp_u=0.05)
    A = smooth_random_fields(n, n, seed=6, amp_rho=0.5)[0] - 1.0
    bx, by = iso_d(A, CY), -iso_d(A, CX)
    with lbmhd.Lbmhd(_params(n, stencil=1), rho, ux, uy, bx, by) as sim:
        sim.step(1)
        d = sim.diagnostics()
    assert d[9] > 1e-3
    assert d[7] < 1e-14 * d[9]


def test_unstable_state_reported_not_faulted():
    n = 64
    rho, ux, uy, bx, by = kh_jet(n, u0=0.3, seed=1)
    s = np.full(9, 1.999)  # nu ~ 1.7e-4: far beyond the stable range for this jet
    p = lbmhd.make_params(n, n, s, 1.999, 2.0, lbmhd.LBMHD_FP64)
    with lbmhd.Lbmhd(p, rho, ux, uy, bx, by) as sim:
        sim.diagnostics()  # the initial state is fine
        with pytest.raises(lbmhd.LbmhdUnstable) as e:
            for _ in range(50):
                sim.step(200)
                sim.diagnostics()
        assert e.value.code == lbmhd.LBMHD_ERR_UNSTABLE
        assert "unstable" in lbmhd.lbmhd_last_error(sim.h)
        # the context stays usable
        sim.set_state(np.zeros(lbmhd.lbmhd_state_bytes(sim.h), np.uint8))
        sim.step(3)
    z = np.zeros((n, n))
    with lbmhd.Lbmhd(_params(n), 1 + z, 0.45 + z, z, z, z) as sim:
        with pytest.raises(lbmhd.LbmhdUnstable):
            sim.diagnostics()


def test_argument_errors_on_a_live_handle():
    fields = kh_jet(32, seed=1)
    with lbmhd.Lbmhd(_params(32), *fields) as sim:
        with pytest.raises(lbmhd.LbmhdError) as e:
            lbmhd.lbmhd_step(sim.h, -1)
        assert e.value.code == lbmhd.LBMHD_ERR_INVALID
        with pytest.raises(lbmhd.LbmhdError):
            sim.set_state(np.zeros(10, np.uint8))
        launches = sim.launches
        sim.step(0)
        assert sim.launches == launches
        sim.step(65)
        assert sim.launches == launches + 65 and sim.steps == 65


@pytest.mark.parametrize("precision", [lbmhd.LBMHD_FP64, lbmhd.LBMHD_FP32, lbmhd.LBMHD_FP16,
                                       lbmhd.LBMHD_FP16_REL])
def test_pipeline_wait_timeout_reported_and_context_usable(precision):
    """Failure detection without a fault: one block leaves out one staged-row copy, so its
    time-bounded mbarrier wait runs out; the step reports LBMHD_ERR_TIMEOUT to the host, the
    context stays usable, and a restored checkpoint continues the run exactly."""
    import time
    fields = kh_jet(96, seed=6)
    with lbmhd.Lbmhd(_params(96, precision), *fields) as ref:
        ref.step(5)
        want = ref.populations()
    with lbmhd.Lbmhd(_params(96, precision), *fields) as sim:
        sim.step(4)
        ck = sim.get_state()
        lbmhd.lbmhd_test_skip_row_copy(sim.h, True)
        t0 = time.perf_counter()
        sim.step(1)
        with pytest.raises(lbmhd.LbmhdError) as e:
            sim.moments()
        assert e.value.code == lbmhd.LBMHD_ERR_TIMEOUT
        assert "timed out" in lbmhd.lbmhd_last_error(sim.h)
        assert time.perf_counter() - t0 > 1.5  # the wait limit, not an early exit
        lbmhd.lbmhd_test_skip_row_copy(sim.h, False)
        sim.set_state(ck)
        sim.step(1)
        sim.moments()  # status clear again
        assert np.array_equal(sim.populations(), want)


@pytest.mark.slow
def test_grid_beyond_2_31_population_elements_matches_its_tile():
    """Maximum-size indexing: a 16384 x 8192 binary32 grid holds 3.6e9 population elements per
    copy (beyond 2^31).  Fields periodic with period 4096 in x evolve exactly as the 4096 x 8192
    run tiled four times: every cell's arithmetic is the same, so any index error shows up."""
    nx, ny, rep = 16384, 8192, 4
    base = smooth_random_fields(nx // rep, ny, seed=21, amp_u=0.04, amp_b=0.03, amp_rho=0.01)
    p_small = _params(1, lbmhd.LBMHD_FP32)
    p_small.nx, p_small.ny = nx // rep, ny
    with lbmhd.Lbmhd(p_small, *base) as small:
        small.step(6)
        ref = small.moments()
    p_big = _params(1, lbmhd.LBMHD_FP32)
    p_big.nx, p_big.ny = nx, ny
    with lbmhd.Lbmhd(p_big, *(np.tile(a, (1, rep)) for a in base)) as big:
        assert lbmhd.lbmhd_state_bytes(big.h) > 2 ** 31 * 4
        big.step(6)
        got = big.moments()
    for a, b in zip(got, ref):
        assert np.array_equal(a, np.tile(b, (1, rep)))
