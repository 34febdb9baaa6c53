"""The bounds-checking build (-DLBMHD_BOUNDS_CHECK) in place of a memory sanitizer: its step
kernels check every staged-row column, the moment ring's extent, every global store and the copy
coordinates, skip an access that fails and report it at the next synchronising call.  It runs
ragged and degenerate grids in every storage form and both stencils, through the captured-graph
path, the corrected step and ensembles, in a process of its own (the checked library replaces
the normal one there), must report no failed check, and must still match the oracle.  With
checks forced to fail (LBMHD_BOUNDS_FORCE) every access they guard is skipped and the next
synchronising call reports exactly the forced bits."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent('''
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1705_09807_gb300 import lbmhd
    from paper_1705_09807_gb300.inputs import smooth_random_fields
    lbmhd.load_library(LIB)
    F = (lbmhd.LBMHD_FP64, lbmhd.LBMHD_FP32, lbmhd.LBMHD_FP16, lbmhd.LBMHD_FP16_REL)
    sizes = [(3, 3), (33, 17), (129, 20), (257, 9), (300, 70), (130, 5), (128, 4)]
    worst = {}
    for (nx, ny) in sizes:
        fields = smooth_random_fields(nx, ny, seed=nx + ny, amp_u=0.05, amp_b=0.04, amp_rho=0.02)
        s, sm = oracle.srt_rates(0.01), oracle.rate_from_diffusivity(0.015)
        for st in (0, 1):
            ref = None
            for prec in F:
                p = lbmhd.make_params(nx, ny, s, sm, 2.0, prec, st)
                with lbmhd.Lbmhd(p, *fields) as sim:
                    sim.step(34)            # one captured graph of 32 steps + 2 launches
                    sim.moments()           # synchronises: reports a failed check
                    pops = sim.populations()
                if ref is None:
                    f0, g0 = oracle.init(*fields)
                    fo, go = oracle.step(f0, g0, s, sm, 2.0, 34, stencil=st)
                    ref = np.concatenate([fo, go.reshape(18, ny, nx)])
                worst[prec] = max(worst.get(prec, 0.0), float(np.max(np.abs(pops - ref))))
    # the corrected step (static correction planes)
    nx, ny = 129, 20
    fields = smooth_random_fields(nx, ny, seed=5, amp_u=0.05, amp_b=0.04, amp_rho=0.02)
    corr = torch.full((4, ny, nx), 1e-6, dtype=torch.float32, device="cuda")
    for prec in (lbmhd.LBMHD_FP64, lbmhd.LBMHD_FP32):
        p = lbmhd.make_params(nx, ny, oracle.srt_rates(0.01), 1.5, 2.0, prec, 0)
        with lbmhd.Lbmhd(p, *fields) as sim:
            lbmhd.lbmhd_set_correction_device(sim.h, corr)
            sim.step(34)
            sim.moments()
    # ensembles of uneven members, both schedules, every storage form and stencil
    for prec, st in ((lbmhd.LBMHD_FP64, 0), (lbmhd.LBMHD_FP32, 0), (lbmhd.LBMHD_FP32, 1),
                     (lbmhd.LBMHD_FP16, 1)):
        mem = []
        for i, (nx, ny) in enumerate([(64, 64), (300, 70), (33, 17), (129, 40), (3, 3)]):
            p = lbmhd.make_params(nx, ny, oracle.srt_rates(0.005), 1.4, 2.0, prec, st)
            mem.append((p, smooth_random_fields(nx, ny, seed=60 + i, amp_u=0.05, amp_b=0.04, amp_rho=0.02)))
        for rows, persistent in ((0, False), (8, True), (1, False)):
            with lbmhd.Ensemble(mem) as ens:
                ens.set_schedule(rows, persistent)
                ens.step(9)
                ens.sync()                  # synchronises: reports a failed check
    print("CLEAN", worst[lbmhd.LBMHD_FP64], worst[lbmhd.LBMHD_FP32], worst[lbmhd.LBMHD_FP16],
          worst[lbmhd.LBMHD_FP16_REL])
''')


def test_bounds_checked_build_runs_clean_and_matches_the_oracle():
    from paper_1705_09807_gb300 import build
    lib = build.build_checked()
    code = f"ROOT = {ROOT!r}\nLIB = {lib!r}\n" + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("CLEAN")][-1]
    e64, e32, e16, e16r = (float(v) for v in line.split()[1:])
    # 34 steps: binary64 differs from the oracle in rounding order only; the binary32 and
    # binary16 stores round the deviations (|f - w| < 0.1) each step, a few ulp of 0.1 in
    # binary32 and ~3e-5 in binary16, growing at most linearly with the step count; the
    # relative binary16 form rounds the smaller f values relative to the local velocity (its g
    # values as binary16 does)
    assert e64 < 1e-13 and e32 < 3e-6 and e16 < 3e-4 and e16r < 3e-4, line


FORCED = textwrap.dedent('''
    import sys
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1705_09807_gb300 import lbmhd
    from paper_1705_09807_gb300.inputs import smooth_random_fields
    lbmhd.load_library(LIB)
    nx, ny = 129, 20
    fields = smooth_random_fields(nx, ny, seed=9, amp_u=0.05, amp_b=0.04, amp_rho=0.02)
    for prec in (lbmhd.LBMHD_FP64, lbmhd.LBMHD_FP32, lbmhd.LBMHD_FP16):
        p = lbmhd.make_params(nx, ny, oracle.srt_rates(0.01), 1.5, 2.0, prec, 0)
        with lbmhd.Lbmhd(p, *fields) as sim:
            before = sim.populations()
            sim.step(2)                 # even: back on the buffer the state was set in
            try:
                sim.moments()
                print("NOT REPORTED", prec)
            except lbmhd.LbmhdError as ex:
                print("REPORTED", prec, ex.code, str(ex))
            # every copy, staged read and store was skipped: the state is the initial one
            print("UNCHANGED", prec, bool(np.array_equal(sim.populations(), before)))
    mem = [(lbmhd.make_params(n, n, oracle.srt_rates(0.01), 1.5, 2.0, lbmhd.LBMHD_FP32, 0),
            smooth_random_fields(n, n, seed=n, amp_u=0.05, amp_b=0.04, amp_rho=0.02)) for n in (16, 40)]
    with lbmhd.Ensemble(mem) as ens:
        ens.step(2)
        try:
            ens.sync()
            print("NOT REPORTED ensemble")
        except lbmhd.LbmhdError as ex:
            print("REPORTED ensemble", ex.code, str(ex))
''')


def test_forced_check_failures_are_skipped_and_reported():
    from paper_1705_09807_gb300 import build, lbmhd
    lib = build.build_checked()
    code = f"ROOT = {ROOT!r}\nLIB = {lib!r}\n" + FORCED
    env = dict(os.environ, LBMHD_BOUNDS_FORCE="0xd")  # staged column, global store, copy
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600,
                       env=env)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = r.stdout.splitlines()
    assert not [ln for ln in out if ln.startswith("NOT REPORTED")], r.stdout
    rep = [ln for ln in out if ln.startswith("REPORTED")]
    assert len(rep) == 4, r.stdout
    for ln in rep:
        assert f" {lbmhd.LBMHD_ERR_INVALID} " in ln and "flags 0xd" in ln, ln
    unchanged = [ln for ln in out if ln.startswith("UNCHANGED")]
    assert len(unchanged) == 3 and all(ln.endswith("True") for ln in unchanged), r.stdout


FULL = textwrap.dedent('''
    import sys
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1705_09807_gb300 import lbmhd
    from paper_1705_09807_gb300.inputs import kh_jet
    lbmhd.load_library(LIB)
    # the benchmark's launch configurations: 2048^2 (54-row binary32 bands, one wave of
    # blocks) and 4096^2, every storage form
    for n, prec, delta, steps in ((2048, lbmhd.LBMHD_FP32, 0.0, 34), (2048, lbmhd.LBMHD_FP16, 2.0, 34),
                                  (2048, lbmhd.LBMHD_FP64, 2.0, 3), (4096, lbmhd.LBMHD_FP32, 2.0, 3),
                                  (4096, lbmhd.LBMHD_FP16, 0.0, 3)):
        p = lbmhd.lbmhd_params_srt(n, n, 5e-4, 5e-4, delta, prec)
        with lbmhd.Lbmhd(p, *kh_jet(n, seed=1)) as sim:
            sim.step(steps)
            rho = sim.moments()[0]
            assert np.all(np.isfinite(rho)) and abs(rho.mean() - 1) < 1e-3
        print("CLEAN", n, prec)
    # the 48-run ensemble (16 each of 128^2, 512^2, 1024^2), both schedules
    mem = []
    for i, n in enumerate([128] * 16 + [512] * 16 + [1024] * 16):
        p = lbmhd.lbmhd_params_srt(n, n, 2e-3, 2e-3, 2.0, lbmhd.LBMHD_FP32)
        mem.append((p, kh_jet(n, seed=100 + i)))
    with lbmhd.Ensemble(mem) as ens:
        for rows, persistent in ((0, False), (8, True)):
            ens.set_schedule(rows, persistent)
            ens.step(3)
            ens.sync()
    print("CLEAN ensemble")
''')


@pytest.mark.slow
def test_bounds_checked_build_at_the_benchmark_sizes():
    from paper_1705_09807_gb300 import build
    lib = build.build_checked()
    code = f"ROOT = {ROOT!r}\nLIB = {lib!r}\n" + FULL
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert r.stdout.count("CLEAN") == 6, r.stdout
