"""LES-vs-DNS comparison (the experiment of Sec. 3), on synthetic initial conditions.

A DNS (Delta = 0) runs on an n x n grid.  Coarse runs on the (n/r)^2 grid start from the r x r
box-filtered DNS initial fields: LES runs with filter widths Delta (in coarse lattice units;
the paper uses Delta = 1 and 2) and an unfiltered coarse run (Delta = 0, the paper's "DNS on
the coarse grid").  All grids keep the Reynolds number: the lattice viscosity scales with the
grid, nu_coarse = nu_dns / r, and one coarse step matches r DNS steps (Sec. 3: on halving the
grid, a DNS step of 2 t0 corresponds to an LES step t0).  At each checkpoint the DNS moments are
box-filtered onto the coarse grid and the shell-summed total (kinetic + magnetic) energy
spectra of the filtered DNS and of every coarse run are compared; the spectral slopes over a
wavenumber range are fitted as in Fig. FinalTotEn.  Every field operation (steps, moments,
box filter, spectra, stability diagnostics) runs in the library's CUDA kernels; this module
only sequences the calls and reduces the returned spectra to a few numbers.

    python -m paper_1705_09807_gb300.les_dns --paper          # the paper's setup (Sec. 3)
    python -m paper_1705_09807_gb300.les_dns --n 2048 --r 8 --nu-dns 8e-3 --fine-steps 20000
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import lbmhd
from .inputs import kh_jet, sech2_jet


def spectral_errors(a, b, kmax):
    """(relative L2, RMS of log10 ratio) of spectrum a against reference b over shells 1..kmax."""
    sa, sb = a[1:kmax + 1], b[1:kmax + 1]
    rel = float(np.linalg.norm(sa - sb) / np.linalg.norm(sb))
    ok = (sa > 0) & (sb > 0)
    logrms = float(np.sqrt(np.mean(np.log10(sa[ok] / sb[ok]) ** 2))) if ok.any() else float("nan")
    return rel, logrms


def fitted_slope(e, k1, k2):
    """Least-squares slope of log E(k) against log k over shells k1..k2."""
    k = np.arange(k1, k2 + 1)
    y = e[k1:k2 + 1]
    ok = y > 0
    if ok.sum() < 3:
        return float("nan")
    return float(np.polyfit(np.log(k[ok]), np.log(y[ok]), 1)[0])


def run_experiment(n=2048, r=2, nu_dns=2e-3, fine_steps=1_560_000, checkpoints=(400_000, 800_000,
                   1_560_000), deltas=(2.0, 1.0, 0.0), precision=lbmhd.LBMHD_FP32, ic="sech2",
                   seed=1, slope_range=None, keep_spectra=True):
    import torch
    m = n // r
    nu_c = nu_dns / r
    fields = sech2_jet(n) if ic == "sech2" else kh_jet(n, seed=seed)
    dns = lbmhd.Lbmhd(lbmhd.lbmhd_params_srt(n, n, nu_dns, nu_dns, 0.0, precision), *fields)
    fine = [torch.tensor(a, device="cuda") for a in fields]
    coarse = [torch.empty((m, m), dtype=torch.float64, device="cuda") for _ in range(5)]
    for a, b in zip(fine, coarse):
        lbmhd.lbmhd_block_mean_device(a, r, b)
    torch.cuda.synchronize()
    runs = {f"delta{d:g}": lbmhd.Lbmhd(lbmhd.lbmhd_params_srt(m, m, nu_c, nu_c, d, precision), *coarse,
                                       device=True) for d in deltas}
    del fine
    nb = m // 2 + 1
    kmax = m // 2 - 1
    k1, k2 = slope_range or (max(2, m // 128), max(8, m // 8))
    work = torch.empty(lbmhd.lbmhd_energy_spectrum_work_bytes(m), dtype=torch.uint8, device="cuda")
    ek = torch.empty(nb, dtype=torch.float64, device="cuda")
    em = torch.empty(nb, dtype=torch.float64, device="cuda")
    fine_mom = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(5)]
    out = {"n_dns": n, "r": r, "n_coarse": m, "nu_dns": nu_dns, "nu_coarse": nu_c, "ic": ic,
           "precision": precision, "deltas": list(deltas), "slope_range": [k1, k2],
           "checkpoints": []}
    alive = {name: True for name in runs}
    done = 0
    t0 = time.perf_counter()
    for cp in checkpoints:
        step = (cp - done) // r * r
        dns.step(step)
        for name, sim in runs.items():
            if alive[name]:
                sim.step(step // r)
        done += step
        dns.moments_device(fine_mom)
        torch.cuda.synchronize()
        for a, b in zip(fine_mom, coarse):
            lbmhd.lbmhd_block_mean_device(a, r, b)
        lbmhd.lbmhd_energy_spectrum_device(coarse[1], coarse[2], coarse[3], coarse[4], nb, ek, em, work)
        torch.cuda.synchronize()
        ref = ek.cpu().numpy() + em.cpu().numpy()
        rec = {"fine_step": done, "coarse_step": done // r,
               "filtered_dns": {"energy": float(ref.sum()), "slope": fitted_slope(ref, k1, k2)}}
        try:
            dns.diagnostics()
        except lbmhd.LbmhdUnstable:
            rec["filtered_dns"]["diverged"] = True
        if keep_spectra:
            rec["filtered_dns"]["spectrum"] = ref.tolist()
        for name, sim in runs.items():
            entry = {}
            if alive[name]:
                try:
                    sim.diagnostics()
                except lbmhd.LbmhdUnstable:
                    alive[name] = False
                    entry["diverged_by_coarse_step"] = done // r
            if alive[name]:
                k_, m_ = sim.spectrum(nb)
                tot = k_ + m_
                rel, logrms = spectral_errors(tot, ref, kmax)
                entry.update({"energy": float(tot.sum()), "slope": fitted_slope(tot, k1, k2),
                              "rel_l2_vs_filtered_dns": rel, "log10_rms_vs_filtered_dns": logrms})
                if keep_spectra:
                    entry["spectrum"] = tot.tolist()
            rec[name] = entry
        out["checkpoints"].append(rec)
    out["seconds"] = round(time.perf_counter() - t0, 3)
    dns.free()
    for sim in runs.values():
        sim.free()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--paper", action="store_true",
                    help="Sec. 3 setup: sech^2 jet, DNS 2048^2 (nu = 2e-3) to 1.56M steps, coarse "
                         "1024^2 runs with Delta = 2, 1, 0 to 780k steps")
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--r", type=int, default=2)
    ap.add_argument("--nu-dns", type=float, default=2e-3)
    ap.add_argument("--fine-steps", type=int, default=40000)
    ap.add_argument("--checkpoints", type=int, default=4)
    ap.add_argument("--deltas", type=str, default="2,1,0")
    ap.add_argument("--precision", choices=["fp64", "fp32", "fp16"], default="fp32")
    ap.add_argument("--ic", choices=["kh", "sech2"], default="sech2")
    ap.add_argument("--no-spectra", action="store_true")
    a = ap.parse_args()
    prec = {"fp64": lbmhd.LBMHD_FP64, "fp32": lbmhd.LBMHD_FP32, "fp16": lbmhd.LBMHD_FP16}[a.precision]
    if a.paper:
        res = run_experiment(2048, 2, 2e-3, 1_560_000, (200_000, 400_000, 800_000, 1_200_000, 1_560_000),
                             (2.0, 1.0, 0.0), prec, "sech2", keep_spectra=not a.no_spectra)
    else:
        cps = tuple(a.fine_steps * (i + 1) // a.checkpoints for i in range(a.checkpoints))
        res = run_experiment(a.n, a.r, a.nu_dns, a.fine_steps, cps,
                             tuple(float(d) for d in a.deltas.split(",")), prec, a.ic,
                             keep_spectra=not a.no_spectra)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
