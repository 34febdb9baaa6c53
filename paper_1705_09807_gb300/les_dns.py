"""LES-vs-DNS comparison (the paper's Sec. 3 experiment, on synthetic initial conditions).

A DNS (Delta = 0) runs on an n x n grid; an LES (Delta = r, the filter width of the coarse grid)
and an unfiltered coarse run (Delta = 0) start from the r x r box-filtered DNS initial fields on
the (n/r)^2 grid.  Both grids keep the Reynolds number: the lattice viscosity scales with the
grid, nu_coarse = nu_dns / r, and one coarse step matches r DNS steps (Sec. 3: halving the grid
halves the number of steps).  At the checkpoints the DNS moments are box-filtered onto the
coarse grid and the shell-summed kinetic and magnetic energy spectra of filtered DNS, LES and
the unfiltered coarse run are compared.  Every field operation (steps, moments, box filter,
spectra) runs in the library's CUDA kernels; this module only sequences the calls and reduces
the returned spectra to a few numbers.

    python -m paper_1705_09807_gb300.les_dns --n 2048 --r 8 --dns-steps 20000
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import lbmhd
from .inputs import kh_jet, sech2_jet


def _spectrum_of_fields(dev, nbins, work):
    import torch
    ek = torch.empty(nbins, dtype=torch.float64, device="cuda")
    em = torch.empty(nbins, dtype=torch.float64, device="cuda")
    lbmhd.lbmhd_energy_spectrum_device(dev[1], dev[2], dev[3], dev[4], nbins, ek, em, work)
    torch.cuda.synchronize()
    return ek.cpu().numpy(), em.cpu().numpy()


def spectral_error(a, b, kmax):
    """Relative L2 distance of two spectra over shells 1..kmax (b is the reference)."""
    sa, sb = a[1:kmax + 1], b[1:kmax + 1]
    return float(np.linalg.norm(sa - sb) / np.linalg.norm(sb))


def run_pair(n=2048, r=8, nu_dns=8e-3, dns_steps=20000, checkpoints=4, precision=lbmhd.LBMHD_FP32,
             ic="kh", seed=1, delta_les=None):
    import torch
    m = n // r
    nu_c = nu_dns / r
    delta_les = float(r) if delta_les is None else delta_les
    fields = kh_jet(n, seed=seed) if ic == "kh" else sech2_jet(n)
    dns = lbmhd.Lbmhd(lbmhd.lbmhd_params_srt(n, n, nu_dns, nu_dns, 0.0, precision), *fields)
    # coarse initial fields: box filter of the DNS initial fields, on the GPU
    fine = [torch.tensor(a, device="cuda") for a in fields]
    coarse = [torch.empty((m, m), dtype=torch.float64, device="cuda") for _ in range(5)]
    for a, b in zip(fine, coarse):
        lbmhd.lbmhd_block_mean_device(a, r, b)
    torch.cuda.synchronize()
    les = lbmhd.Lbmhd(lbmhd.lbmhd_params_srt(m, m, nu_c, nu_c, delta_les, precision), *coarse,
                      device=True)
    raw = lbmhd.Lbmhd(lbmhd.lbmhd_params_srt(m, m, nu_c, nu_c, 0.0, precision), *coarse, device=True)
    nbins = m // 2 + 1
    kmax = m // 2 - 1
    work = torch.empty(lbmhd.lbmhd_energy_spectrum_work_bytes(m), dtype=torch.uint8, device="cuda")
    fine_mom = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(5)]
    out = {"n_dns": n, "r": r, "n_les": m, "nu_dns": nu_dns, "nu_les": nu_c, "delta_les": delta_les,
           "precision": precision, "ic": ic, "checkpoints": []}
    per = dns_steps // checkpoints // r * r
    t0 = time.perf_counter()
    for c in range(1, checkpoints + 1):
        dns.step(per)
        les.step(per // r)
        raw.step(per // r)
        dns.moments_device(fine_mom)
        torch.cuda.synchronize()
        for a, b in zip(fine_mom, coarse):
            lbmhd.lbmhd_block_mean_device(a, r, b)
        ek_f, em_f = _spectrum_of_fields(coarse, nbins, work)
        ek_l, em_l = les.spectrum(nbins)
        ek_r, em_r = raw.spectrum(nbins)
        tot_f, tot_l, tot_r = ek_f + em_f, ek_l + em_l, ek_r + em_r
        out["checkpoints"].append({
            "dns_step": c * per, "les_step": c * per // r,
            "err_total_les": spectral_error(tot_l, tot_f, kmax),
            "err_total_unfiltered": spectral_error(tot_r, tot_f, kmax),
            "err_kin_les": spectral_error(ek_l, ek_f, kmax),
            "err_kin_unfiltered": spectral_error(ek_r, ek_f, kmax),
            "err_mag_les": spectral_error(em_l, em_f, kmax),
            "err_mag_unfiltered": spectral_error(em_r, em_f, kmax),
            "energy_filtered_dns": float(tot_f.sum()), "energy_les": float(tot_l.sum()),
            "energy_unfiltered": float(tot_r.sum()),
        })
    out["seconds"] = round(time.perf_counter() - t0, 3)
    for sim in (dns, les, raw):
        sim.free()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--r", type=int, default=8)
    ap.add_argument("--nu-dns", type=float, default=8e-3)
    ap.add_argument("--dns-steps", type=int, default=20000)
    ap.add_argument("--checkpoints", type=int, default=4)
    ap.add_argument("--precision", choices=["fp64", "fp32", "fp16"], default="fp32")
    ap.add_argument("--ic", choices=["kh", "sech2"], default="kh")
    ap.add_argument("--delta-les", type=float, default=None)
    a = ap.parse_args()
    prec = {"fp64": lbmhd.LBMHD_FP64, "fp32": lbmhd.LBMHD_FP32, "fp16": lbmhd.LBMHD_FP16}[a.precision]
    print(json.dumps(run_pair(a.n, a.r, a.nu_dns, a.dns_steps, a.checkpoints, prec, a.ic,
                              delta_les=a.delta_les)))


if __name__ == "__main__":
    main()
