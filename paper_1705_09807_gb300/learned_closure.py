"""Training and evaluation of the learned subgrid correction (the closure network of the C ABI).

Data: DNS runs of seeded magnetized Kelvin-Helmholtz jets (U0 in [0.03, 0.07], B0 in [0, 0.05])
on an n x n grid; at each snapshot the fine moments are box-filtered by r and turned into a
training pair on the (n/r)^2 grid: features of the filtered state and the residual of the exact
filtered subgrid terms against the analytic closure with filter width Delta (coarse units).
Training: Adam on mean squared error with the library's binary32 kernels.  Evaluation: a
priori, the error of the subgrid terms on held-out runs with the analytic closure alone and with
the network added; a posteriori, LES runs on the coarse grid with and without the network
against the filtered DNS (total-energy spectra).  All field work runs in the library's CUDA
kernels; this module sequences calls, keeps the tensors and reduces a few statistics.

    python -m paper_1705_09807_gb300.learned_closure            # 2048^2 -> 256^2 (x8)
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import lbmhd
from .inputs import kh_jet, splitmix64_uniform


def run_params(seed):
    u = splitmix64_uniform(1000 + seed, 2)
    return 0.03 + 0.04 * u[0], 0.05 * u[1]


def generate_pairs(n, r, seeds, snapshots, nu_dns, delta, scales=None, precision=lbmhd.LBMHD_FP32):
    """Features X [N, 12, m, m] and targets T [N, 4, m, m] (CUDA float32) from DNS snapshots.
    With scales=None the pairs are unscaled (unit scales)."""
    import torch
    m = n // r
    in_s, out_s = (np.ones(12, np.float32), np.ones(4, np.float32)) if scales is None else scales
    cl = lbmhd.Closure(np.zeros(lbmhd.load_library().lbmhd_closure_num_params(), np.float32), in_s, out_s)
    X = torch.empty((len(seeds) * len(snapshots), 12, m, m), dtype=torch.float32, device="cuda")
    T = torch.empty((len(seeds) * len(snapshots), 4, m, m), dtype=torch.float32, device="cuda")
    fine = torch.empty((5, n, n), dtype=torch.float64, device="cuda")
    work = torch.empty(9 * m * m, dtype=torch.float64, device="cuda")
    i = 0
    for seed in seeds:
        u0, b0 = run_params(seed)
        p = lbmhd.lbmhd_params_srt(n, n, nu_dns, nu_dns, 0.0, precision)
        with lbmhd.Lbmhd(p, *kh_jet(n, u0=u0, b0=b0, seed=seed)) as dns:
            done = 0
            for t in snapshots:
                dns.step(t - done)
                done = t
                dns.moments_device([fine[k] for k in range(5)])
                torch.cuda.synchronize()
                cl.training_pair(fine, r, delta, X[i], T[i], work)
                i += 1
    cl.free()
    return X, T


def channel_scales(X, T):
    """Per-channel root-mean-square of features and targets (host statistics)."""
    xs = np.sqrt((X.double() ** 2).mean(dim=(0, 2, 3)).cpu().numpy()).astype(np.float32)
    ts = np.sqrt((T.double() ** 2).mean(dim=(0, 2, 3)).cpu().numpy()).astype(np.float32)
    return np.maximum(xs, 1e-12), np.maximum(ts, 1e-20)


def train(closure, X, T, iters=2000, batch=8, lr=1e-3, seed=0, log_every=0):
    """Adam on random mini-batches of snapshots; returns the loss history."""
    import torch
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    hist = []
    for it in range(iters):
        idx = torch.as_tensor(rng.choice(n, size=min(batch, n), replace=False), device="cuda")
        xb = X.index_select(0, idx).contiguous()
        tb = T.index_select(0, idx).contiguous()
        step_lr = lr * (0.1 ** (it / max(iters, 1)))  # exponential decay to lr/10
        hist.append(closure.train_step(xb, tb, step_lr))
        if log_every and it % log_every == 0:
            print(f"iter {it} loss {hist[-1]:.4e}", flush=True)
    return hist


def a_priori(closure, X, T):
    """Relative RMS error of the four subgrid terms on (X, T): analytic closure alone (= |T|) and
    analytic + network (|T - net(X)|), per channel."""
    import torch
    out = torch.empty_like(T)
    closure.forward(X, out, tensor_cores=True)
    t = T.double()
    e_an = torch.sqrt((t ** 2).mean(dim=(0, 2, 3)))
    e_nn = torch.sqrt(((t - out.double()) ** 2).mean(dim=(0, 2, 3)))
    return {"analytic": e_an.cpu().numpy().tolist(), "analytic_plus_network": e_nn.cpu().numpy().tolist(),
            "ratio": (e_nn / e_an).cpu().numpy().tolist()}


def a_posteriori(closure, n, r, seed, nu_dns, delta, checkpoints, precision=lbmhd.LBMHD_FP32):
    """LES on the coarse grid from the box-filtered DNS initial fields, with the analytic closure
    alone and with the network attached, against the filtered DNS: relative L2 of total-energy
    spectra (shells 1 .. m/2 - 1) at the DNS checkpoints (coarse step = DNS step / r)."""
    import torch
    m = n // r
    u0, b0 = run_params(seed)
    fields = kh_jet(n, u0=u0, b0=b0, seed=seed)
    fine = [torch.tensor(a, device="cuda") for a in fields]
    coarse = [torch.empty((m, m), dtype=torch.float64, device="cuda") for _ in range(5)]
    for a, b in zip(fine, coarse):
        lbmhd.lbmhd_block_mean_device(a, r, b)
    torch.cuda.synchronize()
    del fine
    nu_c = nu_dns / r
    dns = lbmhd.Lbmhd(lbmhd.lbmhd_params_srt(n, n, nu_dns, nu_dns, 0.0, precision), *fields)
    les = lbmhd.Lbmhd(lbmhd.lbmhd_params_srt(m, m, nu_c, nu_c, delta, precision), *coarse, device=True)
    net = lbmhd.Lbmhd(lbmhd.lbmhd_params_srt(m, m, nu_c, nu_c, delta, precision), *coarse, device=True)
    closure.attach(net.h)
    nb = m // 2 + 1
    work = torch.empty(lbmhd.lbmhd_energy_spectrum_work_bytes(m), dtype=torch.uint8, device="cuda")
    ek = torch.empty(nb, dtype=torch.float64, device="cuda")
    em = torch.empty(nb, dtype=torch.float64, device="cuda")
    fm = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(5)]
    out = []
    done = 0
    for cp in checkpoints:
        steps = (cp - done) // r * r
        dns.step(steps)
        les.step(steps // r)
        net.step(steps // r)
        done += steps
        dns.moments_device(fm)
        torch.cuda.synchronize()
        for a, b in zip(fm, coarse):
            lbmhd.lbmhd_block_mean_device(a, r, b)
        lbmhd.lbmhd_energy_spectrum_device(coarse[1], coarse[2], coarse[3], coarse[4], nb, ek, em, work)
        torch.cuda.synchronize()
        ref = (ek + em).cpu().numpy()
        rec = {"dns_step": done}
        for name, sim in (("analytic", les), ("analytic_plus_network", net)):
            k_, m_ = sim.spectrum(nb)
            tot = k_ + m_
            sl = slice(1, m // 2)
            rec[name] = float(np.linalg.norm(tot[sl] - ref[sl]) / np.linalg.norm(ref[sl]))
        out.append(rec)
    lbmhd.lbmhd_detach_closure(net.h)
    for sim in (dns, les, net):
        sim.free()
    return out


def run(n=2048, r=8, nu_dns=8e-3, delta=2.0, train_seeds=range(8), test_seed=100,
        snapshots=tuple(range(2000, 20001, 2000)), iters=3000, batch=8, lr=1e-3, seed=0):
    import torch
    from .inputs import splitmix64_uniform as su
    t0 = time.perf_counter()
    X, T = generate_pairs(n, r, list(train_seeds), list(snapshots), nu_dns, delta)
    in_s, out_s = channel_scales(X, T)
    X /= torch.tensor(in_s, device="cuda")[None, :, None, None]
    T /= torch.tensor(out_s, device="cuda")[None, :, None, None]
    Xt, Tt = generate_pairs(n, r, [test_seed], list(snapshots), nu_dns, delta, scales=(in_s, out_s))
    t_data = time.perf_counter() - t0
    # initial weights: uniform(+-1/sqrt(fan_in)), zero biases, from splitmix64 numbers
    nparams = lbmhd.load_library().lbmhd_closure_num_params()
    u = su(seed + 77, nparams)
    theta = np.zeros(nparams, np.float32)
    o = 0
    for ci, co in ((12, 32), (32, 32), (32, 4)):
        lim = 1.0 / np.sqrt(ci * 9)
        theta[o:o + co * ci * 9] = (2 * u[o:o + co * ci * 9] - 1) * lim
        o += co * ci * 9 + co
    cl = lbmhd.Closure(theta, in_s, out_s)
    prior_before = a_priori(cl, Xt, Tt)
    t1 = time.perf_counter()
    hist = train(cl, X, T, iters=iters, batch=batch, lr=lr, seed=seed)
    t_train = time.perf_counter() - t1
    res = {"n_dns": n, "r": r, "n_les": n // r, "nu_dns": nu_dns, "delta": delta,
           "train_seeds": list(train_seeds), "test_seed": test_seed, "snapshots": list(snapshots),
           "pairs": int(X.shape[0]), "iters": iters, "batch": batch, "lr": lr,
           "seconds_data": round(t_data, 2), "seconds_train": round(t_train, 2),
           "loss_first": hist[0], "loss_last": float(np.mean(hist[-50:])),
           "in_scale": in_s.tolist(), "out_scale": out_s.tolist(),
           "a_priori_untrained": prior_before,
           "a_priori_train": a_priori(cl, X[:16], T[:16]),
           "a_priori_test": a_priori(cl, Xt, Tt)}
    res["a_posteriori_test"] = a_posteriori(cl, n, r, test_seed, nu_dns, delta, list(snapshots)[1::3])
    res["params"] = cl.params().tolist()
    cl.free()
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--r", type=int, default=8)
    ap.add_argument("--nu-dns", type=float, default=8e-3)
    ap.add_argument("--delta", type=float, default=2.0)
    ap.add_argument("--train-seeds", type=int, default=8)
    ap.add_argument("--snapshots", type=int, default=10)
    ap.add_argument("--every", type=int, default=2000)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--no-params", action="store_true")
    a = ap.parse_args()
    res = run(a.n, a.r, a.nu_dns, a.delta, range(a.train_seeds), 100,
              tuple(a.every * (i + 1) for i in range(a.snapshots)), a.iters, a.batch, a.lr)
    if a.no_params:
        res.pop("params")
    print(json.dumps(res))


if __name__ == "__main__":
    main()
