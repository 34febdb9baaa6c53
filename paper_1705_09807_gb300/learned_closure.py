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
    python -m paper_1705_09807_gb300.learned_closure --paper    # the paper's 2048^2 / 1024^2 run
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
    alone, with the network attached and with no closure at all (Delta = 0, the unfiltered
    coarse run), against the filtered DNS: relative L2 of total-energy spectra (shells
    1 .. m/2 - 1) at the DNS checkpoints (coarse step = DNS step / r)."""
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
    bare = lbmhd.Lbmhd(lbmhd.lbmhd_params_srt(m, m, nu_c, nu_c, 0.0, precision), *coarse, device=True)
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
        bare.step(steps // r)
        done += steps
        dns.moments_device(fm)
        torch.cuda.synchronize()
        for a, b in zip(fm, coarse):
            lbmhd.lbmhd_block_mean_device(a, r, b)
        lbmhd.lbmhd_energy_spectrum_device(coarse[1], coarse[2], coarse[3], coarse[4], nb, ek, em, work)
        torch.cuda.synchronize()
        ref = (ek + em).cpu().numpy()
        rec = {"dns_step": done}
        for name, sim in (("analytic", les), ("analytic_plus_network", net), ("no_closure", bare)):
            k_, m_ = sim.spectrum(nb)
            tot = k_ + m_
            sl = slice(1, m // 2)
            rec[name] = float(np.linalg.norm(tot[sl] - ref[sl]) / np.linalg.norm(ref[sl]))
        out.append(rec)
    lbmhd.lbmhd_detach_closure(net.h)
    for sim in (dns, les, net, bare):
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


def random_crops(X, T, batch, crop, rng):
    """`batch` random crop x crop windows (same window in X and T) of random snapshots."""
    n = X.shape[0]
    h, w = X.shape[2], X.shape[3]
    xs, ts = [], []
    for _ in range(batch):
        i = int(rng.integers(n))
        y0, x0 = int(rng.integers(h - crop + 1)), int(rng.integers(w - crop + 1))
        xs.append(X[i, :, y0:y0 + crop, x0:x0 + crop])
        ts.append(T[i, :, y0:y0 + crop, x0:x0 + crop])
    import torch
    return torch.stack(xs).contiguous(), torch.stack(ts).contiguous()


def paper_study(n=2048, r=2, nu_dns=2e-3, delta=2.0, train_until=400_000, every=25_000,
                checkpoints=(200_000, 400_000, 800_000, 1_560_000), iters=3000, batch=8, crop=256,
                lr=1e-3, seed=0, precision=lbmhd.LBMHD_FP32):
    """The learned closure in the paper's own setup (Sec. 3 jet, DNS n^2 against LES (n/r)^2 with
    filter width `delta`): training pairs from the DNS every `every` steps up to `train_until`,
    Adam on random crop x crop windows, then coarse runs from the box-filtered initial fields --
    the analytic closure alone, the analytic closure plus the network, and no closure -- compared
    with the filtered DNS (total-energy spectra) at the checkpoints, most of them after the
    training window."""
    import torch
    from .inputs import sech2_jet
    from .les_dns import fitted_slope, spectral_errors
    t0 = time.perf_counter()
    m = n // r
    nu_c = nu_dns / r
    fields = sech2_jet(n)
    dns = lbmhd.Lbmhd(lbmhd.lbmhd_params_srt(n, n, nu_dns, nu_dns, 0.0, precision), *fields)
    fine = [torch.tensor(a, device="cuda") for a in fields]
    coarse0 = [torch.empty((m, m), dtype=torch.float64, device="cuda") for _ in range(5)]
    for a, b in zip(fine, coarse0):
        lbmhd.lbmhd_block_mean_device(a, r, b)
    del fine
    nb = m // 2 + 1
    kmax = m // 2 - 1
    k1, k2 = max(2, m // 128), max(8, m // 8)
    work_s = torch.empty(lbmhd.lbmhd_energy_spectrum_work_bytes(m), dtype=torch.uint8, device="cuda")
    ek = torch.empty(nb, dtype=torch.float64, device="cuda")
    em = torch.empty(nb, dtype=torch.float64, device="cuda")
    fm = torch.empty((5, n, n), dtype=torch.float64, device="cuda")
    cm = [torch.empty((m, m), dtype=torch.float64, device="cuda") for _ in range(5)]

    def filtered_dns_spectrum():
        dns.moments_device([fm[k] for k in range(5)])
        torch.cuda.synchronize()
        for k in range(5):
            lbmhd.lbmhd_block_mean_device(fm[k], r, cm[k])
        lbmhd.lbmhd_energy_spectrum_device(cm[1], cm[2], cm[3], cm[4], nb, ek, em, work_s)
        torch.cuda.synchronize()
        return ek.cpu().numpy() + em.cpu().numpy()

    # 1. training pairs (unscaled) from the DNS up to train_until; reference spectra on the way
    snaps = list(range(every, train_until + 1, every))
    X = torch.empty((len(snaps), 12, m, m), dtype=torch.float32, device="cuda")
    T = torch.empty((len(snaps), 4, m, m), dtype=torch.float32, device="cuda")
    work = torch.empty(9 * m * m, dtype=torch.float64, device="cuda")
    nparams = lbmhd.load_library().lbmhd_closure_num_params()
    unit = lbmhd.Closure(np.zeros(nparams, np.float32), np.ones(12, np.float32), np.ones(4, np.float32))
    ref = {}
    done = 0
    for i, t in enumerate(snaps):
        dns.step(t - done)
        done = t
        if t in checkpoints:
            ref[t] = filtered_dns_spectrum()
        dns.moments_device([fm[k] for k in range(5)])
        torch.cuda.synchronize()
        unit.training_pair(fm, r, delta, X[i], T[i], work)
    unit.free()
    t_data = time.perf_counter() - t0
    in_s, out_s = channel_scales(X, T)
    X /= torch.tensor(in_s, device="cuda")[None, :, None, None]
    T /= torch.tensor(out_s, device="cuda")[None, :, None, None]
    # 2. training on random windows
    from .inputs import splitmix64_uniform as su
    u = su(seed + 77, nparams)
    theta = np.zeros(nparams, np.float32)
    o = 0
    for ci, co in ((12, 32), (32, 32), (32, 4)):
        lim = 1.0 / np.sqrt(ci * 9)
        theta[o:o + co * ci * 9] = (2 * u[o:o + co * ci * 9] - 1) * lim
        o += co * ci * 9 + co
    cl = lbmhd.Closure(theta, in_s, out_s)
    rng = np.random.default_rng(seed)
    t1 = time.perf_counter()
    hist = []
    for it in range(iters):
        xb, tb = random_crops(X, T, batch, crop, rng)
        hist.append(cl.train_step(xb, tb, lr * (0.1 ** (it / max(iters, 1)))))
    t_train = time.perf_counter() - t1
    prior = a_priori(cl, X[-4:], T[-4:])
    del X, T, work
    # 3. coarse runs from the filtered initial fields
    mk = lambda d: lbmhd.Lbmhd(lbmhd.lbmhd_params_srt(m, m, nu_c, nu_c, d, precision), *coarse0, device=True)
    runs = {"analytic": mk(delta), "analytic_plus_network": mk(delta), "no_closure": mk(0.0)}
    cl.attach(runs["analytic_plus_network"].h)
    out = {"n_dns": n, "r": r, "n_les": m, "nu_dns": nu_dns, "nu_les": nu_c, "delta": delta,
           "train_until": train_until, "snapshots": len(snaps), "iters": iters, "batch": batch,
           "crop": crop, "lr": lr, "seconds_data": round(t_data, 1), "seconds_train": round(t_train, 1),
           "loss_first": hist[0], "loss_last": float(np.mean(hist[-50:])), "in_scale": in_s.tolist(),
           "out_scale": out_s.tolist(), "a_priori_last_snapshots": prior, "slope_range": [k1, k2],
           "checkpoints": []}
    cdone = 0
    t2 = time.perf_counter()
    for cp in checkpoints:
        if cp > done:
            dns.step(cp - done)
            done = cp
            ref[cp] = filtered_dns_spectrum()
        for sim in runs.values():
            sim.step(cp // r - cdone)
        cdone = cp // r
        rec = {"dns_step": cp, "after_training_window": cp > train_until,
               "filtered_dns": {"energy": float(ref[cp].sum()), "slope": fitted_slope(ref[cp], k1, k2)}}
        for name, sim in runs.items():
            k_, m_ = sim.spectrum(nb)
            tot = k_ + m_
            rel, logrms = spectral_errors(tot, ref[cp], kmax)
            rec[name] = {"energy": float(tot.sum()), "slope": fitted_slope(tot, k1, k2),
                         "rel_l2_vs_filtered_dns": rel, "log10_rms_vs_filtered_dns": logrms}
        out["checkpoints"].append(rec)
    out["seconds_runs"] = round(time.perf_counter() - t2, 1)
    lbmhd.lbmhd_detach_closure(runs["analytic_plus_network"].h)
    for sim in runs.values():
        sim.free()
    dns.free()
    cl.free()
    return out


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
    ap.add_argument("--paper", action="store_true",
                    help="the paper's setup: Sec. 3 jet, DNS 2048^2 to 1.56M steps, LES 1024^2, "
                         "trained on the DNS up to 400k steps")
    a = ap.parse_args()
    if a.paper:
        print(json.dumps(paper_study()))
        return
    res = run(a.n, a.r, a.nu_dns, a.delta, range(a.train_seeds), 100,
              tuple(a.every * (i + 1) for i in range(a.snapshots)), a.iters, a.batch, a.lr)
    if a.no_params:
        res.pop("params")
    print(json.dumps(res))


if __name__ == "__main__":
    main()
