"""Train the warm-start network on iterates the method itself generates.

Runs small plain workloads (L = 4 pi, by default M = 128 cells and 2e5 markers,
cubic splines, dt = 0.05) with pump amplitudes 0.05..0.3 and thermal speeds
0.05..0.15 through libpic, and
records, for every marker and step, the features at x^n (cell-relative x, p,
E_x, A_y, A_z, dt) and the converged subsystem-I update, as the residuals of the
explicit predictor scaled by 1/dt^2:
    y0 = (x^{n+1} - x^n - dt p / gamma(p, A(x^n))) / dt^2,
    y1 = (p^{n+1} - p^n - dt E_x(x^n)) / dt^2.
Training uses the library's own fp32 forward/backward kernels and Adam
(pic_mlp_train_step).  Output: an .npz with params (8898 float32) and norm (14).

    python -m paper_2203_06513_gb300.train_warm [out.npz] [--nx 128] [--np 200000]
"""
from __future__ import annotations

import math
import os
import sys
import time

import numpy as np

from . import inputs as I
from . import pic

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "data", "warm_mlp.npz")


def collect(torch, pumps=(0.05, 0.1, 0.2, 0.3), vths=(0.05, 0.1, 0.15), steps=12, np_run=200000,
            seeds=(0, 1), nx=128):
    X, Y = [], []
    for pump in pumps:
        for vth in vths:
            for seed in seeds:
                w = I.Workload("train", nx=nx, degree=3, np=np_run, dt=0.05, vth=vth, pump=pump,
                               seed=100 + seed)
                x, p = I.particles(w)
                ay, az, ey, ez = I.fields(w)
                g = pic.Pic(pic.Config.from_workload(w, precision=pic.PIC_FP64), x, p, ay, az, ey, ez)
                ex_d = torch.empty(w.np, dtype=torch.float64, device="cuda")
                ay_d = torch.empty_like(ex_d)
                az_d = torch.empty_like(ex_d)
                for _ in range(steps):
                    st0 = g.state_numpy()
                    g.gather(pic.PIC_FIELD_EX, ex_d)
                    g.gather(pic.PIC_FIELD_AY, ay_d)
                    g.gather(pic.PIC_FIELD_AZ, az_d)
                    Ex, Ay, Az = ex_d.cpu().numpy(), ay_d.cpu().numpy(), az_d.cpu().numpy()
                    g.substep(pic.PIC_SUBSYSTEM_I)
                    st1 = g.state_numpy()
                    g.substep(pic.PIC_SUBSYSTEM_II)
                    x0, p0 = st0["x"], st0["p"]
                    dxp = np.mod(st1["x"] - x0 + 0.5 * w.L, w.L) - 0.5 * w.L
                    g0 = np.sqrt(1.0 + p0 ** 2 + Ay ** 2 + Az ** 2)
                    u = x0 / w.dx
                    feat = np.column_stack([u - np.floor(u), p0, Ex, Ay, Az, np.full(w.np, w.dt)])
                    tgt = np.column_stack([(dxp - w.dt * p0 / g0) / w.dt ** 2,
                                           (st1["p"] - p0 - w.dt * Ex) / w.dt ** 2])
                    X.append(feat)
                    Y.append(tgt)
                g.close()
    return np.concatenate(X).astype(np.float32), np.concatenate(Y).astype(np.float32)


def normalisation(X, Y):
    shift = X.mean(axis=0)
    sd = X.std(axis=0)
    scale = np.where(sd > 0, 1.0 / np.maximum(sd, 1e-30), 1.0)
    out_scale = Y.std(axis=0)
    out_scale = np.where(out_scale > 0, out_scale, 1.0)
    return np.concatenate([shift, scale, out_scale]).astype(np.float32)


def init_params(seed=0):
    """He-style initial weights (small output layer), packed as the library expects."""
    rng = np.random.default_rng(seed)
    sizes = [(64, 6), (64, 64), (64, 64), (2, 64)]
    parts = []
    for li, (o, i) in enumerate(sizes):
        s = math.sqrt(2.0 / i) * (0.1 if li == len(sizes) - 1 else 1.0)
        parts += [rng.normal(0.0, s, o * i), np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)


def fit(torch, X, Y, norm, epochs=30, batch=4096, lr=2e-3, seed=0, log=print):
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    perm = rng.permutation(n)
    nval = max(1, n // 20)
    val, tr = perm[:nval], perm[nval:]
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    m = pic.Mlp(norm, init_params(seed))
    Xv, Yv = Xd[torch.from_numpy(val).cuda()], Yd[torch.from_numpy(val).cuda()]
    base = m.grad(Xv, Yv)
    t0 = time.time()
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(tr)).cuda()
        lr_ep = lr * 0.5 * (1.0 + math.cos(math.pi * ep / epochs))
        for s in range(0, order.numel() - batch + 1, batch):
            idx = order[s:s + batch]
            m.train_step(Xd[idx].contiguous(), Yd[idx].contiguous(), lr_ep)
        if ep % 5 == 4 or ep == epochs - 1:
            log(f"epoch {ep + 1}: validation loss {m.grad(Xv, Yv):.4e} (initial {base:.4e}), "
                f"{time.time() - t0:.1f} s")
    return m, m.grad(Xv, Yv), base


def main(argv=None):
    import argparse
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("out", nargs="?", default=DEFAULT_OUT)
    ap.add_argument("--nx", type=int, default=128, help="cells of the training runs")
    ap.add_argument("--np", type=int, default=200000, help="markers of each training run")
    args = ap.parse_args(sys.argv[1:] if argv is None else argv)
    out = args.out
    t = time.time()
    X, Y = collect(torch, nx=args.nx, np_run=args.np)
    print(f"collected {X.shape[0]} samples in {time.time() - t:.1f} s", flush=True)
    norm = normalisation(X, Y)
    m, vloss, base = fit(torch, X, Y, norm)
    os.makedirs(os.path.dirname(os.path.abspath(out)), exist_ok=True)
    np.savez(out, params=m.params(), norm=norm, val_loss=vloss, val_loss_initial=base,
             samples=X.shape[0])
    print(f"saved {out}: validation loss {vloss:.4e} (initial {base:.4e})", flush=True)


if __name__ == "__main__":
    main()
