"""Benchmark: particle-steps/s of the energy-conserving PIC step on one GB300.

Workload: L = 4 pi, M = 2048 cells, cubic splines, N_p = 1e8 markers, density
1 + 0.01 cos(0.5 x), Maxwellian p with v_th = 0.1, pump A_y = 0.2 cos(2x),
dt = 0.05.  Forms measured on the same seeded markers:
  * FP32 + learned warm start (the headline): float marker state and arithmetic,
    double deposits / solves / convergence / energy, network proposals for the
    subsystem-I fixed point (weights trained by train_warm.py, shipped in
    paper_2203_06513_gb300/data/warm_mlp.npz);
  * FP32 + explicit predictor x^(0) = x^n + dt p / gamma;
  * plain FP64 (all double, no warm start).
A step is one full Lie--Trotter step (subsystem I then II, all fixed-point
sweeps).  Markers (>= 2.4 GB) exceed the 129 MB L2: no flush between steps.
Besides the timed steps the line reports the energy and Gauss-law drift of the
two FP32 forms over the workload's 1,000 steps, the Gauss residual of the three
deposit accumulations of the FP32 form, and the batched-ensemble workload.  The
energy and convergence figures come last in the line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank advances an
independent replica (seed + rank): weak scaling, no collective on the data path.
"""
from __future__ import annotations

import os

# the oracle's grid algebra runs single-threaded (BLAS included); its marker loops
# run on one thread or, for the all-core figure, on slices in parallel threads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2203_06513_gb300 import inputs as I  # noqa: E402
from paper_2203_06513_gb300 import replicas as R  # noqa: E402

METRIC = "particle-steps/s at rel. energy err ≤1e-10: FP32+learned vs plain FP64"
UNIT = "particle-steps/s"
WORKLOAD = "C2"
WEIGHTS = os.path.join(ROOT, "paper_2203_06513_gb300", "data", "warm_mlp.npz")
# Roofline units of the hot kernels (float form, one marker), as the method must
# move them (a Picard sweep re-reads every marker because e_x couples them all):
#   k_sweep1: read x^n (cell + offset, 8 B), p^n (4 B), x^(k) (8 B); write
#             x^(k+1) (8 B): 28 B (the kernel stores x^(k) as a 4-byte
#             displacement and writes p^(k+1) every sweep: 24 B moved)
#   k_sweep2: read cell, offset, p: 12 B
#   k_warm_mlp: 2 x (6x64 + 64x64 + 64x64 + 64x2) = 17,408 flop (bf16 tensor cores)
BYTES_SWEEP1 = {1: 28, 0: 44}
BYTES_SWEEP2 = 12
FLOP_MLP = 2 * (6 * 64 + 64 * 64 + 64 * 64 + 64 * 2)
# DRAM bytes (read + write) per marker from ncu captures of the current kernels on
# 2e7 markers of the C2 grid (--set full, one launch each; the sweeps with their
# default compensated deposit lanes); per launch = x N_p.
NCU_DRAM_PER_MARKER = {"k_sweep1<3,float>": 22.35, "k_sweep2<3,float>": 12.29, "k_warm_mlp<3,float>": 15.02}
# Warp instructions x 32 per marker from the same captures: the kernels are bound by
# instruction issue, which the "issue" entry compares with the issue-slot peak
# (SMs x 4 schedulers x 1 warp instruction a cycle x the sampled SM clock).
NCU_INST_PER_MARKER = {"k_sweep1<3,float>": 577, "k_sweep2<3,float>": 359, "k_warm_mlp<3,float>": 602}


def peaks():
    """(HBM GB/s, bf16 TFLOP/s sustained, kind): measured on this machine, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured"
    except Exception:
        return 6800.0, 1700.0, "fallback"


def kernel_rooflines(tr, np_, hbm, tflops, kind, sms=None, sm_mhz=None):
    """Per hot kernel of the timed form: achieved against its roof, from the library's
    CUDA-event timing of each launch."""
    out = []
    for name, ms, n, unit_amount, bound in (
            ("k_sweep1<3,float>", tr["sweep1_ms"], tr["sweep1_launches"], BYTES_SWEEP1[1], "hbm"),
            ("k_sweep2<3,float>", tr["sweep2_ms"], tr["sweep2_launches"], BYTES_SWEEP2, "hbm"),
            ("k_warm_mlp<3,float>", tr["warm_ms"], tr["warm_launches"], FLOP_MLP, "tensor")):
        if n <= 0:
            continue
        launch_ms = ms / n
        if bound == "hbm":
            achieved = unit_amount * np_ / (launch_ms / 1e3) / 1e9
            peak, unit = hbm, "GB/s"
        else:
            achieved = unit_amount * np_ / (launch_ms / 1e3) / 1e12
            peak, unit = tflops, "TFLOP/s"
        per_marker = NCU_DRAM_PER_MARKER.get(name)
        entry = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                 "frac": achieved / peak, "peak_kind": kind,
                 "traffic": None if per_marker is None else per_marker * np_,
                 "algorithmic_per_launch": unit_amount * np_, "launch_ms": launch_ms,
                 "launches": n, "share_ms": ms}
        inst = NCU_INST_PER_MARKER.get(name)
        if inst and sms and sm_mhz:
            got = inst / 32.0 * np_ / (launch_ms / 1e3) / 1e9
            top = sms * 4 * sm_mhz / 1e3
            entry["issue"] = {"inst_per_marker": inst, "achieved": got, "peak": top, "unit": "G warp-inst/s",
                              "frac": got / top}
        out.append(entry)
    return out


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_form(pic, torch, w, arrays, precision, warm, steps, warmup, stream, mlp=None, deposit=0,
             kernel_steps=5, split_run=None, warm_field=None):
    """Advance one replica (or, with split_run = (reducer, local count), this rank's
    share of one plasma) from host arrays; CUDA-event timing of `steps` steps.  With a
    warm start the field starts from the proposal's (warm_field) unless told otherwise."""
    x, p, ay, az, ey, ez = arrays
    if warm_field is None:
        warm_field = 1 if warm != pic.PIC_WARM_NONE else 0
    cfg = pic.Config.from_workload(w, precision=precision, warm_start=warm, sort_every=2, deposit=deposit,
                                   warm_field=warm_field)
    reducer = None
    if split_run is not None:
        reducer, cfg.np = split_run
    g = pic.Pic(cfg, x, p, ay, az, ey, ez, stream=stream.cuda_stream, reducer=reducer)
    if mlp is not None:
        mlp.attach(g)
    H0 = g.energy()["total"]
    it_warm = g.step(warmup)
    # timed steps: one CUDA graph per step with device-ended loops (no per-launch
    # events); the launch counter is reset first and read after
    g.timing_enable(False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    it = g.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    launches = g.timing_read()["launches"]
    E = g.energy()
    # per-kernel durations: further steps of the same run with an event pair
    # around every launch (loops driven from the host)
    g.timing_enable(True)
    torch.cuda.synchronize()
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    nk = max(1, min(steps, kernel_steps))
    k0.record(stream)
    it_k = g.step(nk)
    k1.record(stream)
    k1.synchronize()
    tr = g.timing_read()
    tr["steps"] = nk
    tr["ms_per_step_host_loops"] = k0.elapsed_time(k1) / nk
    g.close()
    return {"ms": ms, "iters": it, "iters_warm": it_warm, "timing": tr, "launches": launches, "H0": H0,
            "H": E["total"], "gauss": E["gauss"], "rel_energy_err": abs(E["total"] - H0) / abs(H0)}


def drift_run(pic, torch, w, arrays, precision, warm, steps, stream, mlp=None, every=100):
    """The workload over its configured length: relative energy error and Gauss
    residual sampled every `every` steps (untimed)."""
    x, p, ay, az, ey, ez = arrays
    cfg = pic.Config.from_workload(w, precision=precision, warm_start=warm, sort_every=2,
                                   warm_field=1 if warm != pic.PIC_WARM_NONE else 0)
    g = pic.Pic(cfg, x, p, ay, az, ey, ez, stream=stream.cuda_stream)
    if mlp is not None:
        mlp.attach(g)
    H0 = g.energy()["total"]
    errs, gauss, sw = [], [], [0, 0]
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        n = min(every, steps - done)
        i1, i2 = g.step(n)
        sw[0] += i1
        sw[1] += i2
        done += n
        E = g.energy()
        errs.append(abs(E["total"] - H0) / abs(H0))
        gauss.append(E["gauss"])
    wall = time.perf_counter() - t0
    g.close()
    return {"steps": steps, "sample_every": every, "max_rel_energy_err": max(errs),
            "final_rel_energy_err": errs[-1], "max_gauss_residual": max(gauss),
            "energy_ok": max(errs) <= 1e-10, "sweeps_per_step": {"I": sw[0] / steps, "II": sw[1] / steps},
            "wall_s": wall}


def e2e_run(pic, torch, w, arrays, precision, warm, steps, stream, mlp=None):
    """Whole job through the public API with host buffers: pic_init from pinned
    host arrays (H2D), `steps` steps, pic_get_state back to pinned host (D2H)."""
    x, p, ay, az, ey, ez = arrays
    hx = torch.from_numpy(x).pin_memory().numpy()
    hp = torch.from_numpy(p).pin_memory().numpy()
    out = {k: torch.empty(w.np, dtype=torch.float64).pin_memory().numpy() for k in ("x", "p")}
    out.update({k: np.empty(w.nx) for k in ("ex", "ey", "ez", "ay", "az")})
    cfg = pic.Config.from_workload(w, precision=precision, warm_start=warm, sort_every=2,
                                   warm_field=1 if warm != pic.PIC_WARM_NONE else 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = pic.Pic(cfg, hx, hp, ay, az, ey, ez, stream=stream.cuda_stream)
    if mlp is not None:
        mlp.attach(g)
    ta = time.perf_counter()          # pic_init returns with its work complete
    g.step(steps)
    tb = time.perf_counter()          # pic_step returns with its work complete
    g.get_state(**out)
    t1 = time.perf_counter()
    g.close()
    h2d = 2 * 8 * w.np + 4 * 8 * w.nx
    d2h = 2 * 8 * w.np + 5 * 8 * w.nx
    return {"s": t1 - t0, "h2d": h2d, "d2h": d2h,
            "phases_ms": {"init": 1e3 * (ta - t0), "steps": 1e3 * (tb - ta), "get_state": 1e3 * (t1 - tb)}}


def twod_run(steps: int, np_: int | None = None, oracle_np: int = 100):
    """Subsystem I of the 2D scheme (FP64, Sec. 4.3) on the 2D workload: wall time
    of `steps` substeps after one warm-up (each substep synchronises per sweep),
    marker-substeps/s, sweeps and energy; the 2D oracle timed on a small sample of
    the same workload on one host thread."""
    import dataclasses
    from paper_2203_06513_gb300 import pic2d as P2
    w = I.Workload2D() if np_ is None else dataclasses.replace(I.Workload2D(), np=int(np_))
    x, p = I.particles2d(w)
    ex, ey, az = I.fields2d(w)
    cfg = P2.Config2D(w.L1, w.L2, w.M1, w.M2, w.degree, w.np, w.weight, w.dt)
    g = P2.Pic2D(cfg, x, p, ex, ey, az)
    H0 = g.energy()["total"]
    g.substep1()
    t0 = time.perf_counter()
    sweeps = 0
    for _ in range(steps):
        sweeps += g.substep1()
    dt_s = time.perf_counter() - t0
    H1 = g.energy()["total"]
    g.close()
    out = {"value": w.np * steps / dt_s, "unit": "marker-substeps/s", "ms_per_substep": 1e3 * dt_s / steps,
           "sweeps_per_substep": sweeps / steps, "rel_energy_err": abs(H1 - H0) / abs(H0),
           "us_per_marker_sweep": 1e6 * dt_s / (w.np * max(1, sweeps)),
           "start": "x^(0) = x^n (the explicit predictor measured no fewer sweeps here)",
           "workload": "2D subsystem I: L1=L2=4pi, M1=M2=%d, k=%d, Np=%d, dt=%g, vth %g, A_z %g cos(2 x1) "
                       "cos(x2 2pi/L2), FP64" % (w.M1, w.degree, w.np, w.dt, w.vth, w.amp)}
    if oracle_np:
        from oracle import oracle2d as O2
        ws = dataclasses.replace(w, np=oracle_np)
        xs, ps = I.particles2d(ws)
        orc = O2.Oracle2D(w.L1, w.L2, w.M1, w.M2, w.degree, ws.weight, w.dt)
        t0 = time.perf_counter()
        orc.substep1(xs, ps, ex, ey, az)
        out["cpu_oracle"] = {"value": oracle_np / (time.perf_counter() - t0), "unit": "marker-substeps/s",
                             "cores": 1, "sample": "%d markers of the same workload, one substep" % oracle_np}
    return out


def _member_inputs(w):
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    return x, p, ay, az, ey, ez


def ensemble_inputs(n_runs: int, np_scale: float, seed: int):
    """Inputs of the batched-ensemble workload, generated by a pool of host
    processes (spawned before any CUDA call)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    ws_ = I.ensemble_members(n_runs, seed=seed, np_scale=np_scale)
    workers = max(1, min(16, (os.cpu_count() or 1)))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        ins = list(ex.map(_member_inputs, ws_, chunksize=4))
    return ws_, ins


def ensemble_run(pic, torch, ws_, ins, steps, warmup, stream, use_graph=True):
    """All runs in one ensemble (FP32 form, explicit predictor with the predicted
    start field), schedule picked by the autotuner; device-timed steps, each one
    graph launch (or, with use_graph=False, the same kernels with the loops driven
    from the host)."""
    cfgs = [pic.Config.from_workload(w, precision=pic.PIC_FP32, warm_start=pic.PIC_WARM_EXPLICIT, sort_every=2,
                                     warm_field=1)
            for w in ws_]
    t0 = time.perf_counter()
    ens = pic.Ensemble(cfgs, ins, use_graph=use_graph, stream=stream.cuda_stream)
    t_create = time.perf_counter() - t0
    H0 = [ens.run(r).energy()["total"] for r in range(len(ws_))]
    cache = os.path.join(ROOT, "paper_2203_06513_gb300", "_build", "ensemble_tune.txt")
    im, bps, cached = ens.tune(cache)
    ens.step(warmup)
    l0 = ens.launches
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sw, st = ens.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    launches = ens.launches - l0
    H = [ens.run(r).energy()["total"] for r in range(len(ws_))]
    errs = np.array([abs(a - b) / abs(b) for a, b in zip(H, H0)])
    err = float(errs.max())
    nps = np.array([w.np for w in ws_], dtype=np.float64)
    ens.close()
    total = float(nps.sum())
    ok = errs <= 1e-10
    return {"value": total * steps / (ms / 1e3), "unit": UNIT, "runs": len(ws_), "total_np": int(total),
            "value_runs_at_bar": float(nps[ok].sum()) * steps / (ms / 1e3),
            "runs_above_bar": int((~ok).sum()),
            "min_np_above_bar": int(nps[~ok].min()) if (~ok).any() else None,
            "median_rel_energy_err": float(np.median(errs)),
            "steps": steps, "warmup": warmup, "ms_per_step": ms / steps,
            "schedule": {"item_markers": im, "blocks_per_sm": bps, "from_cache": cached},
            "sweeps_per_step_mean": {"I": float(sw[:, 0].mean() / steps), "II": float(sw[:, 1].mean() / steps)},
            "sweeps_per_step_max": {"I": float(sw[:, 0].max() / steps), "II": float(sw[:, 1].max() / steps)},
            "max_rel_energy_err": err, "failed_runs": int((st != 0).sum()),
            "gpu_launches": int(launches), "create_s": t_create, "graph": bool(use_graph),
            "workload": "C4: %d runs, nx in {256,512,1024,2048}, Np log-uniform [1e5,4e6], pump U[0.01,0.3], "
                        "vth U[0.02,0.15], k=3, dt=0.05, FP32 form" % len(ws_)}


def oracle_sample(n_sample: int, steps: int, warmup: int, threads: int = 1):
    """The FP64 CPU oracle on n_sample markers of the workload's grid; its marker
    loops on `threads` host threads."""
    from oracle import oracle as O
    w = I.workload(WORKLOAD)
    ws_ = I.workload(WORKLOAD, np=n_sample)
    x, p = I.particles(ws_)
    ay, az, ey, ez = I.fields(ws_)
    orc = O.Oracle(w.L, w.nx, w.degree, ws_.weight, w.dt, w.tol, w.max_iter, threads=threads)
    s = O.initial_state(orc, x, p, ay, az, ey, ez)
    for _ in range(warmup):
        s = orc.step(s)
    t0 = time.perf_counter()
    for _ in range(steps):
        s = orc.step(s)
    return n_sample * steps / (time.perf_counter() - t0)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def reference_arm(args, ws, rank):
    """The reference arm: the oracle (plain FP64 CPU program of the same scheme) on
    a bounded sample of the workload (same grid, fewer markers), all host cores,
    the same --steps and --warmup as the GPU arm."""
    if rank != 0:
        return 0
    n_sample = int(os.environ.get("PIC_REF_SAMPLE", "40000"))
    steps, warmup = args.steps, args.warmup
    cores = host_cores()
    v = oracle_sample(n_sample, steps, warmup, threads=cores)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * n_sample / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "C2: L=4pi, M=2048, k=3, dt=0.05, pump 0.2, vth 0.1 "
                                   "(oracle on a marker sample)", "sample_np": n_sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n_sample} markers on the M=2048 grid, {warmup} + {steps} steps, "
                                       f"marker loops on {cores} threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _compact_kernel(k: dict) -> dict:
    out = {key: k[key] for key in ("kernel", "bound", "frac", "achieved", "unit", "launch_ms", "launches")}
    if "issue" in k:
        out["issue_frac"] = k["issue"]["frac"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libpic", choices=["libpic", "reference"])
    ap.add_argument("--np", type=float, default=None, help="override N_p (smaller runs)")
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--no-fp64-warm", action="store_true", help="skip the FP64 runs with a predicted start")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--drift-steps", type=int, default=1000,
                    help="steps of the untimed energy/Gauss drift runs of the FP32 forms (0: skip)")
    ap.add_argument("--deposit-variants", type=int, default=5,
                    help="steps of the FP32 runs that compare the deposit accumulations (0: skip)")
    ap.add_argument("--ensemble-runs", type=int, default=256, help="0: skip the batched-ensemble line")
    ap.add_argument("--ensemble-scale", type=float, default=1.0, help="scale of the runs' marker counts")
    ap.add_argument("--ensemble-host-loop", action="store_true",
                    help="drive the ensemble's loops from the host (same kernels, no graph; for profiling)")
    ap.add_argument("--twod-steps", type=int, default=5, help="substeps of the 2D subsystem-I line (0: skip)")
    ap.add_argument("--twod-np", type=float, default=None, help="markers of the 2D line (smaller runs)")
    ap.add_argument("--split", action="store_true",
                    help="with N > 1: one plasma of N x Np markers split over the ranks (an all-reduce of the "
                         "deposits per sweep) instead of N independent replicas; only the timed forms run")
    args = ap.parse_args()
    ws, rank, local = R.dist_env()
    if args.impl == "reference":
        return reference_arm(args, ws, rank)
    split_mode = args.split and ws > 1
    if split_mode:                      # only the timed forms of the split plasma
        args.ensemble_runs = 0
        args.drift_steps = 0
        args.deposit_variants = 0
        args.no_e2e = True
    ens_in = None
    if args.ensemble_runs > 0:          # host inputs first: the pool starts before any CUDA call
        ens_in = ensemble_inputs(args.ensemble_runs, args.ensemble_scale, seed=R.replica_seed(0, rank))

    import torch
    from paper_2203_06513_gb300 import pic
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    kw = {"seed": R.replica_seed(0, rank)}
    if args.np:
        kw["np"] = int(args.np)
    w = I.workload(WORKLOAD, **kw)
    split_run = None
    if split_mode:
        # one plasma of ws x Np markers (one seed), this rank's contiguous share
        from paper_2203_06513_gb300 import split as S
        w_local = w
        w = I.workload(WORKLOAD, seed=0, np=w_local.np * ws)
        lo, hi = S.shard(w.np, rank, ws)
        x, p = I.particles_range(w, lo, hi, workers=max(1, min(16, os.cpu_count() or 1)))
        split_run = (S.TorchDeviceReducer(), hi - lo)
    else:
        x, p = I.particles(w, workers=max(1, min(16, os.cpu_count() or 1)))
    ay, az, ey, ez = I.fields(w)
    arrays = (x, p, ay, az, ey, ez)
    stream = torch.cuda.Stream()
    mlp = None
    if os.path.exists(WEIGHTS):
        d = np.load(WEIGHTS)
        mlp = pic.Mlp(d["norm"], d["params"], stream=stream.cuda_stream)

    def barrier():
        R.barrier(ws, torch.cuda.synchronize)

    def max_over_ranks(v):
        return R.max_over_ranks(v, ws, device="cuda")

    head_warm = pic.PIC_WARM_MLP if mlp is not None else pic.PIC_WARM_EXPLICIT
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    r_head = run_form(pic, torch, w, arrays, pic.PIC_FP32, head_warm, args.steps, args.warmup, stream,
                      mlp if mlp is not None else None, split_run=split_run)
    clk = clocks.stop()
    barrier()
    r_expl = run_form(pic, torch, w, arrays, pic.PIC_FP32, pic.PIC_WARM_EXPLICIT, args.steps,
                      args.warmup, stream, split_run=split_run)
    barrier()
    k64 = args.fp64_steps if args.fp64_steps is not None else max(1, min(args.steps, 4))
    r64 = run_form(pic, torch, w, arrays, pic.PIC_FP64, pic.PIC_WARM_NONE, k64, max(1, min(args.warmup, 3)),
                   stream, split_run=split_run)
    barrier()
    # the FP64 form started from a proposal and its field: the explicit predictor
    # and the learned one (what the network gains over the plain method)
    r64w = {}
    if not args.no_fp64_warm:
        for name, wm in (("explicit", pic.PIC_WARM_EXPLICIT), ("learned", pic.PIC_WARM_MLP)):
            if wm == pic.PIC_WARM_MLP and mlp is None:
                continue
            r64w[name] = run_form(pic, torch, w, arrays, pic.PIC_FP64, wm, k64, max(1, min(args.warmup, 3)),
                                  stream, mlp if wm == pic.PIC_WARM_MLP else None, split_run=split_run,
                                  kernel_steps=1)
        barrier()
    e2e = None if args.no_e2e else e2e_run(pic, torch, w, arrays, pic.PIC_FP32, head_warm, args.steps,
                                           stream, mlp)
    barrier()
    drift = None
    if args.drift_steps > 0:
        drift = {"learned" if mlp is not None else "explicit_head":
                 drift_run(pic, torch, w, arrays, pic.PIC_FP32, head_warm, args.drift_steps, stream, mlp)}
        drift["explicit"] = drift_run(pic, torch, w, arrays, pic.PIC_FP32, pic.PIC_WARM_EXPLICIT,
                                      args.drift_steps, stream)
        barrier()
    dep = None
    if args.deposit_variants > 0:
        dep = {}
        for name, code in (("float", pic.PIC_ACC_FLOAT), ("compensated", pic.PIC_ACC_COMPENSATED),
                           ("double", pic.PIC_ACC_DOUBLE)):
            r = run_form(pic, torch, w, arrays, pic.PIC_FP32, pic.PIC_WARM_EXPLICIT, args.deposit_variants, 0,
                         stream, deposit=code)
            dep[name] = {"gauss_residual": r["gauss"], "rel_energy_err": r["rel_energy_err"],
                         "sweep1_launch_ms": r["timing"]["sweep1_ms"] / max(1, r["timing"]["sweep1_launches"]),
                         "sweep2_launch_ms": r["timing"]["sweep2_ms"] / max(1, r["timing"]["sweep2_launches"]),
                         "ms_per_step": r["ms"] / args.deposit_variants}
        barrier()
    twod = None
    if args.twod_steps > 0 and not split_mode and rank == 0:
        twod = twod_run(args.twod_steps, np_=args.twod_np, oracle_np=0 if args.no_cpu else 100)
    ens = None
    if ens_in is not None:
        del arrays, x, p
        ens = ensemble_run(pic, torch, ens_in[0], ens_in[1], max(1, min(args.steps, 10)), 1, stream,
                           use_graph=not args.ensemble_host_loop)
        ens_in = None
        barrier()

    ms_head = max_over_ranks(r_head["ms"])
    ms_expl = max_over_ranks(r_expl["ms"])
    ms64 = max_over_ranks(r64["ms"])
    ms64w = {k: max_over_ranks(r["ms"]) for k, r in r64w.items()}
    e2e_s = max_over_ranks(e2e["s"]) if e2e else None
    per_rank = w.np / ws if split_mode else w.np          # markers each rank advances
    value = R.whole_job_rate(per_rank, ws, args.steps, ms_head / 1e3)
    v_expl = R.whole_job_rate(per_rank, ws, args.steps, ms_expl / 1e3)
    v64 = R.whole_job_rate(per_rank, ws, k64, ms64 / 1e3)
    tr = r_head["timing"]
    hbm, tflops, peak_kind = peaks()
    sm_mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz")
    kernels = kernel_rooflines(tr, int(per_rank), hbm, tflops, peak_kind,
                               torch.cuda.get_device_properties(local).multi_processor_count, sm_mhz)
    dominant = max(kernels, key=lambda k: k["share_ms"])
    if rank == 0:
        cpu = None
        if not args.no_cpu:
            n_cpu = int(os.environ.get("PIC_CPU_SAMPLE", "1000000"))
            cores = host_cores()
            v1 = oracle_sample(n_cpu, 1, 0, threads=1)
            vall = oracle_sample(n_cpu, 1, 0, threads=cores)
            cpu = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{n_cpu} markers on the M=2048 grid, 1 step, marker loops on one thread",
                   "all_cores": {"value": vall, "cores": cores,
                                 "sample": f"the same sample, marker loops on {cores} threads"}}

        def sweeps(r, k):
            return {"I": r["iters"][0] / k, "II": r["iters"][1] / k}

        # order: contract keys, measurement context, bulky detail, then the energy
        # and convergence figures last (a reader of the line's tail sees them)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_head / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "C2: L=4pi, M=2048, k=3, Np=%d per GPU, dt=0.05, pump 0.2, vth 0.1"
                                   % per_rank,
                       "form": "FP32 particles + FP64 grid",
                       "warm_start": "learned (MLP)" if mlp is not None else "explicit (no weights file)",
                       "l2": "inputs larger than L2 (markers %.1f GB)" % (w.np * 24 / 1e9),
                       "parallelism": ("one plasma split by markers, all-reduce per sweep" if split_mode
                                       else "replicas" if ws > 1 else "single GPU")},
            "gpu_launches": r_head["launches"],
            "roofline": dominant,
            "clocks": clk,
            "cpu_baseline": cpu,
            "e2e": None if e2e is None else {
                "value": R.whole_job_rate(w.np, ws, args.steps, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": e2e["h2d"] / args.steps,
                "d2h_bytes_per_step": e2e["d2h"] / args.steps,
                "phases_ms": e2e["phases_ms"]},
            "kernels": [_compact_kernel(k) for k in kernels],
            "kernel_ms": {"steps": tr["steps"], "sweep1": tr["sweep1_ms"], "sweep2": tr["sweep2_ms"],
                          "solve": tr["solve_ms"], "warm_start": tr["warm_ms"],
                          "ms_per_step_host_loops": tr["ms_per_step_host_loops"]},
            "ensemble": ens,
            "twod": twod,
            "deposit_accumulation": dep,
            "fp64": {"value": v64, "unit": UNIT, "steps": k64, "ms_per_step": ms64 / k64,
                     "rel_energy_err": r64["rel_energy_err"], "gauss_residual": r64["gauss"],
                     "sweeps_per_step": sweeps(r64, k64),
                     "speedup_fp32_learned_over_fp64": value / v64},
            "fp64_predicted_start": {
                k: {"value": R.whole_job_rate(per_rank, ws, k64, ms64w[k] / 1e3),
                    "ms_per_step": ms64w[k] / k64, "rel_energy_err": r["rel_energy_err"],
                    "sweeps_per_step": sweeps(r, k64)} for k, r in r64w.items()},
            "fp32_explicit": {"value": v_expl, "unit": UNIT, "ms_per_step": ms_expl / args.steps,
                              "rel_energy_err": r_expl["rel_energy_err"],
                              "sweeps_per_step": sweeps(r_expl, args.steps)},
            "drift": drift,
            "warm_start_ms": tr.get("warm_ms"),
            "sweeps_per_step": sweeps(r_head, args.steps),
            "gauss_residual": r_head["gauss"],
            "rel_energy_err": r_head["rel_energy_err"],
            "energy_ok": r_head["rel_energy_err"] <= 1e-10,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
