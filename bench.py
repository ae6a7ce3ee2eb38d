#!/usr/bin/env python
"""Benchmark of the Turret hot path on one GB300 (or N replicas, one per GPU).

Headline workload: the 256 x 256 x 512 sliding turret window (33.5 M cells)
with the spherical-harmonic irregular particle of volume-equivalent diameter
32 (6252 surface markers), Re ~ 1000 (nu = 6.4e-4), kappa = 2, FP32
population storage, the paper's predictor, the force taken on the offset
surface (force_eval 0).  One step = collide+stream over every window cell,
particle update, window slide, stress/velocity on the support box, surface
force/torque and four IBM cycles (replays of the step's CUDA graphs).

Printed JSON line (rank 0):
  value     window cells x steps / s over the timed steps, in GLUPS (all ranks)
  roofline  the step's own collide+stream launches (far cells + near region)
            timed alone: algorithmic bytes (216 per cell in FP32, 108 with
            16-bit storage) / mean time, against the measured HBM copy
            bandwidth; whole_step_frac: the same bytes over the whole step
  e2e       the same metric through the public C ABI from host data:
            context + surface upload + steps with a particle-state read
            after every step
  windows   the other windows and storage formats (the 96 x 96 x 192 prolate
            window, the 192 x 192 x 384 irregular window, FP16 / BF16 /
            BF16 with stochastic rounding), each with its step rate and its
            collide+stream roofline fraction
  cpu_baseline  the FP64 oracle on the host cores, a bounded sample of the
            same workload (and one thread on the 96 x 96 x 192 window)
--impl reference times the oracle alone as the reference arm.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS & %HBM roofline per RR-LBM+IBM step; mixed/batched vs FP32 at ≤1% drag err"
BYTES_PER_CELL = {"f32": 216, "f16": 108, "bf16": 108}
K1_PROFILE = os.path.join(ROOT, "profiles", "k_collide_stream_far_f32_irregular_256x256x512.md")
K1_SOURCES = [os.path.join(ROOT, "paper_2408_15115_gb300", "csrc", f)
              for f in ("lbm_cell.cuh", "lbm_kernels.cu", "lbm_far.cu", "turret_internal.cuh")]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="irregular_large")
    p.add_argument("--storage", default="f32")
    p.add_argument("--no-windows", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-ensemble", action="store_true")
    p.add_argument("--ensemble-steps", type=int, default=100)
    p.add_argument("--no-learned", action="store_true")
    p.add_argument("--case", default=None, choices=["mlp_train", "ensemble_steps", "window"],
                   help="run one small workload for a profiler capture instead of the benchmark")
    p.add_argument("--learned-steps", type=int, default=6000)
    p.add_argument("--runs", type=int, default=64, help="runs of the ensemble_steps profiling case")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Ranks:
    """Replica bookkeeping of a multi-GPU run (one independent window per
    rank, no data-path collective): a barrier around the timed region and the
    maximum of a scalar over ranks.  device None: CPU tensors (gloo)."""

    def __init__(self, world, device=None):
        self.world = world
        self.device = device

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, x):
        if self.world == 1:
            return float(x)
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())


def whole_job_glups(world, cells, steps, ms_max):
    """Cells updated by all ranks per second over the slowest rank's time."""
    return world * cells * steps / (ms_max / 1e3) / 1e9


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def source_hash():
    """Hash of the collide+stream kernel's sources (cell code and kernel)."""
    h = hashlib.sha256()
    for f in K1_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def profile_traffic():
    """DRAM bytes per launch of the collide+stream kernel from the committed ncu
    summary, or None when the kernel source changed since it was taken."""
    try:
        txt = open(K1_PROFILE).read()
    except OSError:
        return None
    src_hash = source_hash()
    vals = {}
    for line in txt.splitlines():
        if line.startswith("machine:"):
            for kv in line[len("machine:"):].split():
                k, _, v = kv.partition("=")
                vals[k] = v
    if vals.get("source_sha256_16") != src_hash or "dram_bytes_per_launch" not in vals:
        return None
    return float(vals["dram_bytes_per_launch"])


def workload(name, storage):
    from paper_2408_15115_gb300 import configs
    fn = configs.WORKLOADS[name]
    return fn(storage=storage) if name != "sphere_box" else fn()


ORACLE_BYTES_PER_CELL = 600  # dense FP64 fields of the oracle: 2 x 27 populations, h, u, sigma, scratch


def oracle_fits(cells):
    """Whether the oracle's dense fields for `cells` cells fit in half of the
    host memory available now."""
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        return True
    return ORACLE_BYTES_PER_CELL * cells < 0.5 * avail


def oracle_sample(cfg, budget_s=15.0, max_steps=None, threads=None):
    """Time the FP64 oracle on the workload: coupled steps of the full window
    from rest; returns (cells*steps/s in GLUPS, threads, steps, seconds)."""
    from oracle import oracle as O
    O.set_threads(threads or os.cpu_count() or 1)
    bc = cfg["bc"]
    s = O.Sim(cfg["nx"], cfg["ny"], cfg["nz"], 3 * cfg["nu"] + 0.5, *bc, sponge=cfg["sponge"], slide=cfg["slide"],
              anchor_frac=cfg["anchor"], kappa=cfg["kappa"], g=cfg["g"])
    s.init_fields()
    s.load_particle(cfg["verts"], cfg["tris"], cfg["r0"])
    cells = cfg["nx"] * cfg["ny"] * cfg["nz"]
    t0 = time.perf_counter()
    s.step(1)
    t1 = time.perf_counter() - t0
    n = max(1, int(budget_s / max(t1, 1e-6)))
    if max_steps is not None:
        n = min(n, max_steps)
    t0 = time.perf_counter()
    s.step(n)
    dt = time.perf_counter() - t0
    used = O.get_threads()
    del s
    return cells * n / dt / 1e9, used, n, dt


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    cfg = workload(args.workload, args.storage)
    cells = cfg["nx"] * cfg["ny"] * cfg["nz"]
    if not oracle_fits(cells):
        print(json.dumps({"impl": "reference", "unavailable": "the FP64 oracle's dense fields (%.1f GB) exceed half of "
                          "this host's available memory" % (ORACLE_BYTES_PER_CELL * cells / 1e9)}))
        return
    # each reference step is one coupled oracle step of the full window; the
    # count is capped so the whole arm ends within a few minutes
    budget = 150.0
    from oracle import oracle as O
    O.set_threads(os.cpu_count() or 1)
    s = O.Sim(cfg["nx"], cfg["ny"], cfg["nz"], 3 * cfg["nu"] + 0.5, *cfg["bc"], sponge=cfg["sponge"],
              slide=cfg["slide"], anchor_frac=cfg["anchor"], kappa=cfg["kappa"], g=cfg["g"])
    s.init_fields()
    s.load_particle(cfg["verts"], cfg["tris"], cfg["r0"])
    cells = cfg["nx"] * cfg["ny"] * cfg["nz"]
    t0 = time.perf_counter()
    s.step(1)
    t1 = time.perf_counter() - t0
    # the first step counts as warm-up; the rest of the requested warm-up runs
    # too, bounded to about 30 s of oracle work
    warm = max(1, min(args.warmup, 1 + int(30.0 / max(t1, 1e-6))))
    if warm > 1:
        s.step(warm - 1)
    k = max(1, min(args.steps, int(budget / max(t1, 1e-6))))
    t0 = time.perf_counter()
    s.step(k)
    dt = time.perf_counter() - t0
    v = cells * k / dt / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GLUPS", "n_gpus": args.gpus,
           "steps": k, "warmup": warm, "ms_per_step": 1e3 * dt / k, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": cfg["name"], "cells": cells, "markers": int(cfg["verts"].shape[0]),
                      "force_eval": 0, "predictor": "paper",
                      "steps_requested": args.steps, "warmup_requested": args.warmup},
           "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": O.get_threads(), "kind": "oracle",
                            "sample": "%d coupled FP64 oracle steps of the full %s window (of %d requested)" %
                                      (k, cfg["name"], args.steps)},
           "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def time_window(cfg, dev, K, W, kernel_launches, peaks, events=None):
    """Step rate of one window and its collide+stream launches alone.

    The coupled step is replayed K times after W warm-up steps (CUDA events on
    the context's stream); then the step's own collide+stream launches
    (lbm_fluid_step: far cells, with the near region beside them)
    `kernel_launches` times.
    Returns the rates, the roofline fractions and the state."""
    import torch

    from paper_2408_15115_gb300 import configs
    cells = cfg["nx"] * cfg["ny"] * cfg["nz"]
    t = configs.make_turret(cfg, device=dev, flags=cfg.get("flags"))
    t.load_surface(cfg["verts"], cfg["tris"], cfg["r0"])
    st = t.stream
    t.step(max(W, 8) if K >= 8 else W)  # capture the one-step and the 8-step graphs before timing
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if events is not None:
        events["before"]()
    ev0.record(st)
    t.step(K)
    ev1.record(st)
    torch.cuda.synchronize(dev)
    if events is not None:
        events["after"]()
    ms = ev0.elapsed_time(ev1)
    state = t.state()
    t.fluid_step(3)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    t.fluid_step(kernel_launches)
    e1.record(st)
    torch.cuda.synchronize(dev)
    k_ms = e0.elapsed_time(e1) / kernel_launches
    t.close()
    bpc = BYTES_PER_CELL[cfg["storage"]]
    hbm = peaks["hbm_gbs"]
    return {"ms": ms, "state": state, "cells": cells,
            "glups": cells * K / (ms / 1e3) / 1e9, "us_per_step": 1e3 * ms / K,
            "kernel_us": 1e3 * k_ms, "kernel_glups": cells / (k_ms / 1e3) / 1e9, "bytes_per_cell": bpc,
            "kernel_gbs": bpc * cells / (k_ms / 1e3) / 1e9,
            "kernel_frac": bpc * cells / (k_ms / 1e3) / 1e9 / hbm,
            "whole_step_frac": bpc * cells / (ms / K / 1e3) / 1e9 / hbm}


def windows_leg(dev, peaks, W, f32_us):
    """Every window size and storage format: the step rate and the
    collide+stream roofline fraction (bytes per cell of the storage format)."""
    legs = [("prolate_turret", "f32", None, 4000, 1000),
            ("irregular_turret", "f32", None, 1000, 300), ("irregular_turret", "f16", None, 1000, 300),
            ("irregular_turret", "bf16", None, 1000, 300),
            ("irregular_turret", "bf16", {"stochastic_rounding": 1}, 1000, 300),
            ("irregular_large", "f16", None, 400, 100), ("irregular_large", "bf16", None, 400, 100),
            ("irregular_large", "bf16", {"stochastic_rounding": 1}, 400, 100)]
    out = {}
    for name, storage, flags, K, KL in legs:
        cfg = workload(name, storage)
        if flags:
            cfg["flags"] = flags
        r = time_window(cfg, dev, K, W, KL, peaks)
        key = "%s/%s%s" % (cfg["name"], storage, "_sr" if flags else "")
        e = {k: r[k] for k in ("glups", "us_per_step", "kernel_us", "kernel_glups", "bytes_per_cell", "kernel_gbs",
                               "kernel_frac", "whole_step_frac")}
        e["steps"] = K
        e["particle_steps_per_s"] = K / (r["ms"] / 1e3)
        if storage == "f32":
            f32_us[cfg["name"]] = (r["us_per_step"], r["kernel_us"])
        elif cfg["name"] in f32_us:
            e["step_speedup_vs_f32"] = f32_us[cfg["name"]][0] / r["us_per_step"]
            e["kernel_speedup_vs_f32"] = f32_us[cfg["name"]][1] / r["kernel_us"]
        out[key] = e
    return out


def ensemble_leg(dev, K, W, tile_cache):
    """The 64-run settling ensemble (seed 4): the plain FP32 form (each run
    alone, one after another, per-run step graphs) against the batched form
    (one launch per phase for all runs, autotuned tiles), in FP32 and with
    storage alternating FP32 / FP16.  Rates in particle-steps/s and GLUPS."""
    import torch

    from paper_2408_15115_gb300 import configs
    from paper_2408_15115_gb300 import turret as T

    base = configs.ensemble(64, seed=4, storage="alternate")
    cells = [c["nx"] * c["ny"] * c["nz"] for c in base]
    total = sum(cells)
    n = len(base)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def rates(ms, steps):
        s = ms / 1e3
        return {"particle_steps_per_s": n * steps / s, "glups": total * steps / s / 1e9, "ms_per_step": ms / steps}

    # plain FP32: every run alone, one after another
    f32 = configs.load_ensemble([dict(c, storage="f32") for c in base], device=dev)
    seq_ms = 0.0
    for t in f32:
        t.step(W)
        torch.cuda.synchronize(dev)
        a, b = ev(), ev()
        a.record(t.stream)
        t.step(K)
        b.record(t.stream)
        torch.cuda.synchronize(dev)
        seq_ms += a.elapsed_time(b)
    out = {"workload": "ensemble_64_seed4", "runs": n, "cells": total,
           "markers": int(sum(c["verts"].shape[0] for c in base)), "steps": K,
           "windows": sorted({"%dx%dx%d" % (c["nx"], c["ny"], c["nz"]) for c in base}),
           "plain_f32_sequential": rates(seq_ms, K)}

    def batched(runs, key):
        b = T.Batch(runs, device=dev)
        choice = b.autotune(cache_path=tile_cache, reps=10)
        b.step(W)
        torch.cuda.synchronize(dev)
        a, e = ev(), ev()
        a.record(b.stream)
        b.step(K)
        e.record(b.stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(e)
        r = rates(ms, K)
        alg = sum(c * (216 if t.storage == "f32" else 108) for c, t in zip(cells, runs))
        r["whole_step_gbs"] = alg / (ms / K / 1e3) / 1e9
        r["tiles"] = {"threads": choice.threads, "minb": choice.minb, "tx": choice.tx}
        r["gpu_launches_per_step"] = 6 + 3 + 1  # collide bulk + near, markers, moments, interp, reduce, 3 cycles, spread
        b.close()
        out[key] = r

    batched(f32, "batched_f32")
    for t in f32:
        t.close()
    del f32
    mixed = configs.load_ensemble(base, device=dev)
    batched(mixed, "batched_mixed")
    for t in mixed:
        t.close()
    out["speedup_batched_mixed_vs_plain_f32"] = (out["batched_mixed"]["particle_steps_per_s"] /
                                                 out["plain_f32_sequential"]["particle_steps_per_s"])
    # the surrogate: trained on the solver's own trajectories, then driving
    # the predictor of the mixed-storage batched ensemble
    net, sur = surrogate_leg(dev)
    out["surrogate"] = sur
    mixed = configs.load_ensemble(base, device=dev)
    for t in mixed:
        t.set_predictor("mlp", net)
    batched(mixed, "batched_mixed_surrogate")
    out["batched_mixed_surrogate"]["gpu_launches_per_step"] += 1  # the prediction
    st = [t.predictor_stats() for t in mixed]
    out["batched_mixed_surrogate"]["network_predictions"] = sum(s["net_steps"] for s in st)
    out["batched_mixed_surrogate"]["fallbacks"] = sum(s["fallbacks"] for s in st)
    for t in mixed:
        t.close()
    net.close()
    out["speedup_batched_mixed_surrogate_vs_plain_f32"] = (
        out["batched_mixed_surrogate"]["particle_steps_per_s"] / out["plain_f32_sequential"]["particle_steps_per_s"])
    # warm-started adaptive IBM cycles (linear extrapolation): fewer cycles
    # per step, at the price of a departure from the paper's step (see the
    # learned-predictor entry for its size)
    mixed = configs.load_ensemble(base, device=dev)
    for t in mixed:
        t.set_predictor("linear", None, warm=True, slip_eps=1e-4)
    batched(mixed, "batched_mixed_warm_linear")
    st = [t.predictor_stats() for t in mixed]
    out["batched_mixed_warm_linear"]["ibm_cycles_per_step"] = (sum(s_["cycles"] for s_ in st) /
                                                               max(sum(s_["steps"] for s_ in st), 1))
    out["batched_mixed_warm_linear"]["gpu_launches_per_step"] += 2  # the prediction, a fourth cycle
    for t in mixed:
        t.close()
    return out


def surrogate_leg(dev):
    """Train the force/torque network on trajectories of a batched settling
    ensemble (32 runs, 1500 steps; early stopping on 8 more) and compare its
    one-step force error on 8 held-out runs with linear extrapolation."""
    import time as _t

    import torch

    from paper_2408_15115_gb300 import configs
    from paper_2408_15115_gb300 import surrogate as S

    mk = lambda n, seed: configs.ensemble(n, seed=seed, storage="f32", d_range=(8.0, 16.0))
    t0 = _t.perf_counter()
    x, y = S.dataset(S.record_ensemble(mk(32, 11), 1500, device=dev))
    xv, yv = S.dataset(S.record_ensemble(mk(8, 12), 1500, device=dev))
    xt, yt = S.dataset(S.record_ensemble(mk(8, 13), 1500, device=dev))
    torch.cuda.synchronize(dev)
    t1 = _t.perf_counter()
    net, hist = S.train(x, y, epochs=30, batch=4096, lr=1e-3, weight_decay=1e-4, val=(xv, yv), device=dev)
    torch.cuda.synchronize(dev)
    t2 = _t.perf_counter()
    e = S.offline_errors(net, xt, yt)
    return net, {"train_pairs": int(x.shape[0]), "epochs": len(hist), "collect_s": t1 - t0, "train_s": t2 - t1,
                 "best_val_loss": min(h[1] for h in hist),
                 "held_out_mean_rel_force_error": {k: float(v.mean()) for k, v in e.items()}}


def learned_leg(dev, steps):
    """The learned-predictor workload: the irregular d = 32 particle (6252
    markers) in the 256 x 256 x 512 window at Re ~ 1000.  Its force/torque
    network is trained on trajectories of the three single-particle workloads
    (sphere box, prolate and irregular turret windows) and of eight
    spherical-harmonic particles at Re 200-600 (d 12-20, one batch).  The
    window then runs with the paper's step and with the predictor modes:
    the network (relative fallback rule), and warm-started adaptive IBM cycles
    driven by linear extrapolation and by the network.  Reported per run: the
    step rate, IBM cycles per step, how often the network drove the step, and
    the drag and settling velocity (mean over the last third) against the
    paper's step; and the one-step force error of the network against linear
    extrapolation on the paper run's own trajectory (never seen in training)."""
    import time as _t

    import numpy as np
    import torch

    from paper_2408_15115_gb300 import configs
    from paper_2408_15115_gb300 import surrogate as S

    t0 = _t.perf_counter()
    recs = []
    for cfg, n in ((configs.sphere_box(), 500), (configs.prolate_turret(), 2000),
                   (configs.irregular_turret(storage="f32"), 1500)):
        t = configs.make_turret(cfg, device=dev)
        t.load_surface(cfg["verts"], cfg["tris"], cfg["r0"])
        recs.append(S.record(t, n))
        t.close()
    rng = np.random.default_rng(21)
    hi_re = []
    for k in range(8):
        d = float(rng.uniform(12.0, 20.0))
        re = float(np.exp(rng.uniform(np.log(200.0), np.log(600.0))))
        hi_re.append(configs.ensemble_member("irregular", d, re, (96, 96, 192), "f32", seed=31 + k))
    recs += S.record_ensemble(hi_re, 1500, device=dev)
    x, y = S.dataset(recs)
    torch.cuda.synchronize(dev)
    t1 = _t.perf_counter()
    net, hist = S.train(x, y, epochs=60, batch=1024, lr=1e-3, weight_decay=1e-4, device=dev)
    torch.cuda.synchronize(dev)
    t2 = _t.perf_counter()
    res = {"workload": "irregular_256x256x512_turret", "storage": "f32", "steps": steps,
           "train_runs": 3 + len(hi_re), "train_pairs": int(x.shape[0]), "collect_s": t1 - t0, "train_s": t2 - t1,
           "final_train_loss": hist[-1]}
    hists = {}
    modes = (("paper", None, False), ("mlp", net, False), ("linear_warm", None, True), ("mlp_warm", net, True))
    for mode, nn_, warm in modes:
        cfg = configs.irregular_large(storage="f32")
        t = configs.make_turret(cfg, device=dev)
        if mode != "paper":
            # the network is used while its running error is at most that of
            # linear extrapolation (the plain predictor) on the same time levels
            t.set_predictor("mlp" if nn_ is not None else "linear", nn_, warm=warm, slip_eps=1e-4, resid_theta=1.0,
                            relative=True)
        t.set_log(steps + 1)
        t.load_surface(cfg["verts"], cfg["tris"], cfg["r0"])
        h, tot_ms = [], 0.0
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(steps // 100):
            ev0.record(t.stream)
            t.step(100)
            ev1.record(t.stream)
            torch.cuda.synchronize(dev)
            tot_ms += ev0.elapsed_time(ev1)
            st = t.state()
            h.append((st["F"][2], st["v"][2]))
        hists[mode] = np.array(h)
        n_steps = 100 * (steps // 100)
        ps = t.predictor_stats()
        entry = {"us_per_step": 1e3 * tot_ms / n_steps, "particle_steps_per_s": n_steps / (tot_ms / 1e3),
                 "ibm_cycles_per_step": ps["cycles"] / max(n_steps, 1)}
        if nn_ is not None:
            entry.update({"network_predictions": ps["net_steps"], "fallbacks": ps["fallbacks"]})
        if mode == "paper":
            xt, yt = S.dataset([t.log_records()])
            e = S.offline_errors(net, xt, yt)
            res["paper_run_one_step_rel_force_error"] = {k: float(v.mean()) for k, v in e.items()}
        res[mode] = entry
        t.close()
    late = slice(2 * len(hists["paper"]) // 3, None)
    b = hists["paper"][late].mean(0)
    for mode in ("mlp", "linear_warm", "mlp_warm"):
        a = hists[mode][late].mean(0)
        res[mode]["vs_paper_rel_dev"] = {"drag": float(abs(a[0] / b[0] - 1.0)),
                                         "settling_velocity": float(abs(a[1] / b[1] - 1.0))}
    err = res["paper_run_one_step_rel_force_error"]
    res["network_beats_linear_extrapolation"] = bool(err["network"] < err["linear"])
    res["within_1pct_of_paper_step"] = {m: bool(max(res[m]["vs_paper_rel_dev"].values()) <= 0.01)
                                        for m in ("mlp", "linear_warm", "mlp_warm")}
    net.close()
    return res


def run_ours(args):
    import numpy as np
    import torch

    from paper_2408_15115_gb300 import build as B
    from paper_2408_15115_gb300 import configs

    rank, world, local = dist_env()
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    cfg = workload(args.workload, args.storage)
    cells = cfg["nx"] * cfg["ny"] * cfg["nz"]
    K, W = args.steps, args.warmup
    peaks, peak_kind = measured_peaks()

    ranks = Ranks(world, dev)
    barrier = ranks.barrier
    max_over_ranks = ranks.max

    # ---- device-resident timed steps, then the step's collide+stream alone --
    clk = Clocks(local)
    r = time_window(cfg, dev, K, W, max(100, min(K, 1000)), peaks,
                    events={"before": lambda: (barrier(), torch.cuda.synchronize(dev), clk.__enter__()),
                            "after": lambda: (clk.__exit__(), barrier())})
    ms = max_over_ranks(r["ms"])
    clocks = clk.summary()
    kps = r["state"]["kernels_per_step"]
    value = whole_job_glups(world, cells, K, ms)
    bpc = BYTES_PER_CELL[cfg["storage"]]
    k_us = r["kernel_us"]
    achieved = bpc * cells / (k_us / 1e6) / 1e9
    traffic = profile_traffic() if cfg["storage"] == "f32" else None

    # ---- end to end through the C ABI from host data ----------------------
    from paper_2408_15115_gb300 import turret as T
    V = np.ascontiguousarray(cfg["verts"])
    Tr = np.ascontiguousarray(cfg["tris"], dtype=np.int32)
    K2 = max(K, 100)
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    t2 = configs.make_turret(cfg, device=dev)
    t2.load_surface(V, Tr, cfg["r0"])
    for _ in range(K2):
        t2.step(1)
        t2.state()
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    t2.close()
    del t2
    e2e = {"value": world * cells * K2 / e2e_s / 1e9, "unit": "GLUPS", "steps": K2,
           "h2d_bytes_per_step": (V.nbytes + Tr.nbytes) / K2,
           "d2h_bytes_per_step": __import__("ctypes").sizeof(T.ParticleState),
           "includes": "context creation, surface upload, and a particle-state read after every step"}

    if rank != 0:
        return
    out = {"metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": K, "warmup": W,
           "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": cfg["storage"], "data": "synthetic",
           "config": {"workload": cfg["name"], "cells": cells, "markers": int(cfg["verts"].shape[0]),
                      "storage": cfg["storage"], "nu": cfg["nu"], "kappa": cfg["kappa"], "g": cfg["g"][2],
                      "predictor": "paper", "force_eval": 0, "ibm_cycles": 4,
                      "l2": "inputs larger than L2 (two population buffers of %d MiB)" % (cells * bpc // 2 // 2**20),
                      "replicas": world},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                        "kernel": "k_collide_stream_far_f32, with the near-region k_collide_stream beside it"
                        if cfg["storage"] == "f32" else "collide+stream (far cells, with the near region beside them)",
                        "algorithmic_bytes_per_launch": bpc * cells,
                        "us_per_launch": k_us, "glups_kernel": cells / (k_us / 1e6) / 1e9,
                        "peak_kind": peak_kind, "particle_steps_per_s": K / (ms / 1e3),
                        "whole_step_frac": (bpc * cells / (ms / K / 1e3) / 1e9) / peaks["hbm_gbs"]},
           "e2e": e2e, "gpu_launches": kps * K, "clocks": clocks}
    if world == 1 and not args.no_windows:
        out["windows"] = windows_leg(dev, peaks, W, {cfg["name"]: (r["us_per_step"], k_us)}
                                     if cfg["storage"] == "f32" else {})
    if world == 1 and not args.no_ensemble:
        out["ensemble"] = ensemble_leg(dev, args.ensemble_steps, max(W, 3),
                                       os.path.join(ROOT, "paper_2408_15115_gb300", "_build", "tiles.json"))
    if world == 1 and not args.no_learned:
        out["learned_predictor"] = learned_leg(dev, args.learned_steps)
    if world == 1 and not args.no_cpu_baseline and oracle_fits(cells):
        v, cores, n, dt = oracle_sample(cfg, budget_s=12.0)
        v1, c1, n1, dt1 = oracle_sample(workload("prolate_turret", "f32"), budget_s=10.0, threads=1)
        out["cpu_baseline"] = {"value": v, "unit": "GLUPS", "cores": cores, "kind": "oracle",
                               "sample": "%d coupled FP64 oracle steps of the full %s window from rest (%.1f s)" %
                                         (n, cfg["name"], dt),
                               "single_thread": {"value": v1, "unit": "GLUPS", "cores": c1,
                                                 "sample": "%d coupled FP64 oracle steps of the full "
                                                           "prolate_96x96x192_turret window, one thread (%.1f s)"
                                                           % (n1, dt1)}}
    print(json.dumps(out))


def run_case(args):
    """Small fixed workloads for profiler captures: `mlp_train`, three BF16
    training steps of the surrogate network at batch 4096; `ensemble_steps`,
    the 64-run ensemble (or its first --runs runs) as one batch with tiles
    (128, 2, 32), 5 + 20 steps in FP32 then 5 + 20 with storage alternating
    FP32/FP16; `window`, the
    --workload window in --storage, --steps coupled steps without graphs
    (one launch per kernel) then three launches of its collide+stream alone."""
    import numpy as np
    import torch

    from paper_2408_15115_gb300 import build as B
    from paper_2408_15115_gb300 import configs
    from paper_2408_15115_gb300 import inputs as I
    from paper_2408_15115_gb300 import turret as T

    B.build()
    dev = torch.device("cuda", 0)
    out = {"case": args.case}
    if args.case == "mlp_train":
        net = T.MLP(I.mlp_init_params(0).astype(np.float32), batch_cap=4096, precision="bf16", device=dev)
        g = torch.Generator(device="cpu").manual_seed(0)
        x = torch.randn(4096, 34, generator=g).to(dev)
        y = torch.randn(4096, 6, generator=g).to(dev)
        for _ in range(3):
            net.train_step(x, y, want_loss=False)
        torch.cuda.synchronize(dev)
        net.close()
    elif args.case == "window":
        cfg = workload(args.workload, args.storage)
        t = configs.make_turret(cfg, device=dev, flags={"no_graph": 1})
        t.load_surface(cfg["verts"], cfg["tris"], cfg["r0"])
        t.step(args.steps)
        t.fluid_step(3)
        torch.cuda.synchronize(dev)
        out.update(workload=cfg["name"], storage=args.storage, steps=args.steps, status=t.state()["status"])
        t.close()
    else:
        for storage in ("f32", "alternate"):
            runs = configs.load_ensemble(configs.ensemble(64, seed=4, storage=storage)[:args.runs], device=dev)
            b = T.Batch(runs, device=dev)
            b.set_tiles(128, 2, [32] * len(runs))
            b.step(5)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(b.stream)
            b.step(20)
            e1.record(b.stream)
            torch.cuda.synchronize(dev)
            out[storage + "_ms_per_step"] = e0.elapsed_time(e1) / 20
            b.close()
            for t in runs:
                t.close()
    print(json.dumps(out))


def main():
    args = parse()
    if args.case:
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
