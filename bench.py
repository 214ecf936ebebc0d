#!/usr/bin/env python
"""Benchmark of the MOND particle-mesh time step on GB300.

Workload: deep-MOND isothermal sphere (Sect. 4.3) of 1e6 equal-mass particles
(b = 8 px, truncated at 0.4 box), 256^3 periodic mesh, Gaussian kernel
sigma = 1.5 px, 4 field iterations per step, dt = 0.25, G = M = a0 = 1;
synthetic, seeded. A step is one pass of the whole hot path: deposit, field
solve, gather and leapfrog push.

Prints one JSON line. ``value`` is time steps (each with one MOND force solve)
per second with inputs resident in HBM; ``e2e`` is the same through host
buffers; ``warm`` is the warm-started variant (previous H, one iteration);
``roofline`` is the dominant HBM-bound kernel's achieved bandwidth against the
measured peak and ``particle_kernels`` the deposit's and gather's tap rates;
``cpu_baseline`` times the CPU oracle on a bounded sample. Side sections:
``density`` (Eq. apparentdensity kernels), ``interp_gather`` (the
mesh-interpolating gather), ``increment`` (the incremental solve), ``learned`` (training and evaluating the learned
warm start), ``ensemble`` (64 systems as one graph per step) and, with
``--scan``, step times against the particle count.
``--impl reference`` times the CPU oracle alone (the reference arm).
Under torchrun each rank steps its own independent replica (the single-system
solve does not shard); ``value`` sums the replicas.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MOND force solves/s and particle-steps/s at 256^3 (plain vs warm-start) at ≤1e-4 rel err"
WL = dict(n=256, pad=1, N=1_000_000, sigma=1.5, b=8.0, rmax=0.4 * 256, K=4, dt=0.25, mu=0, a0=1.0, G=1.0, box=256.0,
          seed=1)
WL_NAME = ("isothermal sphere 1e6 particles, 256^3 mesh, sigma 1.5 px, deep MOND, 4 iterations/step, dt 0.25 "
           "(configs: isothermal)")
REF_ITERS = 40  # converged reference: mean of iterates 40 and 41 (the undamped scheme ends in a 2-cycle)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed
    region: sampling starts before the warm-up (the tool takes a moment to
    come up), every line is stamped on arrival, and only the lines that
    arrive between window() and stop() are kept (one interval's grace)."""

    INTERVAL_MS = 50

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.w0 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def window(self):
        """The timed region begins now."""
        self.w0 = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        w1 = time.perf_counter() + self.INTERVAL_MS / 1000.0
        time.sleep(self.INTERVAL_MS / 1000.0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        time.sleep(0.05)
        w0 = self.w0 if self.w0 is not None else float("-inf")
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if not (w0 <= ts <= w1):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "interval_ms": self.INTERVAL_MS}


def make_workload(rank: int):
    from paper_2312_02968_gb300 import workloads as W

    return W.isothermal(WL["n"] * WL["pad"], WL["box"] / WL["n"], WL["N"], WL["b"], WL["rmax"], seed=WL["seed"] + rank)


def cpu_baseline(p, sample_particles: int):
    """The CPU oracle as it stands on this host: one field solve on the full
    256^3 mesh (K = 4, 42 transforms) plus deposit, gather and push of a
    sample of the particles, scaled to the full particle count."""
    import numpy as np

    import oracle

    n, sigma, K = WL["n"] * WL["pad"], WL["sigma"], WL["K"]
    s = WL["box"] / WL["n"]
    Ns = min(sample_particles, len(p["mass"]))
    sub = {k: np.ascontiguousarray(v[:Ns]) for k, v in p.items()}
    sub["mass"] = (sub["mass"] * (len(p["mass"]) / Ns)).astype(np.float32)
    t0 = time.perf_counter()
    acc, ka, _ = oracle.deposit_fixed(n, sigma, sub["cell"], sub["offset"], sub["mass"])
    t1 = time.perf_counter()
    _, rho = oracle.acc_to_rho(acc, ka, s)
    f = oracle.solve(rho, s, WL["G"], WL["a0"], WL["mu"], K, want=("acc",))
    t2 = time.perf_counter()
    g = oracle.gather(sigma, f["acc"], sub["cell"], sub["offset"])
    oracle.push(n, s, WL["dt"], g, sub["cell"], sub["offset"], sub["vel"])
    t3 = time.perf_counter()
    scale = len(p["mass"]) / Ns
    t_step = (t2 - t1) + scale * ((t1 - t0) + (t3 - t2))
    return {"t_step": t_step, "t_solve": t2 - t1, "t_particles_sample": (t1 - t0) + (t3 - t2), "Ns": Ns,
            "cores": oracle.num_threads(), "cpu_s": t3 - t0}


_REF_FIELD = None


def reference_step(p, sample_particles: int, rng):
    """One bounded sample of a time step for the CPU oracle: one of the 42
    scalar 3-D transforms of a K = 4 solve on the full 256^3 mesh (scaled x42)
    and deposit, gather and push of a random sample of the particles (scaled to
    all of them). The solve's pointwise loops are left out, so the scaled time
    is a lower bound of the oracle's step time."""
    import numpy as np

    import oracle

    n, sigma = WL["n"] * WL["pad"], WL["sigma"]
    s = WL["box"] / WL["n"]
    N = len(p["mass"])
    idx = np.sort(rng.choice(N, size=min(sample_particles, N), replace=False))
    sub = {k: np.ascontiguousarray(v[idx]) for k, v in p.items()}
    global _REF_FIELD
    if _REF_FIELD is None:  # allocated and touched once, as the oracle's solve reuses its arrays
        _REF_FIELD = np.ascontiguousarray(rng.standard_normal((n, n, n)) + 0j)
    t0 = time.perf_counter()
    acc, ka, _ = oracle.deposit_fixed(n, sigma, sub["cell"], sub["offset"], sub["mass"])
    t1 = time.perf_counter()
    oracle.lib().ora_fft3_raw(n, _REF_FIELD.ctypes.data_as(ctypes.c_void_p), -1)
    t2 = time.perf_counter()
    g = oracle.gather(sigma, np.zeros((3, n, n, n)), sub["cell"], sub["offset"])
    oracle.push(n, s, WL["dt"], g, sub["cell"], sub["offset"], sub["vel"])
    t3 = time.perf_counter()
    return 42.0 * (t2 - t1) + (N / len(idx)) * ((t1 - t0) + (t3 - t2))


def optional(fn, *args):
    """Run a rank-0 section that is reported beside the headline (no
    collectives inside); a Python-level failure there is recorded in its place
    instead of costing the headline line."""
    try:
        return fn(*args)
    except Exception as e:  # noqa: BLE001 - any failure of a side section is reported, not raised
        print(f"bench: {fn.__name__} failed: {e!r}", file=sys.stderr, flush=True)
        return {"error": f"{type(e).__name__}: {e}"}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on this host's cores, same workload and metric."""
    if rank != 0:
        return
    import numpy as np

    p = make_workload(0)
    rng = np.random.default_rng(7)
    for _ in range(args.warmup):
        reference_step(p, args.ref_sample, rng)
    ts = [reference_step(p, args.ref_sample, rng) for _ in range(args.steps)]
    cores = os.cpu_count()
    import oracle

    v = 1.0 / statistics.mean(ts)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WL_NAME, "l2": "inputs larger than L2"},
            "particle_steps_per_s": v * WL["N"],
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"per step: one of the 42 scalar 256^3 transforms of a K=4 solve (x42) plus "
                                       f"deposit/gather/push of {args.ref_sample} random particles (x"
                                       f"{WL['N'] // args.ref_sample}); pointwise solve loops omitted (lower bound "
                                       f"on the oracle's step time)"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "host_cores": cores}
    print(json.dumps(line), flush=True)


def run_density(h, B, stream, steps):
    """Time the density kernels (Eq. apparentdensity) on the 256^3 fields of the
    last solve: apparent (3 planes in, 1 out) and phantom (6 in, 1 out), and
    one shell-mass profile (Eq. totalmass); compare the enclosed apparent mass
    of the isothermal sphere with its closed form (Sect. 4.3)."""
    import math

    import torch

    n = WL["n"]
    plane = 4 * n ** 3
    out = torch.empty((n, n, n), dtype=torch.float32, device=torch.device("cuda", torch.cuda.current_device()))
    res = {}
    for name, kind, nin in (("apparent", B.DENS_APPARENT, 3), ("phantom", B.DENS_PHANTOM, 6)):
        for _ in range(3):
            h.density(kind, out)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            h.density(kind, out)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        algo = (nin + 1) * plane
        res[name] = {"ms_per_launch": ms, "algorithmic_bytes": algo, "GBps": algo / (ms / 1e3) / 1e9}
    s = WL["box"] / n
    nb = int(0.45 * n)
    h.shell_mass(B.DENS_APPARENT, [0.0, 0.0, 0.0], s, nb)
    t0 = time.perf_counter()
    shells = h.shell_mass(B.DENS_APPARENT, [0.0, 0.0, 0.0], s, nb)
    res["shell_mass_ms"] = (time.perf_counter() - t0) * 1e3
    b, M, a0, G = WL["b"] * s, 1.0, WL["a0"], WL["G"]
    ratios = {}
    for R in (16, 32, 48):
        closed = math.sqrt(M * a0 / G) * R * s / (1 + (b / (R * s)) ** 1.5)
        ratios[str(R)] = sum(shells[:R]) / closed
    res["enclosed_apparent_mass_vs_closed_form"] = ratios
    res["note"] = "fields of the last solve; inputs larger than L2"
    return res


def run_interp(h, B, stream, t, init, steps, warmup):
    """The mesh-interpolating gather (linear and Keys cubic interpolation of
    the node-smoothed field) in place of Eq. gi: graph-replayed steps per
    second on the same workload, and the force error of each against Eq. gi
    on the same density (relative L2 over the particles)."""
    import torch

    K, dt = WL["K"], WL["dt"]
    res = {}
    try:
        return _run_interp(h, B, stream, t, init, steps, warmup, K, dt, res, torch)
    finally:
        h.set_option(B.OPT_GATHER, 0)  # the steps after this section use Eq. gi


def _run_interp(h, B, stream, t, init, steps, warmup, K, dt, res, torch):
    for order in (1, 3):
        for k in t:
            t[k].copy_(init[k])
        h.set_option(B.OPT_GATHER, order)
        for _ in range(warmup):
            h.step(dt, K, B.WARM_NONE)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            h.step(dt, K, B.WARM_NONE)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        # accuracy on the current particles: exact ball sums, then the interpolation
        h.set_option(B.OPT_GATHER, 0)
        h.deposit()
        h.solve_field(K, B.WARM_NONE)
        g_exact = h.gather().double()
        h.set_option(B.OPT_GATHER, order)
        h.solve_field(K, B.WARM_NONE)
        g_int = h.gather().double()
        err = float(torch.linalg.norm(g_int - g_exact) / torch.linalg.norm(g_exact))
        res["linear" if order == 1 else "cubic"] = {"steps_per_s": 1000.0 / ms, "ms_per_step": ms,
                                                    "force_rel_err_vs_eq_gi": err}
    h.set_option(B.OPT_GATHER, 0)
    h.sync()
    res["note"] = "same workload and K; node-smoothed mesh made by the final pass, interpolated at the particles"
    return res


def run_increment(h, B, stream, t, init, steps, warmup):
    """The incremental solve (Sect. 5.2 item v, MOND_WARM_INCREMENT): after one
    full K-iteration step, graph-replayed steps whose solve is one iteration of
    the linearised steps on the deposit's change; steps per second, and the
    force error of the last incremental solve against the converged field of
    the same density (as the plain and warm errors)."""
    import torch

    K, dt = WL["K"], WL["dt"]
    try:
        h.enable_increment(True)
        for k in t:
            t[k].copy_(init[k])
        h.step(dt, K, B.WARM_NONE)  # the base
        for _ in range(warmup):
            h.step(dt, 1, B.WARM_INCREMENT)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            h.step(dt, 1, B.WARM_INCREMENT)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        # a few more with every launch event-timed: the incremental x-passes
        # against the measured copy peak
        peak, _ = load_peaks()
        h.set_option(B.OPT_TIMING, 1)
        h.kernel_stats()
        for _ in range(5):
            h.step(dt, 1, B.WARM_INCREMENT)
        stats = h.kernel_stats()
        h.set_option(B.OPT_TIMING, 0)
        passes = {}
        for st in stats:
            if st["name"].startswith(("xpass_d", "xpass_inv")) and st["launches"]:
                per = st["ms"] / st["launches"]
                gbps = st["bytes"] / st["launches"] / (per / 1000.0) / 1e9
                passes[st["name"]] = {"ms_per_launch": per, "GBps": gbps, "frac_of_peak": gbps / peak}
        h.deposit()
        h.solve_field(1, B.WARM_INCREMENT)
        g_inc = h.gather().double()
        h.solve_field(REF_ITERS, B.WARM_NONE)
        g_a = h.gather().double()
        h.solve_field(REF_ITERS + 1, B.WARM_NONE)
        g_ref = 0.5 * (g_a + h.gather().double())
        err = float(torch.linalg.norm(g_inc - g_ref) / torch.linalg.norm(g_ref))
        h.sync()
        return {"mode": "incremental, 1 iteration", "steps_per_s": 1000.0 / ms, "ms_per_step": ms,
                "force_rel_err": err, "incremental_steps_since_full_solve": warmup + steps + 6, "passes": passes}
    finally:
        h.enable_increment(False)


def run_scan(dev, steps):
    """Step time against the particle count on two mesh sizes (the runtime
    split of Sect. 5.2, Fig. 13: the transforms cost the same for any N, the
    particle kernels grow linearly): isothermal spheres (b = n/32, deep mu,
    sigma 1.5 px, K = 4), graph-replayed steps, then the same steps with
    event-timed launches for the split."""
    import numpy as np
    import torch

    from paper_2312_02968_gb300 import binding as B
    from paper_2312_02968_gb300 import workloads as W

    rows = []
    for n, Ns in ((128, (1_000, 10_000, 100_000, 1_000_000)), (256, (1_000, 10_000, 100_000, 1_000_000, 10_000_000))):
        for N in Ns:
            p = W.isothermal(n, 1.0, N, n / 32.0, 0.4 * n, seed=3)
            st = torch.cuda.Stream(device=dev)
            with torch.cuda.stream(st):
                h = B.MondPM(n, 1, float(n), 1.0, 1.0, B.MU_DEEP, 1.5, N, stream=st)
                t = [torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")]
            torch.cuda.synchronize()
            h.bind_particles(*t)
            h.set_option(B.OPT_USE_GRAPH, 1)
            for _ in range(3):
                h.step(0.25, 4, B.WARM_NONE)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(steps):
                h.step(0.25, 4, B.WARM_NONE)
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            h.set_option(B.OPT_TIMING, 1)
            h.kernel_stats()
            for _ in range(steps):
                h.step(0.25, 4, B.WARM_NONE)
            stats = h.kernel_stats()
            h.close()
            mesh = sum(s["ms"] for s in stats if s["name"][:5] in ("xpass", "ypass", "zpass")) / steps
            part = sum(s["ms"] for s in stats if s["name"] in ("bin", "deposit", "gather_push")) / steps
            rows.append({"n": n, "N": N, "ms_per_step": ms, "transforms_ms": mesh, "particles_ms": part,
                         "particle_steps_per_s": N * 1000.0 / ms})
    return rows


def run_learned(args, dev):
    """Learned warm start (sphere mixtures, 256^3, standard mu, sigma 1 px,
    G = a0 = 1): train the FNO on solver-made pairs, then time and score
    plain and surrogate-seeded solves on 1e7-particle mixtures."""
    import torch

    from paper_2312_02968_gb300 import binding as B
    from paper_2312_02968_gb300 import surrogate as S
    from paper_2312_02968_gb300 import train_surrogate as T

    st = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    prev = torch.cuda.current_stream(dev)
    torch.cuda.set_stream(st)
    try:
        h = B.MondPM(256, 1, 256.0, 1.0, 1.0, B.MU_STANDARD, 1.0, 10_000_000, stream=st)
        shape = tuple(int(v) for v in args.learned_fno.split(","))
        net = S.FNO(*shape, seed=7, device=dev, stream=st)
        tr = T.train(h, net, args.learned_pairs, args.learned_epochs, 8, 7e-4, seed0=1000, log=None)
        ev = T.evaluate(h, net, list(range(args.learned_eval)), 10_000_000)
        h.close()
    finally:
        torch.cuda.synchronize()
        torch.cuda.set_stream(prev)
    import math

    stages = ev.pop("guess_stages_ms", {})
    plain4 = ev["plain4"]
    best = min((k for k in ev if k.startswith("guess")), key=lambda k: ev[k]["force_err_median"])
    # the plain solve's error at each seeded solve's time (log-linear between the plain points)
    pts = sorted((ev[k]["ms_per_solve"], math.log(ev[k]["force_err_median"])) for k in ev if k.startswith("plain"))

    def plain_log_err(ms):
        for (t0, e0), (t1, e1) in zip(pts, pts[1:]):
            if ms <= t1:
                return e0 + (e1 - e0) * (ms - t0) / (t1 - t0)
        (t0, e0), (t1, e1) = pts[-2], pts[-1]
        return e0 + (e1 - e0) * (ms - t0) / (t1 - t0)

    gain = {k: math.exp(plain_log_err(ev[k]["ms_per_solve"])) / ev[k]["force_err_median"]
            for k in ev if k.startswith("guess")}
    meets = [k for k in ev if ev[k]["force_err_median"] <= 1e-4]
    fastest_meeting = min(meets, key=lambda k: ev[k]["ms_per_solve"]) if meets else None
    return {"workload": "sphere mixtures (1-8 Plummer/Hernquist), 1e7 particles, 256^3, standard mu, sigma 1 px",
            "fno": {"grid": shape[0], "width": shape[1], "modes": shape[2], "layers": shape[3], "weights": "bf16",
                    "accumulate": "f32"},
            "train": {k: tr[k] for k in ("pairs", "epochs", "batch", "lr", "s_pairs", "s_train")} |
                     {"loss_first": tr["loss"][0], "loss_last": tr["loss"][-1]},
            "solves": ev, "ref": "particle forces of the mean of iterates 40 and 41",
            "guess_stages_ms": stages,
            "error_ratio_plain_over_guess_at_equal_time": gain,
            "guess1_vs_plain4_speed": plain4["ms_per_solve"] / ev["guess1"]["ms_per_solve"],
            "best_guess": best, "fastest_at_1e-4": fastest_meeting}


def run_ensemble(args, dev, dist=None):
    """Batched ensemble: independent systems with sides drawn from
    {64, 96, 128, 192} and 1e4-1e6 particles (isothermal, deep mu, b = side/32;
    or Plummer, standard mu, a = side/16), sigma 1 px, 4 iterations, stepped
    together as one CUDA graph per step after per-system autotuning. Under
    several ranks the systems are dealt to the GPUs by estimated cost
    (longest first); each rank steps its share, rank 0 gathers."""
    import numpy as np
    import torch

    from paper_2312_02968_gb300 import binding as B
    from paper_2312_02968_gb300 import replicas as R
    from paper_2312_02968_gb300 import workloads as W

    rank = dist.get_rank() if dist is not None else 0
    world = dist.get_world_size() if dist is not None else 1
    rng = np.random.default_rng(7)
    specs = []
    for _ in range(args.ensemble_systems):
        n = int(rng.choice([64, 96, 128, 192]))
        N = int(round(math.exp(rng.uniform(math.log(1e4), math.log(1e6)))))
        specs.append((n, N, int(rng.integers(0, 2)), int(rng.integers(1 << 30))))
    mine = R.lpt_shard([R.system_cost(n, N) for n, N, _, _ in specs], world)[rank]
    hs, keep, Ns, sides = [], [], [], []
    t0 = time.time()
    for i in mine:
        n, N, kind, seed = specs[i]
        if kind == 0:
            p, mu = W.isothermal(n, 1.0, N, n / 32, 0.4 * n, seed=seed), B.MU_DEEP
        else:
            p, mu = W.plummer(n, 1.0, N, n / 16, 0.4 * n, seed=seed), B.MU_STANDARD
        st = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(st):
            h = B.MondPM(n, 1, float(n), 1.0, 1.0, mu, 1.0, N, stream=st)
            t = [torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")]
        torch.cuda.synchronize()
        h.bind_particles(*t)
        hs.append(h)
        keep.append(t)
        Ns.append(N)
        sides.append(n)
    t_gen = time.time() - t0
    t0 = time.time()
    tuned = [B.autotune(h, 4, 2) for h in hs]
    t_tune = time.time() - t0
    batch = B.Batch(hs)
    dt = 0.25
    batch.step(dt, n_steps=2, n_iter=4)
    batch.sync()
    l0 = batch.kernel_launches()
    if dist is not None:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(batch.stream)
    batch.step(dt, n_steps=args.ensemble_steps, n_iter=4)
    e1.record(batch.stream)
    e1.synchronize()
    batch.sync()
    ms = R.max_over_ranks(e0.elapsed_time(e1), dist, dev)  # the slowest rank's share
    launches = batch.kernel_launches() - l0
    sec = ms / 1000.0
    # the same systems stepped one after another on one stream, for comparison
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    serial_steps = 2
    torch.cuda.synchronize()
    s0.record()
    for h in hs:
        for _ in range(serial_steps):
            h.step(dt, 4, B.WARM_NONE)
        # each handle runs on its own stream: wait before the next one starts
        h.sync()
    s1.record()
    s1.synchronize()
    serial_sps = len(hs) * serial_steps / (s0.elapsed_time(s1) / 1000.0)
    batch.close()
    for h in hs:
        h.close()
    parts = R.gather_to_root({"tuned": tuned, "Ns": Ns, "sides": sides, "launches": launches,
                              "serial_sps": serial_sps}, dist)
    if rank != 0:
        return None
    chunks, allN, allsides = {}, [], []
    for part in parts:
        allN += part["Ns"]
        allsides += part["sides"]
        for c, pp in part["tuned"]:
            key = f"chunk{c}_pipe{pp}"
            chunks[key] = chunks.get(key, 0) + 1
    nsys = len(allN)
    return {"systems": nsys, "ranks": world, "sides": {str(k): allsides.count(k) for k in sorted(set(allsides))},
            "particles": int(sum(allN)), "steps": args.ensemble_steps, "ms": ms,
            "system_steps_per_s": nsys * args.ensemble_steps / sec,
            "particle_steps_per_s": sum(allN) * args.ensemble_steps / sec,
            "one_by_one_system_steps_per_s": sum(p["serial_sps"] for p in parts), "graph_launches_per_step": 1,
            "kernel_launches": sum(p["launches"] for p in parts), "autotuned": chunks, "s_generate": t_gen,
            "s_autotune": t_tune}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-sample", type=int, default=10_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch the timed steps directly, not as a CUDA graph")
    ap.add_argument("--learned-pairs", type=int, default=1024, help="training pairs of the learned warm start (0: skip)")
    ap.add_argument("--learned-epochs", type=int, default=12)
    ap.add_argument("--learned-eval", type=int, default=2, help="evaluation systems (1e7 particles each)")
    ap.add_argument("--learned-fno", default="32,32,16,4", help="network grid side, width, modes, layers")
    ap.add_argument("--ensemble-systems", type=int, default=64, help="systems of the batched ensemble (0: skip)")
    ap.add_argument("--ensemble-steps", type=int, default=20)
    ap.add_argument("--scan", action="store_true", help="also time steps against N on 128^3 and 256^3")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    args.warmup = max(args.warmup, 3)

    # the CPU baseline runs before any GPU work (no CUDA context in the oracle)
    p = make_workload(rank)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p, 50_000)

    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2312_02968_gb300 import binding as B
    from paper_2312_02968_gb300 import replicas as R

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    n, pad, N = WL["n"], WL["pad"], WL["N"]
    t = {k: torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")}
    init = {k: v.clone() for k, v in t.items()}
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    torch.cuda.set_stream(stream)  # torch's own copies below run in order with the handle's work
    h = B.MondPM(n, pad, WL["box"], WL["a0"], WL["G"], WL["mu"], WL["sigma"], N, stream=stream)
    h.bind_particles(t["cell"], t["offset"], t["vel"], t["mass"])
    K, dt = WL["K"], WL["dt"]
    h.set_option(B.OPT_USE_GRAPH, 0 if args.no_graph else 1)

    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        h.step(dt, K, B.WARM_NONE)
    h.sync()

    # ---- timed region: plain 4-iteration steps (one CUDA graph per step) -------
    barrier()
    sampler.window()
    l0 = h.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        h.step(dt, K, B.WARM_NONE)
    e1.record(stream)
    e1.synchronize()
    clocks = sampler.stop()
    barrier()
    launches = h.kernel_launches() - l0
    ms = e0.elapsed_time(e1)
    h.sync()

    # ---- the same steps with every launch bracketed by CUDA events --------------
    # (per-kernel durations for the roofline; direct launches, so a little slower)
    h.set_option(B.OPT_TIMING, 1)
    h.kernel_stats()
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(args.steps):
        h.step(dt, K, B.WARM_NONE)
    k1.record(stream)
    k1.synchronize()
    ms_timed_mode = k0.elapsed_time(k1)
    stats = h.kernel_stats()
    h.set_option(B.OPT_TIMING, 0)
    h.sync()
    ms = R.max_over_ranks(ms, dist, dev)
    ms_step = ms / args.steps
    value = world * args.steps / (ms / 1000.0)

    # ---- warm-started steps (previous H, one iteration) ------------------------
    for k in t:
        t[k].copy_(init[k])
    h.deposit()
    h.solve_field(K, B.WARM_NONE)
    h.gather_push(dt)
    for _ in range(args.warmup):
        h.step(dt, 1, B.WARM_PREV)
    barrier()
    w0 = torch.cuda.Event(enable_timing=True)
    w1 = torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    for _ in range(args.steps):
        h.step(dt, 1, B.WARM_PREV)
    w1.record(stream)
    w1.synchronize()
    barrier()
    wms = w0.elapsed_time(w1)
    wms = R.max_over_ranks(wms, dist, dev)
    warm_value = world * args.steps / (wms / 1000.0)

    # ---- accuracy against the converged field (not timed) ----------------------
    acc_info = None
    if not args.no_accuracy:
        h.deposit()
        h.solve_field(1, B.WARM_PREV)  # the warm solve as the timed loop runs it
        g_warm = h.gather().double()
        h.solve_field(K, B.WARM_NONE)
        g_plain = h.gather().double()
        h.solve_field(REF_ITERS, B.WARM_NONE)
        g_a = h.gather().double()
        h.solve_field(REF_ITERS + 1, B.WARM_NONE)
        g_b = h.gather().double()
        g_ref = 0.5 * (g_a + g_b)
        nr = float(torch.linalg.norm(g_ref))
        acc_info = {"ref": f"mean of iterates {REF_ITERS} and {REF_ITERS + 1} from H=0",
                    "plain_K4_rel_err": float(torch.linalg.norm(g_plain - g_ref)) / nr,
                    "warm_K1_rel_err": float(torch.linalg.norm(g_warm - g_ref)) / nr,
                    "ref_two_cycle_rel": float(torch.linalg.norm(g_a - g_b)) / nr}
        h.sync()

    # ---- densities of Eq. apparentdensity from the last solve's fields ---------
    dens_info = None
    if rank == 0:
        dens_info = optional(run_density, h, B, stream, args.steps)

    interp_info = None
    if rank == 0:
        interp_info = optional(run_interp, h, B, stream, t, init, args.steps, args.warmup)

    inc_info = None
    if rank == 0:
        inc_info = optional(run_increment, h, B, stream, t, init, args.steps, args.warmup)

    # ---- end to end through host buffers -------------------------------------
    cell_h = init["cell"].cpu().pin_memory()
    off_h = init["offset"].cpu().pin_memory()
    vel_h = init["vel"].cpu().pin_memory()
    for _ in range(2):
        h.step_host(dt, K, B.WARM_NONE, cell_h, off_h, vel_h)
    barrier()
    tq = time.perf_counter()
    for _ in range(args.steps):
        h.step_host(dt, K, B.WARM_NONE, cell_h, off_h, vel_h)
    barrier()
    e2e_s = time.perf_counter() - tq
    e2e_s = R.max_over_ranks(e2e_s, dist, dev)
    e2e_value = world * args.steps / e2e_s

    learned = ensemble = scan = None
    if rank == 0 and args.scan:
        scan = optional(run_scan, dev, args.steps)
    if rank == 0 and args.learned_pairs > 0:
        learned = optional(run_learned, args, dev)
    if args.ensemble_systems > 0:
        ensemble = run_ensemble(args, dev, dist)

    if rank == 0:
        peak, peak_src = load_peaks()
        hbm = [s for s in stats if s["name"].startswith(("xpass", "ypass", "zpass"))]
        dom = max(hbm, key=lambda s: s["ms"]) if hbm else None
        traffic = None
        try:
            with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
                tj = json.load(f)
            traffic = tj.get(dom["name"], {}).get("bytes_per_launch") if dom else None
        except Exception:
            traffic = None
        roof = None
        if dom:
            per_launch_ms = dom["ms"] / dom["launches"]
            algo = dom["bytes"] / dom["launches"]
            ach = algo / (per_launch_ms / 1000.0) / 1e9
            roof = {"bound": "hbm", "kernel": dom["name"], "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "peak_source": peak_src, "traffic": traffic,
                    "algorithmic_bytes_per_launch": algo, "ms_per_launch": per_launch_ms}
        # the particle kernels are not HBM-bound: their tap rate, live, and the share
        # of the L1/shared-memory pipe they use (ncu, profiles/particles.json)
        r = int(math.ceil(4 * WL["sigma"])) + 1
        taps = sum(1 for dz in range(-r, r + 1) for dy in range(-r, r + 1) for dx in range(-r, r + 1)
                   if dx * dx + dy * dy + dz * dz < 16 * WL["sigma"] ** 2)
        try:
            with open(os.path.join(ROOT, "profiles", "particles.json")) as f:
                pj = json.load(f)
        except Exception:
            pj = {}
        part = {}
        for s in stats:
            if s["name"] in ("deposit", "gather_push"):
                ms1 = s["ms"] / s["launches"]
                part[s["name"]] = {"ms_per_launch": ms1, "taps_per_launch": taps * N,
                                   "taps_per_s": taps * N / (ms1 / 1000.0),
                                   "l1tex_pipe_frac_ncu": pj.get(s["name"], {}).get("l1tex_throughput_frac")}
        kern = [{"name": s["name"], "launches": s["launches"], "ms": round(s["ms"], 4),
                 "share": round(s["ms"] / sum(x["ms"] for x in stats), 4),
                 "GBps": round(s["bytes"] / (s["ms"] / 1000.0) / 1e9, 1) if s["ms"] > 0 else None} for s in stats]
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WL_NAME, "l2": "inputs larger than L2 (1.4 GB of fields per step)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "particle_steps_per_s": value * N,
                "warm": {"value": warm_value, "unit": "solves/s", "mode": "previous H, 1 iteration",
                         "particle_steps_per_s": warm_value * N, "speedup_vs_plain": warm_value / value},
                "accuracy": acc_info,
                "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 36 * N,
                        "d2h_bytes_per_step": 36 * N},
                "gpu_launches": launches, "clocks": clocks, "roofline": roof, "particle_kernels": part,
                "kernels": kern,
                "ms_per_step_event_timed": ms_timed_mode / args.steps,
                "density": dens_info, "interp_gather": interp_info, "increment": inc_info, "learned": learned, "ensemble": ensemble}
        if scan is not None:
            line["scan"] = scan
        if cpu:
            line["cpu_baseline"] = {"value": 1.0 / cpu["t_step"], "unit": "solves/s", "cores": cpu["cores"],
                                    "kind": "oracle",
                                    "sample": f"one full 256^3 K=4 oracle solve ({cpu['t_solve']:.1f} s) plus "
                                              f"deposit/gather/push of {cpu['Ns']} of the {N} particles scaled "
                                              f"x{N // cpu['Ns']}; {cpu['cpu_s']:.1f} s of CPU work"}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    h.close()


if __name__ == "__main__":
    main()
