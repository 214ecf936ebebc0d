"""Train and evaluate the learned warm start on solver-generated pairs.

    python -m paper_2312_02968_gb300.train_surrogate --pairs 2000 --epochs 10 --out fno.pt

Pairs: a sphere mixture (1-8 Plummer/Hernquist spheres, seeds from --seed0)
on the n^3 mesh, its Newtonian field as the input and the H the plain
iteration converges to as the target (the mean of iterates 40 and 41). The
network runs on the (n/4)^3 grid. Evaluation: particle sets drawn from the
same kind of mixtures; each solve's particle accelerations are compared with
those of the converged field, and each solve is timed with CUDA events as
one CUDA graph replay.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def build_handle(B, n: int, N_max: int, mu: int = 2, sigma: float = 1.0, a0: float = 1.0, G: float = 1.0):
    """A handle on its own stream (graph capture needs a non-default stream)."""
    import torch

    return B.MondPM(n, 1, float(n), a0, G, mu, sigma, N_max, stream=torch.cuda.Stream())


def train(h, net, pairs: int, epochs: int, batch: int, lr: float, seed0: int = 1000, log=print):
    from . import surrogate as S
    from .workloads import mixture_spheres

    t0 = time.time()
    xs, ts = S.make_pairs(h, net.n, list(range(seed0, seed0 + pairs)), 1.0, mixture_spheres)
    t_pairs = time.time() - t0
    t0 = time.time()
    hist = net.train(xs, ts, epochs=epochs, batch=batch, lr=lr, seed=seed0, log=log)
    h.sync()
    t_train = time.time() - t0
    del xs, ts
    return {"pairs": pairs, "epochs": epochs, "batch": batch, "lr": lr, "loss": hist, "s_pairs": t_pairs,
            "s_train": t_train}


def evaluate(h, net, seeds, n_particles: int, ks_plain=(1, 2, 3, 4, 5, 6), ks_guess=(1, 2, 3), ks_mean=(2, 3, 4),
             ks_guess_mean=(2,), reps: int = 5):
    """Median particle-force error against the converged field and mean solve
    time (Newton solve included, each solve one CUDA graph replay) for plain
    and surrogate-seeded solves, each also with the mean of the last two
    iterations (MOND_OPT_CYCLE_MEAN). The converged field is the midpoint of
    the period-2 cycle the iteration ends in: the mean of iterations 40 and 41."""
    import torch

    from . import binding as B
    from . import surrogate as S
    from .workloads import sphere_mixture

    gs = S.GuessSolver(h, net, 1.0)
    dev = h.device
    st = h.stream
    errs = {f"plain{k}": [] for k in ks_plain}
    errs.update({f"guess{k}": [] for k in ks_guess})
    errs.update({f"mean{k}": [] for k in ks_mean})
    errs.update({f"guess_mean{k}": [] for k in ks_guess_mean})
    times = {k: [] for k in errs}
    stages = {}
    for sd in seeds:
        p, _ = sphere_mixture(h.nf, n_particles, sd)
        t = [torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")]
        h.bind_particles(*t)
        with torch.cuda.stream(st):
            h.deposit()
            h.set_option(B.OPT_CYCLE_MEAN, 1)
            h.solve_field(S.REF_ITERS + 1, B.WARM_NONE)
            h.set_option(B.OPT_CYCLE_MEAN, 0)
            ref = h.gather().double()
            nref = float(ref.norm())

            def with_mean(fn):
                h.set_option(B.OPT_CYCLE_MEAN, 1)
                try:
                    fn()
                finally:
                    h.set_option(B.OPT_CYCLE_MEAN, 0)

            def graph_of(fn):
                # every solve is timed as one CUDA graph replay, so that host
                # launch overhead does not favour the shorter kernel sequence
                fn()
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=st, capture_error_mode="relaxed"):
                    fn()
                return g

            def replay_ms(g):
                g.replay()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for _ in range(reps):
                    g.replay()
                e1.record(st)
                e1.synchronize()
                return e0.elapsed_time(e1) / reps

            dep_ms = replay_ms(graph_of(h.deposit))

            def run(name, fn):
                fn()
                errs[name].append(float((h.gather().double() - ref).norm()) / nref)
                # the deposit invalidates the stored Newton field, so every
                # replay pays for the Newton solve; its own time is taken out
                g = graph_of(lambda: (h.deposit(), fn()))
                times[name].append(replay_ms(g) - dep_ms)

            for k in ks_plain:
                run(f"plain{k}", lambda k=k: h.solve_field(k, B.WARM_NONE))
            for k in ks_guess:
                run(f"guess{k}", lambda k=k: gs.solve(k))
            for k in ks_mean:
                run(f"mean{k}", lambda k=k: with_mean(lambda: h.solve_field(k, B.WARM_NONE)))
            for k in ks_guess_mean:
                run(f"guess_mean{k}", lambda k=k: with_mean(lambda: gs.solve(k)))
            if not stages:
                # where a seeded solve's time goes (first system): each stage one graph replay
                newton = replay_ms(graph_of(lambda: (h.deposit(), h.solve_field(0, B.WARM_NONE)))) - dep_ms
                stages["newton"] = newton
                stages["features"] = replay_ms(graph_of(
                    lambda: S.features(gs.gN, h.nf, net.n, 1.0, gs.x, gs.scale, st)))
                stages["forward"] = replay_ms(graph_of(lambda: net.forward(gs.x, gs.y)))
                stages["upsample"] = replay_ms(graph_of(
                    lambda: S.upsample(gs.y, h.nf, net.n, gs.scale, gs.H, st, gs.up_scratch)))
                stages["solve1_from_guess"] = replay_ms(graph_of(lambda: (
                    h.deposit(), h.solve_field(0, B.WARM_NONE), h.solve_field(1, B.WARM_GUESS_RAW, gs.H)))) \
                    - dep_ms - newton
        h.sync()
    out = {k: {"force_err_median": float(np.median(errs[k])), "force_err_max": float(np.max(errs[k])),
               "ms_per_solve": float(np.mean(times[k]))} for k in errs}
    out["guess_stages_ms"] = stages
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mesh", type=int, default=256)
    ap.add_argument("--fno", default="64,32,16,4", help="coarse side, width, modes, layers")
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--eval-seeds", type=int, default=8)
    ap.add_argument("--eval-particles", type=int, default=10_000_000)
    ap.add_argument("--out", default=None, help="save the float32 parameters (torch.save)")
    args = ap.parse_args()

    import torch

    from . import binding as B
    from . import surrogate as S
    from .build import build

    build()
    h = build_handle(B, args.mesh, args.eval_particles)
    shape = tuple(int(v) for v in args.fno.split(","))
    net = S.FNO(*shape, seed=7, device=h.device, stream=h.stream)
    tr = train(h, net, args.pairs, args.epochs, args.batch, args.lr, args.seed0)
    if args.out:
        torch.save({"shape": shape, "params": net.params.cpu()}, args.out)
    ev = evaluate(h, net, list(range(args.eval_seeds)), args.eval_particles)
    print(json.dumps({"train": tr, "eval": ev}))


if __name__ == "__main__":
    main()
