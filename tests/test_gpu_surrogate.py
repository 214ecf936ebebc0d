"""What the trained surrogate gains: a small network trained on the GPU by
the library's own forward/backward kernels, on pairs the solver makes, seeds
an iteration that then lands closer to the converged field than the same
number of plain iterations from H = 0; the plain iteration measures the error."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_MESH, FNO_SHAPE = 64, (16, 16, 6, 4)
A0 = G = 1.0


def rel(a, b):
    return float((a - b).norm() / b.norm())


def test_trained_guess_beats_plain_iterations():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2312_02968_gb300 import binding as B
    from paper_2312_02968_gb300 import surrogate as S
    from paper_2312_02968_gb300.workloads import mixture_spheres

    h = B.MondPM(N_MESH, 1, float(N_MESH), A0, G, B.MU_STANDARD, 1.0, 16)
    net = S.FNO(*FNO_SHAPE, seed=5, device=h.device, stream=h.stream)
    xs, ts = S.make_pairs(h, FNO_SHAPE[0], list(range(1000, 1096)), A0, mixture_spheres)
    hist = net.train(xs, ts, epochs=30, batch=8, lr=3e-3, seed=0)
    assert hist[-1] < 0.5 * hist[0], hist

    gs = S.GuessSolver(h, net, A0)
    rho = torch.empty((N_MESH,) * 3, device=h.device)
    errs = {"plain1": [], "guess1": [], "plain2": [], "guess2": [], "plain4": []}
    with torch.cuda.stream(h.stream):
        for sd in range(8):
            keep = S.mixture_density(N_MESH, h.s, mixture_spheres(N_MESH, sd), 0.4 * N_MESH, rho, h.stream)
            h.set_density(rho)
            h.solve_field(S.REF_ITERS, B.WARM_NONE)
            ra = h.get_field(B.FIELD_ACC).double()
            h.solve_field(S.REF_ITERS + 1, B.WARM_NONE)
            ref = 0.5 * (ra + h.get_field(B.FIELD_ACC).double())
            for k in (1, 2, 4):
                h.solve_field(k, B.WARM_NONE)
                errs[f"plain{k}"].append(rel(h.get_field(B.FIELD_ACC).double(), ref))
            for k in (1, 2):
                gs.solve(k)
                errs[f"guess{k}"].append(rel(h.get_field(B.FIELD_ACC).double(), ref))
            del keep
    med = {k: float(np.median(v)) for k, v in errs.items()}
    print("median force-mesh error vs converged:", med, "train loss", hist[0], "->", hist[-1])
    assert med["guess1"] < 0.5 * med["plain1"], med
    assert med["guess2"] < med["plain2"], med
