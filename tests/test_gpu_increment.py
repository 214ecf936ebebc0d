"""Incremental solve (Sect. 5.2 item v, MOND_WARM_INCREMENT) on the GPU against
the oracle's incremental solve, each side from its own base: the oracle's base
is its own FP64 solve of its own deposit, never a field read from the GPU.

Bars: the total fields after the increment agree to 1e-5 relative L2, as the
full solves do. The increments alone (GPU: new minus base state, both FP32)
carry the FP32 rounding of the base fields, about 1e-6 of |acc|, so their bar
is 1e-5 |acc| / |d acc| (ten times that). The base fields themselves, g_M
included, agree to 1e-5. A zero increment leaves every field bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2312_02968_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5

torch = pytest.importorskip("torch")


def rel(a, b, scale=None):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b if scale is None else scale)
    return np.linalg.norm(a - b) / max(den, 1e-300)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2312_02968_gb300 import binding

    return binding


def make(B, n, pad, p, sigma, mu, a0=1.0, box=None):
    dev = torch.device("cuda", 0)
    h = B.MondPM(n, pad, box if box is not None else float(n), a0, 1.0, mu, sigma, len(p["mass"]))
    t = [torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")]
    h.bind_particles(*t)
    return h, t


def moved(p, seed, frac=0.3, step=0.35):
    """A copy of p with a seeded fraction of the particles shifted by up to
    `step` pixels per axis, carried into the neighbouring cell where the
    offset leaves [-1/2, 1/2] (the push's convention)."""
    rng = np.random.default_rng(seed)
    q = {k: v.copy() for k, v in p.items()}
    sel = rng.random(len(q["mass"])) < frac
    pos = q["cell"].astype(np.float64) + q["offset"]
    pos[sel] += rng.uniform(-step, step, size=(int(sel.sum()), 3))
    c = np.floor(pos + 0.5)
    q["cell"] = c.astype(np.int32)
    q["offset"] = (pos - c).astype(np.float32)
    return q


def oracle_rho(p, n, sigma, s, kacc=None):
    acc, ka, _ = oracle.deposit_fixed(n, sigma, p["cell"], p["offset"], p["mass"], kacc)
    return acc, ka, oracle.acc_to_rho(acc, ka, s)[1]


@pytest.mark.parametrize("n,pad,mu,a0,K0,K", [(32, 1, 0, 1.0, 4, 1), (32, 1, 2, 0.02, 4, 3), (16, 2, 1, 0.05, 3, 2),
                                              (48, 1, 3, 1.0, 2, 2), (96, 1, 0, 1.0, 3, 2)])
def test_increment_matches_oracle(B, n, pad, mu, a0, K0, K):
    nf, sigma, s = n * pad, 1.5, 1.0
    p = W.isothermal(nf, s, 3000, nf / 10, 0.3 * nf, seed=nf + K)
    q = moved(p, seed=K + 11, frac=1.0, step=2.0)  # |field| / |increment| between 10 and 35
    h, t = make(B, n, pad, p, sigma, mu, a0, box=float(n))
    h.set_option(B.OPT_KEEP_PHI, 1)
    h.enable_increment(True)
    h.deposit()
    h.solve_field(K0, B.WARM_NONE)
    g0 = {f: h.get_field(getattr(B, "FIELD_" + f)).cpu().numpy().astype(np.float64)
          for f in ("ACC", "GN", "H", "GM")}
    # oracle base: its own solve of its own deposit, finished so that H and g_M are those the
    # next solve linearises about
    acc0, ka, rho0 = oracle_rho(p, nf, sigma, s)
    b = oracle.solve(rho0, s, 1.0, a0, mu, K0, finish_h=True, want=("gN", "H", "acc", "gM"))
    assert rel(g0["ACC"], b["acc"]) < TOL
    assert rel(g0["GM"], b["gM"]) < TOL
    assert rel(g0["H"], b["H"], scale=b["gN"]) < TOL
    # the new positions, deposited and solved incrementally
    for k, key in ((0, "cell"), (1, "offset")):
        t[k].copy_(torch.from_numpy(q[key]))
    h.deposit()
    h.solve_field(K, B.WARM_INCREMENT)
    g1 = {f: h.get_field(getattr(B, "FIELD_" + f)).cpu().numpy().astype(np.float64)
          for f in ("ACC", "GN", "H", "GM")}
    acc1, _, _ = oracle_rho(q, nf, sigma, s, ka)
    drho = oracle.delta_rho(acc1, acc0, ka, s)
    inc = oracle.solve_increment(drho, s, 1.0, a0, mu, K, b["gN"], b["H"], b["gM"])
    exp = {"ACC": b["acc"] + inc["dacc"], "GN": b["gN"] + inc["dgN"], "H": b["H"] + inc["dH"],
           "GM": b["gM"] + inc["dgM"]}
    assert rel(g1["ACC"], exp["ACC"]) < TOL
    assert rel(g1["GN"], exp["GN"]) < TOL
    assert rel(g1["GM"], exp["GM"]) < TOL
    assert rel(g1["H"], exp["H"], scale=exp["GN"]) < TOL
    # the increments themselves, against the bar their FP32 difference allows
    for f, d in (("ACC", "dacc"), ("GN", "dgN"), ("GM", "dgM")):
        ratio = np.linalg.norm(exp[f]) / np.linalg.norm(inc[d])
        assert ratio < 100  # a real increment, not rounding
        assert rel(g1[f] - g0[f], inc[d]) < TOL * ratio, f


def test_zero_increment_leaves_fields_bit_for_bit(B):
    n, sigma = 32, 1.5
    p = W.isothermal(n, 1.0, 2000, 3.2, 10.0, seed=5)
    h, _ = make(B, n, 1, p, sigma, 0)
    h.enable_increment(True)
    h.deposit()
    h.solve_field(4, B.WARM_NONE)
    before = {f: h.get_field(f).cpu().numpy().copy() for f in (B.FIELD_ACC, B.FIELD_GN, B.FIELD_H, B.FIELD_GM)}
    h.deposit()  # same positions: the accumulators are equal, the density increment is 0
    h.solve_field(2, B.WARM_INCREMENT)
    for f, v in before.items():
        assert np.array_equal(h.get_field(f).cpu().numpy().view(np.uint32), v.view(np.uint32)), f


def test_newtonian_increment_equals_a_full_solve(B):
    # nu = mu = 1: the incremental solve is exact, so a base plus increment is
    # the full solve of the new density up to FP32 rounding, here on the GPU alone
    n, sigma = 48, 1.5
    p = W.isothermal(n, 1.0, 5000, 4.8, 14.0, seed=6)
    q = moved(p, seed=3, frac=0.5)
    h, t = make(B, n, 1, p, sigma, 3)
    h.enable_increment(True)
    h.deposit()
    h.solve_field(2, B.WARM_NONE)
    for k, key in ((0, "cell"), (1, "offset")):
        t[k].copy_(torch.from_numpy(q[key]))
    h.deposit()
    h.solve_field(2, B.WARM_INCREMENT)
    a_inc = h.get_field(B.FIELD_ACC).cpu().numpy()
    h.solve_field(2, B.WARM_NONE)  # same density: the stored g_N is reused
    a_full = h.get_field(B.FIELD_ACC).cpu().numpy()
    assert rel(a_inc, a_full) < TOL


def test_incremental_steps_graph_equals_direct(B):
    # a captured step replays the same launches: bit-identical particles
    n, sigma = 32, 1.5
    p = W.isothermal(n, 1.0, 3000, 3.2, 10.0, seed=8)
    st = torch.cuda.Stream()
    out = []
    for graph in (0, 1):
        with torch.cuda.stream(st):
            h, t = make(B, n, 1, p, sigma, 0)
        h.enable_increment(True)
        h.set_option(B.OPT_USE_GRAPH, graph)
        h.step(0.25, 4, B.WARM_NONE)
        for _ in range(3):
            h.step(0.25, 1, B.WARM_INCREMENT)
        h.sync()
        out.append([x.cpu().numpy().copy() for x in t[:3]])
    for a, b in zip(*out):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_increment_state_errors(B):
    n, sigma = 16, 1.5
    p = W.isothermal(n, 1.0, 500, 1.6, 5.0, seed=2)
    h, t = make(B, n, 1, p, sigma, 0)
    h.deposit()
    h.solve_field(2, B.WARM_NONE)
    with pytest.raises(B.MondError) as e:  # no workspace
        h.solve_field(1, B.WARM_INCREMENT)
    assert e.value.code == -8
    h.enable_increment(True)
    with pytest.raises(B.MondError) as e:  # attached after the solve: no base yet
        h.solve_field(1, B.WARM_INCREMENT)
    assert e.value.code == -8
    with pytest.raises(B.MondError) as e:
        h.get_field(B.FIELD_GM)
    assert e.value.code == -8
    h.solve_field(2, B.WARM_NONE)
    h.solve_field(1, B.WARM_INCREMENT)  # now there is one
    with pytest.raises(B.MondError) as e:
        h.solve_field(0, B.WARM_INCREMENT)
    assert e.value.code == -1
    h.set_h_state(h.get_field(B.FIELD_H))
    with pytest.raises(B.MondError) as e:  # the H state was replaced
        h.solve_field(1, B.WARM_INCREMENT)
    assert e.value.code == -8
    h.solve_field(2, B.WARM_PREV)
    h.set_option(B.OPT_KEEP_PHI, 1)
    with pytest.raises(B.MondError) as e:  # the base has no potential
        h.step(0.1, 1, B.WARM_INCREMENT)
    assert e.value.code == -8
    h.set_option(B.OPT_KEEP_PHI, 0)
    h.step(0.1, 1, B.WARM_INCREMENT)
    # other masses change the fixed-point scale: the base deposit is not comparable
    heavy = t[3] * 1024
    h.bind_particles(t[0], t[1], t[2], heavy)
    h.deposit()
    with pytest.raises(B.MondError) as e:
        h.solve_field(1, B.WARM_INCREMENT)
    assert e.value.code == -8
    h.sync()
