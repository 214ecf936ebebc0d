"""GPU path vs the CPU oracle, element by element on the same seeded inputs.

Bars: the deposit is bit-exact (integer accumulator and FP32 density);
fields and forces agree to a relative L2 error of 1e-5 (FP32 transforms
against FP64: about log2(n) rounding steps per transform, 42 transforms, and a
nonlinear step that at most doubles relative errors give a few 1e-6).
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


def force_scale(sigma, acc_mesh, cell, off):
    """Per-particle sum of w |a| over the ball: the size of the terms of Eq. gi.
    FP32 rounding of the mesh is relative to these terms, not to their sum,
    which cancels when a particle's own field dominates its ball."""
    return oracle.gather(sigma, np.abs(acc_mesh), cell, off)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2312_02968_gb300 import binding

    return binding


def make(B, n, pad, p, sigma, mu=0, box=None, a0=1.0, G=1.0, maxp=None):
    dev = torch.device("cuda", 0)
    h = B.MondPM(n, pad, box if box is not None else float(n), a0, G, mu, sigma, maxp or max(1, len(p["mass"])))
    t = [torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")]
    h.bind_particles(*t)
    return h, t


# ---------------------------------------------------------------------------
# deposit: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,sigma,N,seed", [(16, 1.0, 1, 0), (16, 1.5, 37, 1), (32, 1.0, 5000, 2), (32, 2.0, 777, 3),
                                            (32, 1.25, 6000, 7), (48, 1.75, 9000, 8),
                                            (48, 1.5, 20000, 4), (64, 1.0, 100000, 5), (32, 0.75, 3000, 6)])
def test_deposit_bit_exact(B, n, sigma, N, seed):
    p = W.uniform_random(n, N, seed=seed)  # covers the periodic wrap at the faces
    h, _ = make(B, n, 1, p, sigma)
    h.deposit()
    acc, ka = h.get_deposit_acc()
    acc = acc.cpu().numpy().view(np.uint64)
    ref, ka_ref, _ = oracle.deposit_fixed(n, sigma, p["cell"], p["offset"], p["mass"])
    assert ka == ka_ref
    assert np.array_equal(acc, ref)
    rho = h.get_field(B.FIELD_RHO).cpu().numpy()
    r32, _ = oracle.acc_to_rho(ref, ka_ref, 1.0)
    assert np.array_equal(rho.view(np.uint32), r32.view(np.uint32))


def test_deposit_dense_cluster_bit_exact(B):
    """Many particles per tile (shared-memory path) and sparse tiles (global path)."""
    n = 64
    p = W.isothermal(n, 1.0, 200000, 3.0, 25.0, seed=9)
    h, _ = make(B, n, 1, p, 1.5)
    h.deposit()
    acc, ka = h.get_deposit_acc()
    ref, ka_ref, _ = oracle.deposit_fixed(n, 1.5, p["cell"], p["offset"], p["mass"])
    assert ka == ka_ref and np.array_equal(acc.cpu().numpy().view(np.uint64), ref)


@pytest.mark.parametrize("chunk", [256, 4096])
def test_deposit_dense_cells_signed_masses_bit_exact(B, chunk):
    """Work items of up to 4096 particles piled into a few cells, masses of
    both signs and spread exponents: the shared tile's digit planes must sum
    exactly modulo 2^64."""
    n = 32
    rng = np.random.default_rng(17)
    N = 12000
    pos = rng.normal(0.0, 0.6, size=(N, 3))
    cell, off = W.to_cells(pos, n)
    mass = (rng.choice([-1.0, 1.0], N) * np.exp(rng.uniform(-6, 0, N)) / N).astype(np.float32)
    p = {"cell": cell, "offset": off, "vel": np.zeros((N, 3), np.float32), "mass": mass}
    h, _ = make(B, n, 1, p, 1.0)
    h.set_option(B.OPT_CHUNK, chunk)
    h.deposit()
    acc, ka = h.get_deposit_acc()
    ref, ka_ref, _ = oracle.deposit_fixed(n, 1.0, p["cell"], p["offset"], p["mass"])
    assert ka == ka_ref and np.array_equal(acc.cpu().numpy().view(np.uint64), ref)


def test_deposit_edge_cases(B):
    n = 16
    # empty set
    p = W.uniform_random(n, 0, seed=0)
    h, _ = make(B, n, 1, p, 1.0, maxp=4)
    h.deposit()
    acc, _ = h.get_deposit_acc()
    assert int(acc.abs().sum()) == 0
    # offsets exactly +-1/2, all particles in one cell, negative mass
    cell = np.array([[3, 3, 3], [3, 3, 3], [15, 0, 7], [8, 8, 8]], np.int32)
    off = np.array([[0.5, -0.5, 0.5], [-0.5, 0.5, -0.5], [0.4999999, -0.4999999, 0.0], [0, 0, 0]], np.float32)
    mass = np.array([1.0, 2.0, 0.5, -0.25], np.float32)
    p = {"cell": cell, "offset": off, "vel": np.zeros((4, 3), np.float32), "mass": mass}
    h, _ = make(B, n, 1, p, 1.0)
    h.deposit()
    acc, ka = h.get_deposit_acc()
    ref, ka_ref, _ = oracle.deposit_fixed(n, 1.0, cell, off, mass)
    assert ka == ka_ref and np.array_equal(acc.cpu().numpy().view(np.uint64), ref)


def test_empty_particle_set_steps(B):
    """No particles: deposit, solve, gather and push run and leave the
    (empty) state alone; the field of an empty density is zero."""
    n = 32
    p = W.uniform_random(n, 0, seed=0)
    h, _ = make(B, n, 1, p, 1.5, maxp=8)
    h.step(0.5, 4)
    h.sync()
    assert float(h.get_field(B.FIELD_ACC).abs().max()) == 0.0
    h.deposit()  # a step leaves the field stale (the particles moved): solve again before a gather
    h.solve_field(4)
    assert h.gather().numel() == 0


def test_deposit_invalid_particle_reported(B):
    n = 16
    cell = np.array([[3, 3, 3], [16, 0, 0]], np.int32)
    off = np.zeros((2, 3), np.float32)
    p = {"cell": cell, "offset": off, "vel": np.zeros((2, 3), np.float32), "mass": np.ones(2, np.float32)}
    h, _ = make(B, n, 1, p, 1.0)
    h.deposit()
    with pytest.raises(B.MondError) as e:
        h.sync()
    assert e.value.code == -5
    acc, ka = h.get_deposit_acc()
    ref, _, sk = oracle.deposit_fixed(n, 1.0, cell, off, np.ones(2, np.float32), ka)
    assert sk == 1 and np.array_equal(acc.cpu().numpy().view(np.uint64), ref)


# ---------------------------------------------------------------------------
# field solve
# ---------------------------------------------------------------------------
def oracle_fields(p, n, sigma, mu, K, s=1.0, a0=1.0, G=1.0, H0=None, finish=False):
    acc, ka, _ = oracle.deposit_fixed(n, sigma, p["cell"], p["offset"], p["mass"])
    _, rho = oracle.acc_to_rho(acc, ka, s)
    return oracle.solve(rho, s, G, a0, mu, K, H0=H0, finish_h=finish)


@pytest.mark.parametrize("n,mu,K,a0", [(16, 0, 0, 1.0), (32, 0, 1, 1.0), (32, 0, 4, 1.0), (48, 1, 3, 0.05),
                                       (32, 2, 4, 0.02), (32, 3, 2, 1.0), (64, 0, 4, 1.0), (96, 2, 2, 0.05)])
def test_solve_matches_oracle(B, n, mu, K, a0):
    p = W.isothermal(n, 1.0, 4000, n / 10, 0.4 * n, seed=n + K)
    sigma = 1.5
    h, _ = make(B, n, 1, p, sigma, mu=mu, a0=a0)
    h.set_option(B.OPT_KEEP_PHI, 1)
    h.deposit()
    h.solve_field(K)
    ref = oracle_fields(p, n, sigma, mu, K, a0=a0)
    assert rel(h.get_field(B.FIELD_GN).cpu().numpy(), ref["gN"]) < TOL
    assert rel(h.get_field(B.FIELD_ACC).cpu().numpy(), ref["acc"]) < TOL
    assert rel(h.get_field(B.FIELD_PHI).cpu().numpy() - 0, ref["phi"]) < TOL
    if K >= 2:
        # H is the correction in F = g_N + H; its rounding error scales with |F|
        assert rel(h.get_field(B.FIELD_H).cpu().numpy(), ref["H"], scale=ref["gN"]) < TOL


def conditioning(p, n, sigma, mu, K, eps=1e-7):
    """Relative change of the oracle's acceleration mesh when its density is
    perturbed by eps (relative, seeded noise): how much the iteration amplifies
    rounding at the inputs. Near zeros of the field the map is locally unstable,
    so FP32 parity is bounded by a multiple of this, not by FP32 epsilon."""
    acc, ka, _ = oracle.deposit_fixed(n, sigma, p["cell"], p["offset"], p["mass"])
    _, rho = oracle.acc_to_rho(acc, ka, 1.0)
    a = oracle.solve(rho, 1.0, 1.0, 1.0, mu, K, want=("acc",))["acc"]
    noise = np.random.default_rng(0).standard_normal(rho.shape)
    b = oracle.solve(rho * (1 + eps * noise), 1.0, 1.0, 1.0, mu, K, want=("acc",))["acc"]
    return rel(b, a)


def test_solve_padded_grid_two_body(B):
    """pad = 2: 64^3 physical mesh in a 128^3 periodic domain (the two-body set-up).
    Here the iteration amplifies input rounding about 400-fold by K = 4, so the
    bar is the larger of 1e-5 and four times the oracle's own sensitivity."""
    n, pad, sigma = 64, 2, 2.0
    p, _ = W.two_body(n * pad, 1.0, 16.0, 0.5, 0.5)
    h, _ = make(B, n, pad, p, sigma, mu=1, box=64.0)
    h.deposit()
    h.solve_field(4)
    g = h.gather().cpu().numpy()
    ref = oracle_fields(p, n * pad, sigma, 1, 4)
    g_ref = oracle.gather(sigma, ref["acc"], p["cell"], p["offset"])
    tol = max(TOL, 4 * conditioning(p, n * pad, sigma, 1, 4))
    assert tol < 5e-4
    assert rel(h.get_field(B.FIELD_ACC).cpu().numpy(), ref["acc"]) < tol
    assert rel(g, g_ref, scale=force_scale(sigma, ref["acc"], p["cell"], p["offset"])) < tol
    assert rel(g, g_ref) < 10 * tol  # the two self-fields cancel to about 1/10 of the ball terms


@pytest.mark.parametrize("warm", ["prev", "guess", "guess_raw"])
def test_warm_start_matches_oracle(B, warm):
    n, sigma, mu = 32, 1.5, 0
    p = W.isothermal(n, 1.0, 3000, 3.0, 12.0, seed=21)
    h, _ = make(B, n, 1, p, sigma, mu=mu)
    h.deposit()
    if warm == "prev":
        h.solve_field(3)  # leaves the H of its iteration 2
        H0 = h.get_field(B.FIELD_H).cpu().numpy().astype(np.float64)
        h.solve_field(1, B.WARM_PREV)
    else:
        rng = np.random.default_rng(3)
        guess = (1e-3 * rng.standard_normal((3, n, n, n))).astype(np.float32)
        if warm == "guess":
            h.solve_field(1, B.WARM_GUESS, torch.from_numpy(guess).cuda())
            H0 = oracle.project_div(guess.astype(np.float64), 1.0)
        else:
            h.solve_field(1, B.WARM_GUESS_RAW, torch.from_numpy(guess).cuda())
            H0 = guess.astype(np.float64)
    ref = oracle_fields(p, n, sigma, mu, 1, H0=H0, finish=True)
    assert rel(h.get_field(B.FIELD_ACC).cpu().numpy(), ref["acc"]) < TOL
    if warm != "guess_raw":  # a raw guess is used once and leaves no H state
        assert rel(h.get_field(B.FIELD_H).cpu().numpy(), ref["H"], scale=ref["gN"]) < TOL


def test_newton_field_reused_within_one_density(B):
    """A second solve on the same density starts from the stored g_N and gives
    the same acceleration bit for bit; a density uploaded with set_density
    equal to the deposit's gives the same result up to the rounding of a
    differently compiled x-transform (the compiler may contract a*b+c
    differently in the two kernels)."""
    n, sigma = 32, 1.5
    p = W.isothermal(n, 1.0, 4000, 3.0, 12.0, seed=23)
    h, _ = make(B, n, 1, p, sigma, mu=2)
    h.deposit()
    h.solve_field(4)
    a1 = h.get_field(B.FIELD_ACC).cpu().numpy()
    h.solve_field(4)
    a2 = h.get_field(B.FIELD_ACC).cpu().numpy()
    rho = h.get_field(B.FIELD_RHO).clone()
    h.set_density(rho)
    h.solve_field(4)
    a3 = h.get_field(B.FIELD_ACC).cpu().numpy()
    assert np.array_equal(a1, a2)
    assert rel(a3, a1) < 1e-6


# ---------------------------------------------------------------------------
# gather, smoothing, push, diagnostics
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("sigma", [0.75, 1.0, 1.25, 1.5, 1.75, 2.0])  # reach r = 2 .. 7: every kernel variant
def test_gather_matches_oracle(B, sigma):
    n = 32
    p = W.uniform_random(n, 3000, seed=int(10 * sigma))  # includes particles whose ball wraps
    h, _ = make(B, n, 1, p, sigma)
    h.deposit()
    h.solve_field(2)
    g = h.gather().cpu().numpy()
    ref = oracle_fields(p, n, sigma, 0, 2)
    g_ref = oracle.gather(sigma, ref["acc"], p["cell"], p["offset"])
    assert rel(g, g_ref) < TOL


def test_smooth_is_gather_at_nodes(B):
    """Node-smoothed field = Eq. gi for a particle sitting on each pixel centre."""
    n, sigma = 16, 1.0
    p = W.uniform_random(n, 500, seed=4)
    h, _ = make(B, n, 1, p, sigma)
    h.deposit()
    h.solve_field(2)
    h.smooth()
    sm = h.get_field(B.FIELD_SMOOTH).cpu().numpy()
    ref = oracle_fields(p, n, sigma, 0, 2)
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cells = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(np.int32)
    g = oracle.gather(sigma, ref["acc"], cells, np.zeros_like(cells, dtype=np.float32))
    want = np.stack([g[:, a].reshape(n, n, n) for a in range(3)])
    assert rel(sm, want) < TOL


def test_step_kick_drift_matches_oracle(B):
    n, sigma, dt = 32, 1.5, 0.5
    p = W.isothermal(n, 1.0, 2000, 3.0, 12.0, seed=5)
    h, t = make(B, n, 1, p, sigma)
    h.step(dt, 4)
    h.sync()
    c2, o2, v2, g, _, _ = oracle.step(n, 1.0, 1.0, 1.0, 0, sigma, 4, dt, p["cell"], p["offset"], p["vel"], p["mass"])
    vel = t[2].cpu().numpy()
    assert rel(vel - p["vel"], v2 - p["vel"]) < TOL
    pos = t[0].cpu().numpy() + t[1].cpu().numpy().astype(np.float64)
    pos_ref = c2 + o2
    d = np.abs(((pos - pos_ref) + n / 2) % n - n / 2)
    assert d.max() < 1e-5
    assert np.all(np.abs(t[1].cpu().numpy()) <= 0.5)


def test_half_kick_and_diagnostics(B):
    n = 64
    p, meta = W.two_body(n, 1.0, 16.0, 0.6, 0.4)
    h, t = make(B, n, 1, p, 1.0)
    d = h.diagnostics()
    ref = oracle.particle_diag(n, 1.0, p["cell"], p["offset"], p["vel"], p["mass"])
    assert abs(d["mass"] - ref["mass"]) < 1e-12
    assert np.allclose(d["momentum"], ref["P"], atol=1e-9)
    assert np.allclose(d["com"], ref["R"], atol=1e-9)
    assert np.allclose(d["ang_mom"], ref["L"], rtol=1e-9, atol=1e-12)
    assert abs(d["e_kin"] - ref["Ekin"]) < 1e-12
    h.deposit()
    h.solve_field(2)
    h.half_kick(0.1)
    v = t[2].cpu().numpy()
    ref_f = oracle_fields(p, n, 1.0, 0, 2)
    g = oracle.gather(1.0, ref_f["acc"], p["cell"], p["offset"])
    assert rel(v - p["vel"], 0.1 * g) < TOL
    assert np.array_equal(t[0].cpu().numpy(), p["cell"])  # no drift


def test_track_dh(B):
    n = 32
    p = W.isothermal(n, 1.0, 3000, 3.0, 12.0, seed=8)
    h, _ = make(B, n, 1, p, 1.5)
    h.set_option(B.OPT_TRACK_DH, 1)
    h.deposit()
    h.solve_field(5)
    d = h.diagnostics()
    dh = np.array(d["dH"][:4])
    assert np.all(np.isfinite(dh)) and dh[1] < dh[0]
    assert np.isnan(d["dH"][4])


@pytest.mark.parametrize("n,mu,K", [(32, 0, 0), (32, 0, 4), (48, 2, 3), (64, 1, 2)])
def test_pipelined_passes_match_unpipelined(B, n, mu, K):
    """The TMA-pipelined y/z passes do the same arithmetic per element as the
    one-tile-per-CTA passes; only the compiler's fused multiply-add choices
    differ. Fields agree to FP32 rounding; H, a difference field, carries
    that rounding amplified, so the bar is the parity bar of 1e-5."""
    p = W.isothermal(n, 1.0, 3000, n / 10, 0.4 * n, seed=n + 7)
    out = []
    for pipe in (0, 1):
        h, _ = make(B, n, 1, p, 1.5, mu=mu, a0=0.05 if mu else 1.0)
        h.set_option(B.OPT_PIPELINED, pipe)
        h.set_option(B.OPT_KEEP_PHI, 1)
        h.deposit()
        h.solve_field(K)
        f = [h.get_field(B.FIELD_ACC).cpu(), h.get_field(B.FIELD_PHI).cpu(), h.get_field(B.FIELD_GN).cpu()]
        if K > 0:
            g = torch.from_numpy((1e-3 * np.random.default_rng(1).standard_normal((3, n, n, n))).astype(np.float32))
            h.solve_field(1, B.WARM_GUESS, g.cuda())
            h.smooth()
            f += [h.get_field(B.FIELD_ACC).cpu(), h.get_field(B.FIELD_H).cpu(), h.get_field(B.FIELD_SMOOTH).cpu()]
        out.append(f)
    for a, b in zip(out[0], out[1]):
        assert rel(a.numpy(), b.numpy()) < TOL


@pytest.mark.parametrize("n,mu,K,keep_phi,warm", [(32, 0, 2, 1, False), (64, 0, 4, 0, False), (48, 2, 3, 1, False),
                                                  (32, 0, 2, 1, True), (128, 0, 4, 0, False)])
def test_cycle_mean_matches_oracle(B, n, mu, K, keep_phi, warm):
    """MOND_OPT_CYCLE_MEAN: the potential is the mean of the last two
    iterations' (the midpoint of the period-2 cycle of reading R14), the
    oracle's mean_last2, for plain and previous-H warm-started solves, with
    and without the potential plane; 128^3 spans several z-pass tiles."""
    p = W.isothermal(n, 1.0, 6000, n / 12, 0.4 * n, seed=n + 3 * K)
    sigma = 1.5
    h, _ = make(B, n, 1, p, sigma, mu=mu, a0=1.0 if mu == 0 else 0.05)
    h.set_option(B.OPT_KEEP_PHI, keep_phi)
    h.set_option(B.OPT_CYCLE_MEAN, 1)
    h.deposit()
    H0 = None
    if warm:
        h.solve_field(3)
        H0 = h.get_field(B.FIELD_H).cpu().numpy().astype(np.float64)
        h.solve_field(K, B.WARM_PREV)
    else:
        h.solve_field(K)
    acc, ka, _ = oracle.deposit_fixed(n, sigma, p["cell"], p["offset"], p["mass"])
    rho = oracle.acc_to_rho(acc, ka, 1.0)[0].astype(np.float64)
    ref = oracle.solve(rho, 1.0, 1.0, 1.0 if mu == 0 else 0.05, mu, K, H0=H0, finish_h=warm, mean_last2=True)
    assert rel(h.get_field(B.FIELD_ACC).cpu().numpy(), ref["acc"]) < TOL
    if keep_phi:
        assert rel(h.get_field(B.FIELD_PHI).cpu().numpy(), ref["phi"]) < TOL
    plain = oracle.solve(rho, 1.0, 1.0, 1.0 if mu == 0 else 0.05, mu, K, H0=H0, finish_h=warm, want=("acc",))
    assert rel(plain["acc"], ref["acc"]) > 10 * TOL  # the option changes the result
    if not warm:  # off again: the plain solve
        h.set_option(B.OPT_CYCLE_MEAN, 0)
        h.solve_field(K)
        assert rel(h.get_field(B.FIELD_ACC).cpu().numpy(), plain["acc"]) < TOL


@pytest.mark.parametrize("box_over_n", [1.0, 0.5, 0.7])
def test_density_rule_bit_exact_at_extreme_totals(B, box_over_n):
    """The deposit's FP32 density, float(double(acc) 2^-Kacc / s^3), bit for bit
    against the oracle's, where the totals reach the ends of their range: one
    pile of the largest masses in one cell (its total past the 53 bits of a
    double), one lone particle, masses of both signs, and empty neighbours.
    Pixel widths 1 and 0.5 make the scale a power of two (the x-pass rounds on
    the integer), 0.7 does not (it takes the FP64 route)."""
    n = 32
    rng = np.random.default_rng(23)
    pos = np.concatenate([np.zeros((1, 3)), rng.normal(0.0, 0.3, size=(3000, 3)) + 5.0,
                          rng.uniform(-14, 14, size=(500, 3))])
    cell, off = W.to_cells(pos, n)
    mass = np.concatenate([[1.0], np.full(3000, 1.0), rng.choice([-1.0, 1.0], 500) * np.exp(rng.uniform(-12, 0, 500))])
    p = {"cell": cell, "offset": off, "vel": np.zeros((len(mass), 3), np.float32), "mass": mass.astype(np.float32)}
    dev = torch.device("cuda", 0)
    t = [torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")]
    s = box_over_n
    h = B.MondPM(n, 1, n * s, 1.0, 1.0, 0, 1.5, len(mass))
    h.bind_particles(*t)
    h.deposit()
    acc, ka = h.get_deposit_acc()
    ref, ka_ref, _ = oracle.deposit_fixed(n, 1.5, p["cell"], p["offset"], p["mass"])
    assert ka == ka_ref and np.array_equal(acc.cpu().numpy().view(np.uint64), ref)
    assert int(np.abs(ref.view(np.int64)).max()) > 2 ** 53  # the double rounding is exercised
    rho = h.get_field(B.FIELD_RHO).cpu().numpy()
    r32, _ = oracle.acc_to_rho(ref, ka_ref, s)
    assert np.array_equal(rho.view(np.uint32), r32.view(np.uint32))
    h.close()


@pytest.mark.parametrize("n,mu,K,keep_phi,mean,gather", [(32, 0, 0, 1, 0, 0), (64, 0, 4, 1, 1, 0), (96, 2, 3, 0, 0, 0),
                                                         (128, 0, 4, 0, 1, 0), (64, 1, 2, 1, 0, 3),
                                                         (192, 0, 2, 0, 1, 0)])
def test_folded_passes_match_oracle(B, n, mu, K, keep_phi, mean, gather):
    """MOND_OPT_FOLD (the default): the curl-free, final and Newton steps carry
    one scalar and its z-derivative between their y- and z-passes, the tiles on
    the Nyquist planes of x and y three components as before. Against the
    oracle at the parity bar, and against the three-component passes to FP32
    rounding, for the Newton-only solve, the mean of the last two iterations,
    the potential plane and the smoothing spectrum of the interpolating gather;
    192^3 spans many tiles of both passes and a ragged last z-block."""
    p = W.isothermal(n, 1.0, 5000, n / 11, 0.4 * n, seed=n + K + 17)
    sigma = 1.5
    a0 = 1.0 if mu == 0 else 0.05
    fields = []
    for fold in (1, 0):
        h, _ = make(B, n, 1, p, sigma, mu=mu, a0=a0)
        h.set_option(B.OPT_FOLD, fold)
        h.set_option(B.OPT_KEEP_PHI, keep_phi)
        h.set_option(B.OPT_CYCLE_MEAN, mean)
        h.set_option(B.OPT_GATHER, gather)
        h.deposit()
        h.solve_field(K)
        f = [h.get_field(B.FIELD_ACC).cpu().numpy(), h.get_field(B.FIELD_GN).cpu().numpy()]
        if keep_phi:
            f.append(h.get_field(B.FIELD_PHI).cpu().numpy())
        if K >= 2:
            f.append(h.get_field(B.FIELD_H).cpu().numpy())
        fields.append(f)
    nh = 1 if K >= 2 else 0  # H last: its rounding scales with g_N
    for a, b in zip(fields[0][:len(fields[0]) - nh], fields[1]):
        assert rel(a, b) < TOL / 4
    if nh:
        assert rel(fields[0][-1], fields[1][-1], scale=fields[1][1]) < TOL / 4
    acc, ka, _ = oracle.deposit_fixed(n, sigma, p["cell"], p["offset"], p["mass"])
    rho = oracle.acc_to_rho(acc, ka, 1.0)[0].astype(np.float64)
    ref = oracle.solve(rho, 1.0, 1.0, a0, mu, K, mean_last2=bool(mean) and K >= 2, want=("acc", "gN", "phi", "H"))
    acc_ref = oracle.node_smoothed(sigma, ref["acc"]) if gather else ref["acc"]
    assert rel(fields[0][0], acc_ref) < TOL
    assert rel(fields[0][1], ref["gN"]) < TOL
    if keep_phi:
        assert rel(fields[0][2], ref["phi"]) < TOL
    if nh:
        assert rel(fields[0][-1], ref["H"], scale=ref["gN"]) < TOL


@pytest.mark.parametrize("cap", [7, 152])
def test_grid_cap_changes_nothing(B, cap):
    """MOND_OPT_GRID_CAP: the persistent kernels with fewer CTAs take more
    tiles or work items each; a step gives the same bits (each tile's
    arithmetic and the integer deposit do not depend on which CTA runs them)."""
    n = 64
    p = W.isothermal(n, 1.0, 20000, n / 10, 0.4 * n, seed=41)
    out = []
    for c in (0, cap):
        h, t = make(B, n, 1, p, 1.5)
        h.set_option(B.OPT_GRID_CAP, c)
        h.set_option(B.OPT_CYCLE_MEAN, 1)
        h.deposit()
        acc_dep = h.get_deposit_acc()[0].cpu().numpy()
        h.solve_field(4)
        h.gather_push(0.25)
        h.sync()
        out.append([acc_dep, h.get_field(B.FIELD_ACC).cpu().numpy(), t[0].cpu().numpy(), t[1].cpu().numpy(),
                    t[2].cpu().numpy()])
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [384, 512])
def test_folded_passes_match_three_component_passes_at_large_sides(B, n):
    """At the sides with 8-column y tiles and 4-column folded tiles (n >= 384)
    the folded passes agree with the three-component ones to FP32 rounding
    (the oracle at these sides is covered through the ring configuration)."""
    p = W.isothermal(n, 1.0, 20000, n / 16, 0.4 * n, seed=n + 5)
    fields = []
    for fold in (1, 0):
        h, _ = make(B, n, 1, p, 1.5)
        h.set_option(B.OPT_FOLD, fold)
        h.set_option(B.OPT_KEEP_PHI, 1)
        h.set_option(B.OPT_CYCLE_MEAN, 1)
        h.deposit()
        h.solve_field(3)
        fields.append([h.get_field(B.FIELD_ACC).cpu().numpy(), h.get_field(B.FIELD_PHI).cpu().numpy(),
                       h.get_field(B.FIELD_GN).cpu().numpy()])
        h.close()
    for a, b in zip(fields[0], fields[1]):
        assert rel(a, b) < TOL / 4
