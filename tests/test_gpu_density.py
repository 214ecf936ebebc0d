"""Densities from the solver's fields (Eq. apparentdensity) and the masses
they imply (Eq. totalmass), GPU against the oracle.

Two comparisons for each quantity:
- on the same input (the GPU's own FP32 fields, read back): the kernels alone,
  to FP32 rounding of a few differences;
- end to end (the oracle's FP64 solve of the same deposit): the kernels on top
  of the solver's 1e-5 field bar.
Shell membership is decided in IEEE double on both sides, so shell sums agree
to FP64 accumulation order on every bin, including cells whose distance falls
exactly on a shell boundary.
"""
import numpy as np
import pytest

import oracle
from paper_2312_02968_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KINDS = (0, 1, 2)  # baryonic, apparent, phantom


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2312_02968_gb300 import binding

    return binding


def oracle_density(kind, gN, acc, s, G):
    if kind == 0:
        return oracle.field_density(gN, s, G)
    if kind == 1:
        return oracle.field_density(acc, s, G)
    return oracle.field_density(acc, s, G) - oracle.field_density(gN, s, G)


def oracle_box(kind, gN, acc, s, G, lo, hi):
    if kind == 0:
        return oracle.box_flux_mass(gN, s, G, lo, hi)
    if kind == 1:
        return oracle.box_flux_mass(acc, s, G, lo, hi)
    return oracle.box_flux_mass(acc, s, G, lo, hi) - oracle.box_flux_mass(gN, s, G, lo, hi)


@pytest.fixture(scope="module", params=[(48, 1.0, 1.5, 20000, 0), (64, 0.8, 1.0, 60000, 2)],
            ids=["n48", "n64"])
def solved(B, request):
    n, s, sigma, N, mu = request.param
    G, a0 = 1.3, 0.7
    p = W.isothermal(n, s, N, 4.0, 0.35 * n, seed=11)
    dev = torch.device("cuda", 0)
    h = B.MondPM(n, 1, n * s, a0, G, mu, sigma, N)
    t = [torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")]
    h.bind_particles(*t)
    h.deposit()
    h.solve_field(4)
    gN = h.get_field(B.FIELD_GN).cpu().numpy().astype(np.float64)
    acc = h.get_field(B.FIELD_ACC).cpu().numpy().astype(np.float64)
    dep, ka, _ = oracle.deposit_fixed(n, sigma, p["cell"], p["offset"], p["mass"])
    _, rho = oracle.acc_to_rho(dep, ka, s)
    ref = oracle.solve(rho, s, G, a0, mu, 4, want=("gN", "acc"))
    yield dict(h=h, t=t, n=n, s=s, G=G, gN=gN, acc=acc, ref=ref)
    h.close()


@pytest.mark.parametrize("kind", KINDS)
def test_density_same_fields(B, solved, kind):
    d = solved
    got = d["h"].density(kind).cpu().numpy()
    want = oracle_density(kind, d["gN"], d["acc"], d["s"], d["G"])
    assert rel(got, want) < 2e-6
    assert np.max(np.abs(got - want)) < 1e-5 * np.max(np.abs(want))


@pytest.mark.parametrize("kind", KINDS)
def test_density_end_to_end(B, solved, kind):
    d = solved
    got = d["h"].density(kind).cpu().numpy()
    want = oracle_density(kind, d["ref"]["gN"], d["ref"]["acc"], d["s"], d["G"])
    # the divergence weights the field's highest wavenumbers, where the FP32
    # transforms' relative error is largest; 1e-5 on the field becomes a few
    # 1e-5 on its divergence
    assert rel(got, want) < 5e-5


@pytest.mark.parametrize("kind", KINDS)
def test_shell_mass(B, solved, kind):
    d = solved
    n, s = d["n"], d["s"]
    dens_same = oracle_density(kind, d["gN"], d["acc"], s, d["G"])
    # an off-grid centre, and a cell centre with dr = s, where many distances
    # (3-4-0 triples and the axes) fall exactly on shell boundaries
    for center, dr, nb in [([0.37 * s, -1.21 * s, 2.05 * s], 0.7 * s, 60), ([0.0, 0.0, 0.0], s, n),
                           ([-3.0 * s, 5.0 * s, 0.0], 2.0 * s, 4096)]:
        got = np.array(d["h"].shell_mass(kind, center, dr, nb))
        want = oracle.shell_mass(dens_same, s, center, dr, nb)
        scale = np.max(np.abs(want))
        assert np.max(np.abs(got - want)) < 2e-6 * scale, (center, dr)
    # every cell in some shell: the total over the periodic box vanishes
    tot = np.sum(d["h"].shell_mass(kind, [0.0, 0.0, 0.0], s, n))
    assert abs(tot) < 1e-5 * np.abs(dens_same).sum() * s ** 3


@pytest.mark.parametrize("kind", KINDS)
def test_box_mass(B, solved, kind):
    d = solved
    n, s, G = d["n"], d["s"], d["G"]
    h = d["h"]
    boxes = [([n // 4, n // 4, n // 4], [3 * n // 4 - 1, 3 * n // 4 - 1, 3 * n // 4 - 1]),  # the central half
             ([-5, 3, n // 2], [6, n // 2, n // 2 + 9]),  # wraps on x
             ([7, 7, 7], [7, 7, 7]),  # one cell
             ([0, 0, 0], [n - 1, n - 1, n - 1])]  # the whole box: zero
    dens_same = oracle_density(kind, d["gN"], d["acc"], s, G)
    for lo, hi in boxes:
        got = h.box_mass(kind, lo, hi)
        want = oracle_box(kind, d["gN"], d["acc"], s, G, lo, hi)
        # and the discrete Gauss theorem through the GPU's own density
        zi = np.arange(lo[2], hi[2] + 1) % n
        yi = np.arange(lo[1], hi[1] + 1) % n
        xi = np.arange(lo[0], hi[0] + 1) % n
        mag = np.abs(dens_same[np.ix_(zi, yi, xi)]).sum() * s ** 3 + 1e-30
        assert abs(got - want) < 1e-9 * mag + 1e-12, (lo, hi)
        dsum = d["h"].density(kind).cpu().numpy().astype(np.float64)[np.ix_(zi, yi, xi)].sum() * s ** 3
        assert abs(got - dsum) < 1e-5 * mag, (lo, hi)


def test_central_mass_baryonic_vs_deposit(B, solved):
    # the central half of the box holds nearly all particles: its baryonic
    # mass is the deposited mass minus the uniform background the periodic
    # solve removes (the mean density times the box volume)
    d = solved
    n, s = d["n"], d["s"]
    rho = d["h"].get_field(B.FIELD_RHO).cpu().numpy().astype(np.float64)
    lo, hi = [n // 4] * 3, [3 * n // 4 - 1] * 3
    sl = slice(n // 4, 3 * n // 4)
    want = (rho[sl, sl, sl].sum() - rho.mean() * (n // 2) ** 3) * s ** 3
    got = d["h"].box_mass(0, lo, hi)
    assert abs(got / want - 1) < 0.02


def test_errors(B):
    dev = torch.device("cuda", 0)
    n = 16
    p = W.isothermal(n, 1.0, 100, 2.0, 5.0, seed=1)
    h = B.MondPM(n, 1, float(n), 1.0, 1.0, 0, 1.0, 100)
    t = [torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")]
    h.bind_particles(*t)
    with pytest.raises(B.MondError):  # no solve yet
        h.density(1)
    h.deposit()
    h.solve_field(2)
    with pytest.raises(B.MondError):
        h.density(7)
    buf = torch.empty(n ** 3 + 4, dtype=torch.float32, device=dev)
    with pytest.raises(B.MondError):  # misaligned
        h.density(1, out=buf[1:])
    with pytest.raises(B.MondError):
        h.shell_mass(1, [0, 0, 0], 1.0, 0)
    with pytest.raises(B.MondError):
        h.shell_mass(1, [0, 0, 0], 0.0, 4)
    with pytest.raises(B.MondError):
        h.box_mass(1, [0, 0, 0], [n, 0, 0])  # n + 1 cells wide
    with pytest.raises(B.MondError):
        h.box_mass(1, [3, 0, 0], [2, 0, 0])
    # the handle stays usable, and the fields survive a step
    h.density(2)
    h.gather_push(0.1)
    assert np.isfinite(h.density(1).cpu().numpy()).all()
    h.close()


@pytest.mark.parametrize("axis,mu", [(2, 0), (0, 2), (1, 3)])
def test_dipole_layer_solve(B, axis, mu):
    """The external-field dipole layer (Sect. 5.3) in the solve, against the
    oracle's solve of the deposit plus the layer's density."""
    n, s, sigma, N, M = 32, 1.0, 1.0, 3000, 3.0
    p = W.isothermal(n, s, N, 3.0, 0.3 * n, seed=12)
    dev = torch.device("cuda", 0)
    h = B.MondPM(n, 1, n * s, 1.0, 1.0, mu, sigma, N)
    t = [torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")]
    h.bind_particles(*t)
    h.set_dipole_layer(axis, M)
    h.deposit()
    K = 0 if mu == 3 else 4
    h.solve_field(K)
    dep, ka, _ = oracle.deposit_fixed(n, sigma, p["cell"], p["offset"], p["mass"])
    rho32, rho = oracle.acc_to_rho(dep, ka, s)
    # the deposit's own density is untouched by the layer
    assert np.array_equal(h.get_field(B.FIELD_RHO).cpu().numpy(), rho32)
    ref = oracle.solve(rho + oracle.dipole_layer(n, s, axis, M), s, 1.0, 1.0, mu, K, want=("gN", "acc"))
    assert rel(h.get_field(B.FIELD_GN).cpu().numpy(), ref["gN"]) < 1e-5
    assert rel(h.get_field(B.FIELD_ACC).cpu().numpy(), ref["acc"]) < 1e-5
    # removing the layer gives the plain solve back
    h.set_dipole_layer(-1, 0.0)
    h.solve_field(K)
    plain = oracle.solve(rho, s, 1.0, 1.0, mu, K, want=("acc",))["acc"]
    assert rel(h.get_field(B.FIELD_ACC).cpu().numpy(), plain) < 1e-5
    h.close()


def test_dipole_layer_graph_recapture(B):
    n, s, N = 32, 1.0, 2000
    p = W.isothermal(n, s, N, 3.0, 0.3 * n, seed=13)
    st = torch.cuda.Stream()
    out = []
    for masses in ((2.0, 2.0), (2.0, 5.0)):
        with torch.cuda.stream(st):
            h = B.MondPM(n, 1, n * s, 1.0, 1.0, 0, 1.0, N, stream=st)
            t = [torch.from_numpy(np.ascontiguousarray(p[k])).cuda() for k in ("cell", "offset", "vel", "mass")]
        torch.cuda.synchronize()
        h.bind_particles(*t)
        h.set_option(B.OPT_USE_GRAPH, 1)
        for m in masses:
            h.set_dipole_layer(2, m)
            h.step(0.1, 2, B.WARM_NONE)
        h.sync()
        out.append(t[2].cpu().numpy().copy())
        h.close()
    # the second run changed the mass between steps: the replayed graph must see it
    assert not np.array_equal(out[0], out[1])


def test_density_on_a_padded_grid(B):
    # pad = 2: the physical 24^3 box in the middle of a 48^3 periodic domain;
    # the densities cover the whole domain
    n, pad, N = 24, 2, 4000
    nf = n * pad
    p = W.isothermal(nf, 1.0, N, 2.5, 0.2 * nf, seed=14)
    dev = torch.device("cuda", 0)
    h = B.MondPM(n, pad, float(n), 1.0, 1.0, 0, 1.0, N)
    t = [torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")]
    h.bind_particles(*t)
    h.deposit()
    h.solve_field(3)
    gN = h.get_field(B.FIELD_GN).cpu().numpy().astype(np.float64)
    acc = h.get_field(B.FIELD_ACC).cpu().numpy().astype(np.float64)
    for kind in KINDS:
        got = h.density(kind).cpu().numpy()
        assert got.shape == (nf, nf, nf)
        assert rel(got, oracle_density(kind, gN, acc, 1.0, 1.0)) < 2e-6
    lo, hi = [nf // 4] * 3, [3 * nf // 4 - 1] * 3
    assert h.box_mass(1, lo, hi) == pytest.approx(oracle.box_flux_mass(acc, 1.0, 1.0, lo, hi), rel=1e-6)
    h.close()
