"""Failure detection and recovery, with every fault made on the host (no
kernel is made to fault, trap or hang), plus the two properties the rest of
the suite leans on: the deposit does not depend on the particles' order (a
lost or doubled atomic add would show), and a run resumes bit for bit from a
checkpoint of its particles and H state."""
import io

import numpy as np
import pytest

import oracle
from paper_2312_02968_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2312_02968_gb300 import binding

    return binding


def make(B, n, p, sigma=1.0, mu=0, maxp=None):
    dev = torch.device("cuda", 0)
    h = B.MondPM(n, 1, float(n), 1.0, 1.0, mu, sigma, maxp or len(p["mass"]))
    t = [torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")]
    h.bind_particles(*t)
    return h, t


def test_deposit_independent_of_particle_order(B):
    n = 32
    p = W.isothermal(n, 1.0, 30000, 3.0, 10.0, seed=5)
    h, _ = make(B, n, p, sigma=1.5)
    h.deposit()
    ref, ka = h.get_deposit_acc()
    ref = ref.cpu().numpy()
    rng = np.random.default_rng(9)
    for _ in range(10):
        perm = rng.permutation(len(p["mass"]))
        q = {k: np.ascontiguousarray(v[perm]) for k, v in p.items()}
        g, _ = make(B, n, q, sigma=1.5)
        g.deposit()
        acc, kb = g.get_deposit_acc()
        assert kb == ka and np.array_equal(acc.cpu().numpy(), ref)
        g.close()
    h.close()


def test_nan_in_the_density_is_reported_and_the_handle_recovers(B):
    n = 32
    p = W.isothermal(n, 1.0, 2000, 3.0, 10.0, seed=6)
    h, _ = make(B, n, p)
    h.deposit()
    rho = h.get_field(B.FIELD_RHO)
    bad = rho.clone()
    bad[5, 6, 7] = float("nan")
    h.set_density(bad)
    h.solve_field(2)
    with pytest.raises(B.MondError) as e:
        h.sync()
    assert e.value.code == -6  # MOND_ENAN
    # the status was read and cleared: a valid density solves again and matches the oracle
    h.set_density(rho)
    h.solve_field(2)
    a = h.get_field(B.FIELD_ACC).cpu().numpy()
    ref = oracle.solve(rho.cpu().numpy().astype(np.float64), 1.0, 1.0, 1.0, 0, 2, want=("acc",))["acc"]
    assert np.linalg.norm(a - ref) / np.linalg.norm(ref) < 1e-5


def test_nan_particle_is_skipped_and_reported(B):
    n = 16
    p = W.isothermal(n, 1.0, 50, 2.0, 5.0, seed=7)
    p["offset"] = p["offset"].copy()
    p["offset"][3, 1] = np.nan
    h, _ = make(B, n, p)
    h.deposit()
    with pytest.raises(B.MondError) as e:
        h.sync()
    assert e.value.code == -5  # MOND_EDOMAIN: the particle was skipped
    acc, ka = h.get_deposit_acc()
    keep = np.ones(50, bool)
    keep[3] = False
    ref, _, _ = oracle.deposit_fixed(n, 1.0, p["cell"][keep], p["offset"][keep], p["mass"][keep], ka)
    assert np.array_equal(acc.cpu().numpy().view(np.uint64), ref)


def test_bad_arguments_are_rejected(B):
    with pytest.raises(B.MondError):
        B.MondPM(100, 1, 100.0, 1.0, 1.0, 0, 1.0, 10)  # unsupported side
    with pytest.raises(B.MondError):
        B.MondPM(32, 1, 32.0, 1.0, 1.0, 0, 0.5, 10)  # kernel narrower than the fixed-point bound allows
    with pytest.raises(B.MondError):
        B.MondPM(32, 3, 32.0, 1.0, 1.0, 0, 1.0, 10)  # padding factor
    n = 16
    p = W.isothermal(n, 1.0, 20, 2.0, 5.0, seed=8)
    h, _ = make(B, n, p)
    with pytest.raises(B.MondError):
        h.solve_field(2)  # before a deposit
    h.deposit()
    with pytest.raises(B.MondError):
        h.solve_field(65)
    with pytest.raises(B.MondError):
        h.set_option(B.OPT_CHUNK, 300)
    h.solve_field(1)  # still usable
    h.close()


@pytest.mark.parametrize("warm", ["none", "prev"])
def test_resume_from_checkpoint_is_bit_identical(B, warm):
    n, dt, K = 32, 0.2, 3
    p = W.isothermal(n, 1.0, 5000, 3.0, 10.0, seed=10)
    w = B.WARM_PREV if warm == "prev" else B.WARM_NONE
    k = 1 if warm == "prev" else K

    def first(h):
        h.deposit()
        h.solve_field(K, B.WARM_NONE)
        h.gather_push(dt)

    h, t = make(B, n, p)
    first(h)
    for _ in range(5):
        h.step(dt, k, w)
    h.sync()
    full = [x.cpu().numpy().copy() for x in t[:3]]
    h.close()

    h1, t1 = make(B, n, p)
    first(h1)
    for _ in range(2):
        h1.step(dt, k, w)
    buf = io.BytesIO()
    h1.checkpoint(buf, step=3)
    h1.close()
    buf.seek(0)
    q = W.isothermal(n, 1.0, 5000, 3.0, 10.0, seed=11)  # other contents, same shapes: all overwritten
    h2, t2 = make(B, n, q)
    assert h2.restore(buf) == 3
    for _ in range(3):
        h2.step(dt, k, w)
    h2.sync()
    for a, b in zip(full, [x.cpu().numpy() for x in t2[:3]]):
        assert np.array_equal(a, b)
    h2.close()


@pytest.mark.parametrize("tile", [0, 400])
def test_lost_tile_copy_times_out_and_the_handle_recovers(B, tile):
    """A bounded device wait that runs out, made without a fault: the test
    hook keeps one tile copy of the next pipelined y-pass from being issued
    (tile 0: the first copy of a CTA; tile 400 of 640 on 128^3: a later one,
    with the CTA's next copy already in flight, which it waits for before it
    stops). The wait for the lost copy gives up after a short bound, the
    solve's next synchronising call reports MOND_ETIMEOUT, and the next solve
    on the same handle matches the oracle."""
    import time

    n = 128
    p = W.isothermal(n, 1.0, 20000, 4.0, 40.0, seed=8)
    h, _ = make(B, n, p)
    h.deposit()
    h.solve_field(2)
    h.sync()
    with pytest.raises(B.MondError):
        h.set_option(B.OPT_USE_GRAPH, 1)
        h.set_option(B.OPT_TEST_LOST_LOAD, tile + 1)  # not with graph replay
    h.set_option(B.OPT_USE_GRAPH, 0)
    h.set_option(B.OPT_TEST_LOST_LOAD, tile + 1)
    t0 = time.perf_counter()
    h.deposit()
    h.solve_field(2)
    with pytest.raises(B.MondError) as e:
        h.sync()
    assert e.value.code == -7  # MOND_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # the hook was one-shot and the status was read and cleared
    h.deposit()
    h.solve_field(2)
    a = h.get_field(B.FIELD_ACC).cpu().numpy()
    rho = h.get_field(B.FIELD_RHO).cpu().numpy().astype(np.float64)
    ref = oracle.solve(rho, 1.0, 1.0, 1.0, 0, 2, want=("acc",))["acc"]
    assert np.linalg.norm(a - ref) / np.linalg.norm(ref) < 1e-5
    h.close()
