"""Captured steps and batches: a step replayed from a CUDA graph, a batch of
systems of different sizes stepped as one graph, and every work-item size and
pass variant the autotuner chooses between give the same particle state as
direct launches (bit for bit: the deposit is exact, the gather sums each
particle's taps in a fixed order and the launches are the same); the two
pass variants agree to FP32 rounding."""
import numpy as np
import pytest

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


def system(B, n, N, seed, mu, stream):
    p = W.isothermal(n, 1.0, N, n / 32, 0.4 * n, seed=seed) if mu == B.MU_DEEP else \
        W.sphere_mixture(n, N, seed, n_spheres=1)[0]
    with torch.cuda.stream(stream):
        h = B.MondPM(n, 1, float(n), 1.0, 1.0, mu, 1.0, N, stream=stream)
        t = [torch.from_numpy(np.ascontiguousarray(p[k])).cuda() for k in ("cell", "offset", "vel", "mass")]
    torch.cuda.synchronize()
    h.bind_particles(*t)
    return h, t


def state(t):
    torch.cuda.synchronize()
    return [x.cpu().numpy().copy() for x in t[:3]]


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_graph_step_matches_direct_steps(B):
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    h1, t1 = system(B, 64, 20000, 3, B.MU_DEEP, s1)
    h2, t2 = system(B, 64, 20000, 3, B.MU_DEEP, s2)
    h2.set_option(B.OPT_USE_GRAPH, 1)
    for _ in range(3):
        h1.step(0.5, 4, B.WARM_NONE)
        h2.step(0.5, 4, B.WARM_NONE)
    h1.sync()
    h2.sync()
    assert same(state(t1), state(t2))
    # a changed argument recaptures
    h1.step(0.25, 2, B.WARM_NONE)
    h2.step(0.25, 2, B.WARM_NONE)
    h1.sync()
    h2.sync()
    assert same(state(t1), state(t2))
    assert h2.kernel_launches() == h1.kernel_launches()


def test_batch_of_uneven_systems_matches_individual_steps(B):
    sizes = [(64, 30000, 11, B.MU_DEEP), (96, 50000, 12, B.MU_STANDARD), (48, 8000, 13, B.MU_DEEP),
             (128, 60000, 14, B.MU_STANDARD)]
    ref, bat = [], []
    for n, N, sd, mu in sizes:
        ref.append(system(B, n, N, sd, mu, torch.cuda.Stream()))
        bat.append(system(B, n, N, sd, mu, torch.cuda.Stream()))
    for h, _ in ref:
        for _ in range(4):
            h.step(0.5, 4, B.WARM_NONE)
        h.sync()
    batch = B.Batch([h for h, _ in bat])
    batch.step(0.5, n_steps=3, n_iter=4)
    batch.step(0.5, n_steps=1, n_iter=4)
    batch.sync()
    for (h, t), (hr, tr) in zip(bat, ref):
        assert same(state(t), state(tr))
    assert batch.kernel_launches() > 0
    batch.close()


def test_batch_of_incremental_steps_matches_individual_steps(B):
    # members with an increment workspace: one full step, then incremental
    # steps (Sect. 5.2 v), in one graph per step against each stepped alone
    sizes = [(64, 20000, 31, B.MU_DEEP), (96, 30000, 32, B.MU_STANDARD)]
    ref, bat = [], []
    for n, N, sd, mu in sizes:
        ref.append(system(B, n, N, sd, mu, torch.cuda.Stream()))
        bat.append(system(B, n, N, sd, mu, torch.cuda.Stream()))
    for h, _ in ref + bat:
        h.enable_increment(True)
    for h, _ in ref:
        h.step(0.5, 4, B.WARM_NONE)
        for _ in range(3):
            h.step(0.5, 1, B.WARM_INCREMENT)
        h.sync()
    batch = B.Batch([h for h, _ in bat])
    batch.step(0.5, n_steps=1, n_iter=4)
    batch.step(0.5, n_steps=3, n_iter=1, warm=B.WARM_INCREMENT)
    batch.sync()
    for (h, t), (hr, tr) in zip(bat, ref):
        assert same(state(t), state(tr))
    batch.close()


def test_autotune_choices_give_identical_states(B):
    s = torch.cuda.Stream()
    h, t = system(B, 96, 40000, 21, B.MU_DEEP, s)
    before = state(t)
    chunk, pipe = B.autotune(h, n_iter=4, trials=2)
    assert chunk in (512, 1024, 2048, 4096) and pipe in (0, 1)
    assert same(state(t), before)  # zero-length trial steps move nothing

    def run(c, p):
        hh, tt = system(B, 96, 40000, 21, B.MU_DEEP, torch.cuda.Stream())
        hh.set_option(B.OPT_CHUNK, c)
        hh.set_option(B.OPT_PIPELINED, p)
        for _ in range(2):
            hh.step(0.5, 4, B.WARM_NONE)
        hh.sync()
        return state(tt)

    # the work-item size changes nothing
    for p in (0, 1):
        assert same(run(512, p), run(4096, p))
    # the two pass variants differ only by FP32 rounding (the compiler may
    # contract a*b+c differently in the two kernels)
    a, b = run(chunk, 0), run(chunk, 1)
    pa = a[0] + a[1].astype(np.float64)
    pb = b[0] + b[1].astype(np.float64)
    assert np.max(np.abs(pa - pb)) < 1e-4
    assert np.linalg.norm(a[2] - b[2]) <= 1e-5 * np.linalg.norm(a[2])


def test_autotune_cache(B, tmp_path):
    # a second handle of the same key takes the stored choice without timing
    n = 32
    p = W.isothermal(n, 1.0, 20000, 3.0, 10.0, seed=21)
    cache = str(tmp_path / "tune.json")
    st = torch.cuda.Stream()
    hs = []
    for _ in range(2):
        with torch.cuda.stream(st):
            h = B.MondPM(n, 1, float(n), 1.0, 1.0, 0, 1.0, len(p["mass"]), stream=st)
            t = [torch.from_numpy(np.ascontiguousarray(p[k])).cuda() for k in ("cell", "offset", "vel", "mass")]
        torch.cuda.synchronize()
        h.bind_particles(*t)
        hs.append((h, t))
    first = B.autotune(hs[0][0], 2, 2, cache=cache)
    import json

    table = json.load(open(cache))
    assert list(table.values()) == [{"chunk": first[0], "pipelined": first[1]}]
    l0 = hs[1][0].kernel_launches()
    second = B.autotune(hs[1][0], 2, 2, cache=cache)
    assert second == first and hs[1][0].kernel_launches() == l0  # nothing was timed
    for h, _ in hs:
        h.close()


@pytest.mark.parametrize("graph", [0, 1])
def test_step_host_matches_device_steps(B, graph):
    """mond_pm_step_host (the particle state in and out through pinned host
    buffers, the velocities uploaded on a copy stream beside the deposit and
    the solve, the gather waiting for them) gives the particle state of
    mond_pm_step on device buffers, bit for bit, direct and captured."""
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    h1, t1 = system(B, 64, 20000, 5, B.MU_DEEP, s1)
    h2, t2 = system(B, 64, 20000, 5, B.MU_DEEP, s2)
    h2.set_option(B.OPT_USE_GRAPH, graph)
    host = [x.cpu().pin_memory() for x in t2[:3]]
    for _ in range(3):
        h1.step(0.5, 4, B.WARM_NONE)
        h2.step_host(0.5, 4, B.WARM_NONE, *host)
    h1.sync()
    assert same(state(t1), [x.numpy() for x in host])
    # device steps on the same handle afterwards (a different captured step) continue from it
    h1.step(0.5, 4, B.WARM_NONE)
    h2.step(0.5, 4, B.WARM_NONE)
    h1.sync()
    h2.sync()
    assert same(state(t1), state(t2))
