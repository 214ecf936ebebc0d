"""Parity of the surrogate's CUDA kernels (include/mond_fno.h) with the FP64
FNO oracle: bfloat16 cast bit for bit; forward, gradients, loss, Adam and the
mesh <-> network-grid maps to FP32 tolerances. Both sides use the same
bfloat16-rounded weights, so the differences are FP32 accumulation only."""
import numpy as np
import pytest

from oracle import fno_oracle as F

pytestmark = pytest.mark.gpu

SHAPES = [(8, 4, 2, 2), (16, 8, 4, 3), (24, 6, 5, 2), (64, 32, 16, 4)]


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2312_02968_gb300 import surrogate as S

    return torch, S


def rel(a, b):
    a = np.asarray(a)
    a = a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rand_params(sh, seed):
    """Random weights with the spectral and the pointwise paths of each layer
    of comparable size on white-noise input."""
    rng = np.random.default_rng(seed)
    d = {"P": rng.normal(0, 0.5, (sh.C, 4)), "p": rng.normal(0, 0.1, sh.C), "W": [], "b": [], "R": [],
         "Q": rng.normal(0, 1 / np.sqrt(sh.C), (3, sh.C)), "q": rng.normal(0, 0.1, 3)}
    sr = 0.5 * np.sqrt(sh.V / (2.0 * sh.K * sh.C))
    for _ in range(sh.L):
        d["W"].append(rng.normal(0, 0.7 / np.sqrt(sh.C), (sh.C, sh.C)))
        d["b"].append(rng.normal(0, 0.1, sh.C))
        d["R"].append(rng.normal(0, sr, (sh.K, sh.C, sh.C)) + 1j * rng.normal(0, sr, (sh.K, sh.C, sh.C)))
    return F.pack(d, sh).astype(np.float32)


def make(env, shape, seed=3):
    torch, S = env
    net = S.FNO(*shape, seed=seed, device="cuda:0")
    p = rand_params(F.Shape(*shape), seed)
    net.load(torch.from_numpy(p).cuda())
    torch.cuda.synchronize()
    return net, F.bf16_round(p)


def test_cast_is_bit_exact(env):
    torch, S = env
    net = S.FNO(8, 4, 2, 2, seed=1, device="cuda:0")
    rng = np.random.default_rng(0)
    vals = (rng.normal(size=net.count) * np.exp(rng.uniform(-30, 30, net.count))).astype(np.float32)
    net.params.copy_(torch.from_numpy(vals))
    net.cast()
    torch.cuda.synchronize()
    got = net.params_bf16.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    want = F.bf16_round(vals).astype(np.float32).view(np.uint32)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_and_gradients_match_oracle(env, shape):
    torch, S = env
    n, C, M, L = shape
    net, flat = make(env, shape)
    sh = F.Shape(n, C, M, L)
    rng = np.random.default_rng(n + C)
    x = rng.normal(size=(4, n, n, n)).astype(np.float32)
    t = rng.normal(size=(3, n, n, n)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    y = torch.empty_like(td)
    dy = torch.empty_like(td)
    net.forward(xd, y)
    net.loss_acc.zero_()
    net.loss(y, td, dy, 0.5)
    net.grad.zero_()
    net.backward(xd, dy)
    torch.cuda.synchronize()
    y_o, cache = F.forward(flat, x, sh)
    ey = rel(y.cpu().numpy(), y_o)
    assert ey < 2e-5, ey
    # gradient of the oracle loss at the GPU's output (the FP32 forward error
    # would otherwise enter dy at relative size ey / |y - t|)
    L_o, dy_o = F.loss(y.cpu().numpy().astype(np.float64), t, 0.5)
    assert float(net.loss_acc[0].item()) == pytest.approx(L_o, rel=1e-6)
    assert rel(dy.cpu().numpy(), dy_o) < 1e-6
    g_o = F.backward(flat, cache, dy.cpu().numpy().astype(np.float64), sh)
    g = net.grad.cpu().numpy()
    go = F.unpack(g_o, sh)
    gg = F.unpack(g, sh)
    for key in ("P", "p", "Q", "q"):
        assert rel(gg[key], go[key]) < 5e-5, key
    for l in range(L):
        for key in ("W", "b", "R"):
            e = rel(gg[key][l], go[key][l])
            assert e < 5e-5, (key, l, e)


def test_adam_matches_oracle(env):
    torch, S = env
    net = S.FNO(8, 4, 2, 2, seed=2, device="cuda:0")
    rng = np.random.default_rng(9)
    p0 = net.params.cpu().numpy().astype(np.float64)
    m = np.zeros(net.count)
    v = np.zeros(net.count)
    p = p0.copy()
    for step in range(1, 4):
        g = rng.normal(size=net.count).astype(np.float32)
        net.grad.copy_(torch.from_numpy(g))
        net.adam(1e-2, 0.9, 0.99, 1e-6)
        p, m, v = F.adam(p, g.astype(np.float64), m, v, 1e-2, 0.9, 0.99, 1e-6, step)
    torch.cuda.synchronize()
    assert np.max(np.abs(net.params.cpu().numpy() - p)) < 1e-6
    assert float(net.grad.abs().max()) == 0.0


def test_features_upsample_coarsen_mixture(env):
    torch, S = env
    N, n = 64, 16
    st = torch.cuda.current_stream()
    rng = np.random.default_rng(11)
    g = rng.normal(size=(3, N, N, N)).astype(np.float32)
    g[0] += 2.0
    gd = torch.from_numpy(g).cuda()
    x = torch.empty((4, n, n, n), device="cuda")
    scale = torch.empty(4, device="cuda")
    S.features(gd, N, n, 0.7, x, scale, st)
    torch.cuda.synchronize()
    x_o, s_o = F.features(g.astype(np.float64), n, 0.7)
    assert float(scale[0]) == pytest.approx(s_o, rel=1e-6)
    assert rel(x.cpu().numpy(), x_o) < 1e-6
    y = rng.normal(size=(3, n, n, n)).astype(np.float32)
    H = torch.empty((3, N, N, N), device="cuda")
    S.upsample(torch.from_numpy(y).cuda(), N, n, scale, H, st)
    c = torch.empty((3, n, n, n), device="cuda")
    g2 = rng.normal(size=(3, N, N, N)).astype(np.float32)
    S.coarsen(gd, N, n, 3, c, scale, st, fine2=torch.from_numpy(g2).cuda())
    torch.cuda.synchronize()
    assert rel(H.cpu().numpy(), F.upsample(y.astype(np.float64), N, float(scale[0]))) < 1e-6
    want = F.coarsen(0.5 * (g.astype(np.float64) + g2), n) / float(scale[0])
    assert rel(c.cpu().numpy(), want) < 1e-6
    sp = {"centre": np.array([[3.0, -5.0, 2.0], [-10.0, 4.0, 0.0]]), "mass": np.array([0.3, 0.05]),
          "radius": np.array([6.0, 9.5]), "kind": np.array([0, 1])}
    rho = torch.empty((N, N, N), device="cuda")
    keep = S.mixture_density(N, 0.5, sp, 25.6, rho, st)
    torch.cuda.synchronize()
    del keep
    want = F.mixture_density(N, 0.5, sp["centre"], sp["mass"], sp["radius"], sp["kind"], 25.6)
    assert rel(rho.cpu().numpy(), want) < 1e-5


@pytest.mark.parametrize("N,n", [(48, 16), (64, 8), (96, 8), (32, 32)])
def test_upsample_factors(env, N, n):
    # odd, even and unit factors; the fine rows of every coarse interval,
    # including the interval that wraps through the periodic face
    torch, S = env
    st = torch.cuda.current_stream()
    rng = np.random.default_rng(N + n)
    y = rng.normal(size=(3, n, n, n)).astype(np.float32)
    scale = torch.tensor([1.7, 0.0, 0.0, 0.0], device="cuda")
    H = torch.empty((3, N, N, N), device="cuda")
    S.upsample(torch.from_numpy(y).cuda(), N, n, scale, H, st)
    torch.cuda.synchronize()
    assert rel(H.cpu().numpy(), F.upsample(y.astype(np.float64), N, 1.7)) < 1e-6
