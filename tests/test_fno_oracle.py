"""Pins of the FP64 FNO oracle (the learned warm start) against facts that do
not come from the oracle itself: brute-force sums, closed forms, finite
differences and an independent bfloat16 conversion."""
import math

import numpy as np
import pytest

from oracle import fno_oracle as F


def brute_dft(v, n, M):
    """s_j(k) = sum_x v_j(x) exp(-2 pi i k.x / n) by direct summation."""
    C = v.shape[0]
    freqs = list(range(M)) + list(range(-M, 0))
    out = np.zeros((C, 2 * M, 2 * M, M), np.complex128)
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    for a, kz in enumerate(freqs):
        for b, ky in enumerate(freqs):
            for kx in range(M):
                e = np.exp(-2j * np.pi * (kz * zz + ky * yy + kx * xx) / n)
                out[:, a, b, kx] = np.tensordot(v, e, axes=([1, 2, 3], [0, 1, 2]))
    return out.reshape(C, -1)


def test_truncated_transform_matches_direct_sum():
    rng = np.random.default_rng(0)
    for n, M in [(4, 2), (6, 2), (8, 3)]:
        v = rng.normal(size=(2, n, n, n))
        assert np.allclose(F.spec_fwd(v, M), brute_dft(v, n, M), rtol=0, atol=1e-10)


def band_limited(n, M, C, rng):
    """Real field built from cosines/sines at kept modes, kx < M and |ky|,|kz| < M
    (no -M component: the kept set holds only one of +-M on those axes)."""
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    v = np.zeros((C, n, n, n))
    for _ in range(6):
        kz, ky = rng.integers(-M + 1, M, 2)
        kx = rng.integers(0, M)
        ph = 2 * np.pi * (kz * zz + ky * yy + kx * xx) / n
        v += rng.normal(size=(C, 1, 1, 1)) * np.cos(ph) + rng.normal(size=(C, 1, 1, 1)) * np.sin(ph)
    return v


def test_spectral_layer_is_identity_on_band_limited_fields():
    rng = np.random.default_rng(1)
    n, M, C = 8, 3, 3
    v = band_limited(n, M, C, rng)
    K = M * 4 * M * M
    R = np.zeros((K, C, C), np.complex128)
    R[:, np.arange(C), np.arange(C)] = 1.0
    out = F.spec_inv(F.mix(F.spec_fwd(v, M), R), n, M)
    assert np.allclose(out, v, atol=1e-10)


def test_spectral_layer_single_mode_closed_form():
    # one channel, a constant weight w at mode (kz, ky, kx) = (1, -1, 1) and its
    # input a cosine at that mode: output = Re(w e^{i phase}) scaled by 1
    n, M = 8, 2
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ph = 2 * np.pi * (1 * zz - 1 * yy + 1 * xx) / n
    v = np.cos(ph)[None]
    K = M * 4 * M * M
    R = np.zeros((K, 1, 1), np.complex128)
    w = 0.3 - 0.7j
    R[:, 0, 0] = w
    out = F.spec_inv(F.mix(F.spec_fwd(v, M), R), n, M)
    # the cosine has +-k components; kx >= 0 keeps (1,-1,1); its mirror (-1,1,-1)
    # is represented by the conjugate half, so the output is Re(w e^{i ph})
    assert np.allclose(out[0], (w * np.exp(1j * ph)).real, atol=1e-12)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    sh = F.Shape(4, 3, 2, 2)
    flat = rng.normal(scale=0.4, size=sh.count())
    x = rng.normal(size=(4, 4, 4, 4))
    t = rng.normal(size=(3, 4, 4, 4))
    y, cache = F.forward(flat, x, sh)
    L0, dy = F.loss(y, t)
    g = F.backward(flat, cache, dy, sh)
    # sample parameters from every block
    C, K = sh.C, sh.K
    idx = list(rng.integers(0, 5 * C, 6))
    for l in range(sh.L):
        base = 5 * C + l * sh.layer_size()
        idx += list(base + rng.integers(0, C * C + C, 6))
        idx += list(base + C * C + C + rng.integers(0, 2 * K * C * C, 10))
    base = 5 * C + sh.L * sh.layer_size()
    idx += list(base + rng.integers(0, 3 * C + 3, 6))
    h = 1e-6
    for i in idx:
        fp = flat.copy()
        fp[i] += h
        fm = flat.copy()
        fm[i] -= h
        Lp = F.loss(F.forward(fp, x, sh)[0], t)[0]
        Lm = F.loss(F.forward(fm, x, sh)[0], t)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_gradient_is_the_derivative():
    rng = np.random.default_rng(3)
    y = rng.normal(size=50)
    t = rng.normal(size=50)
    L, dy = F.loss(y, t, weight=0.5)
    assert L == pytest.approx(0.5 * np.sum((y - t) ** 2) / np.sum(t * t))
    e = np.zeros(50)
    e[7] = 1e-6
    fd = (F.loss(y + e, t, 0.5)[0] - F.loss(y - e, t, 0.5)[0]) / 2e-6
    assert fd == pytest.approx(dy[7], rel=1e-7)


def test_bf16_rounding_hand_values_and_torch():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 1.0 + 2 ** -7 + 2 ** -9, 3.0e-30, 65504.0],
                    np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2 ** -6, -2.5, 1.0 + 2 ** -7, None, 65536.0], dtype=object)
    got = F.bf16_round(vals)
    for g, w in zip(got, want):
        if w is not None:
            assert g == w
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    a = (rng.normal(size=20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(F.bf16_round(a), ref)


def test_gelu_tanh_form_against_erf_form():
    z = np.linspace(-6, 6, 1201)
    exact = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in z])
    assert np.max(np.abs(F.gelu(z) - exact)) < 1e-3
    assert F.gelu(np.array([0.0]))[0] == 0.0
    h = 1e-6
    assert np.allclose((F.gelu(z + h) - F.gelu(z - h)) / (2 * h), F.gelu_grad(z), atol=1e-7)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(5)
    p = rng.normal(size=100)
    g = rng.normal(size=100)
    p1, m, v = F.adam(p, g, np.zeros(100), np.zeros(100), 1e-3, 0.9, 0.999, 1e-8, 1)
    assert np.allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), atol=1e-12)


def test_coarsen_and_upsample():
    rng = np.random.default_rng(6)
    fine = rng.normal(size=(2, 16, 16, 16))
    c = F.coarsen(fine, 4)
    assert c.shape == (2, 4, 4, 4)
    assert np.allclose(c.mean(axis=(1, 2, 3)), fine.mean(axis=(1, 2, 3)))
    assert c[1, 2, 1, 3] == pytest.approx(fine[1, 8:12, 4:8, 12:16].mean())
    const = np.full((1, 4, 4, 4), 2.5)
    assert np.allclose(F.upsample(const, 16, 2.0), 5.0)
    # a field linear in x on the coarse cells interpolates linearly in between
    # (away from the periodic seam)
    n, N = 8, 32
    lin = np.broadcast_to(np.arange(n, dtype=float)[None, None, None, :], (1, n, n, n)).copy()
    up = F.upsample(lin, N, 1.0)
    f = N // n
    X = np.arange(N)
    u = (X + 0.5) / f - 0.5
    inner = (u >= 1) & (u <= n - 2)  # all four taps on the same side of the seam
    assert np.allclose(up[0, 3, 5, inner], u[inner])
    # and a quadratic one exactly (cubic convolution is third-order accurate)
    quad = lin ** 2
    upq = F.upsample(quad, N, 1.0)
    assert np.allclose(upq[0, 3, 5, inner], u[inner] ** 2)
    assert np.allclose(F.cubic_weights(np.linspace(0, 0.99, 7)).sum(0), 1.0)


def test_mixture_density_masses():
    N, s = 96, 1.0
    # Plummer: mass inside rmax is M rmax^3 / (rmax^2 + a^2)^{3/2}
    rho = F.mixture_density(N, s, [[0.0, 0.0, 0.0]], [1.0], [6.0], [0], 40.0)
    want = 40.0 ** 3 / (40.0 ** 2 + 36.0) ** 1.5
    assert rho.sum() * s ** 3 == pytest.approx(want, rel=2e-3)
    # Hernquist: M rmax^2 / (rmax + a)^2 (the r >= 1/2 floor removes a little mass at the centre)
    rho = F.mixture_density(N, s, [[3.0, -2.0, 1.0]], [0.5], [8.0], [1], 40.0)
    want = 0.5 * 40.0 ** 2 / 48.0 ** 2
    assert rho.sum() * s ** 3 == pytest.approx(want, rel=2e-2)
    # the profile is centred where asked
    k = np.unravel_index(np.argmax(rho), rho.shape)
    assert (k[2] - N // 2, k[1] - N // 2, k[0] - N // 2) == (3, -2, 1)
