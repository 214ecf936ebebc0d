"""Pins of the oracle's mesh-interpolating gather: the node-smoothed field
(Eq. gi at pixel centres) and its linear / Keys-cubic interpolation at the
particles, against polynomial exactness, the Gaussian's Fourier transform
(App. Fourier) and the convergence order towards Eq. gi."""
import math

import numpy as np
import pytest

import oracle


def interior_particles(n, N, seed, margin=3):
    rng = np.random.default_rng(seed)
    cell = rng.integers(margin, n - margin, (N, 3)).astype(np.int32)
    off = (rng.random((N, 3)) - 0.5).astype(np.float32).astype(np.float64)
    return cell, off


def poly_field(n, coef, degree):
    c = np.arange(n, dtype=np.float64)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    out = []
    for a in range(3):
        p = coef[a][0] + coef[a][1] * x + coef[a][2] * y + coef[a][3] * z
        if degree >= 2:
            p = p + coef[a][4] * x * x + coef[a][5] * y * z + coef[a][6] * z * z + coef[a][7] * x * y
        if degree >= 3:
            p = p + coef[a][8] * x * x * x
        out.append(p)
    return np.stack(out)


def poly_at(coef, degree, pos):
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    out = []
    for a in range(3):
        p = coef[a][0] + coef[a][1] * x + coef[a][2] * y + coef[a][3] * z
        if degree >= 2:
            p = p + coef[a][4] * x * x + coef[a][5] * y * z + coef[a][6] * z * z + coef[a][7] * x * y
        if degree >= 3:
            p = p + coef[a][8] * x * x * x
        out.append(p)
    return np.stack(out, axis=1)


@pytest.mark.parametrize("order,degree,exact", [(1, 1, True), (1, 2, False), (3, 1, True), (3, 2, True),
                                                (3, 3, False)])
def test_polynomial_reproduction(order, degree, exact):
    # linear interpolation reproduces linear fields, the Keys kernel (a = -1/2)
    # quadratics; neither reproduces the next degree
    n = 16
    rng = np.random.default_rng(order * 10 + degree)
    coef = rng.normal(size=(3, 9)) * 0.1
    S = poly_field(n, coef, degree)
    cell, off = interior_particles(n, 500, degree)
    got = oracle.interp_gather(order, S, cell, off)
    want = poly_at(coef, degree, cell + off)
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    if exact:
        assert err < 1e-12
    else:
        assert err > 1e-6


@pytest.mark.parametrize("order", [1, 3])
def test_zero_offset_gives_node_values_and_wraps(order):
    n = 8
    rng = np.random.default_rng(5)
    S = rng.normal(size=(3, n, n, n))
    cell = rng.integers(0, n, (300, 3)).astype(np.int32)
    got = oracle.interp_gather(order, S, cell, np.zeros((300, 3)))
    want = S[:, cell[:, 2], cell[:, 1], cell[:, 0]].T
    assert np.allclose(got, want, atol=1e-14)
    # a constant field, particles at the faces of the periodic box
    cell[:, 0] = 0
    off = np.full((300, 3), -0.49)
    const = np.broadcast_to(np.array([1.5, -2.0, 0.25])[:, None, None, None], (3, n, n, n)).copy()
    assert np.allclose(oracle.interp_gather(order, const, cell, off), [1.5, -2.0, 0.25], atol=1e-14)


def test_node_smoothed_single_mode_is_the_gaussian_spectrum():
    # App. Fourier: smoothing with the Gaussian multiplies a mode by
    # exp(-sigma^2 k^2 / 2); the ball truncation and sampling leave 2e-3
    n, sigma = 32, 1.5
    c = np.arange(n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    k = 2 * np.pi * np.array([2, 1, 3]) / n
    mode = np.cos(k[0] * x + k[1] * y + k[2] * z)
    S = oracle.node_smoothed(sigma, np.stack([mode, 2 * mode, -mode]))
    factor = math.exp(-0.5 * sigma ** 2 * float(k @ k))
    for a, amp in enumerate((1.0, 2.0, -1.0)):
        assert np.max(np.abs(S[a] - amp * factor * mode)) < 2e-3 * abs(amp)


def test_interpolation_converges_to_eq_gi():
    # against the exact ball sum at the particles, for modes of wavelength 32
    # and 16 px: linear interpolation loses a factor ~4 when the wavelength
    # halves (second order); the cubic is far closer at both
    n, sigma = 64, 1.5
    rng = np.random.default_rng(6)
    cell = rng.integers(0, n, (3000, 3)).astype(np.int32)
    off = (rng.random((3000, 3)) - 0.5).astype(np.float32)
    c = np.arange(n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    err = {}
    for lam in (32, 16):
        k = 2 * np.pi / lam
        a = np.stack([np.sin(k * x + 0.3) * np.cos(k * y), np.cos(k * z + 1.0), np.sin(k * (x + y + z))])
        S = oracle.node_smoothed(sigma, a)
        ex = oracle.gather(sigma, a, cell, off)
        for order in (1, 3):
            g = oracle.interp_gather(order, S, cell, off.astype(np.float64))
            err[lam, order] = np.linalg.norm(g - ex) / np.linalg.norm(ex)
    assert 3.0 < err[16, 1] / err[32, 1] < 5.0
    assert err[32, 3] < err[32, 1] / 5 and err[16, 3] < err[16, 1] / 10
