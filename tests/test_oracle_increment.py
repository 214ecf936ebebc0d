"""Pins of the oracle's incremental solve (Sect. 5.2 (v): increments of the
fields with the nu and mu steps linearised about the base state) against
central differences of the oracle's own nu/mu and of its full iteration, the
exact linearity of the Newtonian iteration, and the fixed-point deposit's
exact integer increment. Nothing here compares a function with itself."""
import numpy as np
import pytest

import oracle

N16 = 16
KINDS = (oracle.MU_DEEP, oracle.MU_SIMPLE, oracle.MU_STANDARD)


def _grid(n):
    return np.meshgrid(*(np.arange(n),) * 3, indexing="ij")


def _blob(c, w, m, n=N16):
    z, y, x = _grid(n)
    d2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
    return m * np.exp(-d2 / (2 * w * w)) / (2 * np.pi * w * w) ** 1.5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


RHO0 = _blob((7.3, 8.1, 7.7), 2.0, 1.0) + _blob((4, 5, 10), 1.5, 0.3)
# mass moved from the main blob to a neighbouring one: zero net increment
DRHO = _blob((9.5, 6.5, 8.5), 1.7, 0.2) - _blob((7.3, 8.1, 7.7), 2.0, 0.2)


@pytest.mark.parametrize("kind", KINDS + (oracle.MU_NEWTON,))
def test_derivative_factors_are_central_differences_of_nu_and_mu(kind):
    # y nu'(y) and x mu'(x) against central differences of nu and mu (whose
    # pair relation is pinned separately)
    for y in (0.03, 0.4, 1.0, 2.7, 40.0):
        h = 1e-6 * y
        fd_nu = y * (oracle.nu(kind, y + h) - oracle.nu(kind, y - h)) / (2 * h)
        fd_mu = y * (oracle.mu(kind, y + h) - oracle.mu(kind, y - h)) / (2 * h)
        L = oracle.lib()
        assert L.ora_ynu_prime(kind, y) == pytest.approx(fd_nu, rel=1e-7, abs=1e-12)
        assert L.ora_xmu_prime(kind, y) == pytest.approx(fd_mu, rel=1e-7, abs=1e-12)


@pytest.mark.parametrize("kind", KINDS + (oracle.MU_NEWTON,))
@pytest.mark.parametrize("which", (0, 1))
def test_linearised_step_is_the_directional_derivative(kind, which):
    # J(P) dv = d/de [f(|P + e dv|/a0) (P + e dv)] at e = 0, f = nu or mu
    rng = np.random.default_rng(5 + 2 * kind + which)
    a0 = 0.7
    f = oracle.nu if which == 0 else oracle.mu
    for _ in range(6):
        P = rng.normal(size=3) * rng.choice([0.05, 1.0, 30.0])
        dv = rng.normal(size=3)
        g = lambda v: f(kind, np.linalg.norm(v) / a0) * v
        e = 1e-6 * np.linalg.norm(P)
        fd = (g(P + e * dv) - g(P - e * dv)) / (2 * e)
        assert np.allclose(oracle.linearised(kind, which, a0, P, dv), fd, rtol=1e-6, atol=1e-9 * np.abs(fd).max())


def test_linearised_step_at_zero_field():
    # identity for the Newtonian kind, zero otherwise (the zero-field reading)
    dv = np.array([0.3, -1.2, 0.5])
    for which in (0, 1):
        assert np.array_equal(oracle.linearised(oracle.MU_NEWTON, which, 1.0, np.zeros(3), dv), dv)
        for kind in KINDS:
            assert np.array_equal(oracle.linearised(kind, which, 1.0, np.zeros(3), dv), np.zeros(3))


@pytest.mark.parametrize("K", (1, 3))
def test_newtonian_increment_equals_difference_of_full_solves(K):
    # nu = mu = 1: the iteration is linear in (rho, H), so the increment about
    # the solve of rho0 is exactly solve(rho0 + drho) - solve(rho0), field by field
    s, G, a0 = 1.0, 1.0, 1.0
    want = ("acc", "H", "gN", "gM")
    f0 = oracle.solve(RHO0, s, G, a0, oracle.MU_NEWTON, K, finish_h=True, want=want)
    f1 = oracle.solve(RHO0 + DRHO, s, G, a0, oracle.MU_NEWTON, K, finish_h=True, want=want)
    inc = oracle.solve_increment(DRHO, s, G, a0, oracle.MU_NEWTON, K, f0["gN"], f0["H"], f0["gM"])
    for a, b in (("dacc", "acc"), ("dH", "H"), ("dgN", "gN"), ("dgM", "gM")):
        assert _rel(inc[a], f1[b] - f0[b]) < 1e-11, a


def test_increment_is_linear_in_the_density_increment():
    s, G, a0 = 1.0, 1.0, 1.0
    b = oracle.solve(RHO0, s, G, a0, oracle.MU_DEEP, 4, finish_h=True, want=("gN", "H", "gM"))
    i1 = oracle.solve_increment(DRHO, s, G, a0, oracle.MU_DEEP, 4, b["gN"], b["H"], b["gM"])
    i2 = oracle.solve_increment(-2.5 * DRHO, s, G, a0, oracle.MU_DEEP, 4, b["gN"], b["H"], b["gM"])
    for k in i1:
        assert _rel(i2[k], -2.5 * i1[k]) < 1e-13, k


@pytest.mark.parametrize("kind", KINDS)
def test_increment_is_the_derivative_of_the_iteration_at_a_fixed_point(kind):
    # About a converged base (H0 a fixed point of the iteration for rho0), K full
    # iterations from H0 for rho0 +- eps drho differ by 2 eps times the K-iteration
    # increment up to O(eps^2): the error falls fourfold as eps halves
    s, G, a0, K = 1.0, 1.0, 1.0, 3
    b = oracle.solve(RHO0, s, G, a0, kind, 400, finish_h=True, want=("gN", "H", "gM", "dH"))
    assert b["dH"][-1] < 1e-13  # converged base
    inc = oracle.solve_increment(DRHO, s, G, a0, kind, K, b["gN"], b["H"], b["gM"])
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        fp = oracle.solve(RHO0 + eps * DRHO, s, G, a0, kind, K, H0=b["H"], finish_h=True, want=("acc", "H"))
        fm = oracle.solve(RHO0 - eps * DRHO, s, G, a0, kind, K, H0=b["H"], finish_h=True, want=("acc", "H"))
        e_acc = _rel(inc["dacc"], (fp["acc"] - fm["acc"]) / (2 * eps))
        e_h = _rel(inc["dH"], (fp["H"] - fm["H"]) / (2 * eps))
        errs.append((e_acc, e_h))
    assert errs[0][0] < 3e-5 and errs[0][1] < 2e-4
    for (a0_, h0_), (a1_, h1_) in zip(errs, errs[1:]):
        assert 3.6 < a0_ / a1_ < 4.4 and 3.6 < h0_ / h1_ < 4.4


def test_deposit_increment_is_exact():
    # the integer accumulators of two deposits with the same Kacc differ by the
    # deposit of the moved particles' old and new positions, exactly (rule R1),
    # and the FP32 increment is that integer rounded once: within 2^-24 of it
    # per cell, where the difference of the two FP32 densities is not
    n, sigma = 24, 1.5
    rng = np.random.default_rng(8)
    N = 300
    cell = rng.integers(8, n - 8, size=(N, 3)).astype(np.int32)
    off = (rng.random((N, 3)) - 0.5).astype(np.float32)
    mass = np.full(N, 1.0 / N, np.float32)
    k = oracle.kacc(mass)
    acc0 = oracle.deposit_fixed(n, sigma, cell, off, mass, k)[0]
    moved = np.arange(0, N, 7)
    off1 = off.copy()
    off1[moved] = np.clip(off1[moved] + 0.21, -0.5, 0.5)
    acc1 = oracle.deposit_fixed(n, sigma, cell, off1, mass, k)[0]
    a_old = oracle.deposit_fixed(n, sigma, cell[moved], off[moved], mass[moved], k)[0]
    a_new = oracle.deposit_fixed(n, sigma, cell[moved], off1[moved], mass[moved], k)[0]
    d = acc1.astype(np.int64) - acc0.astype(np.int64)
    assert np.array_equal(d, a_new.astype(np.int64) - a_old.astype(np.int64))
    exact = d.astype(np.float64) * 2.0 ** -k
    drho = oracle.delta_rho(acc1, acc0, k, 1.0).astype(np.float64)
    nz = exact != 0
    assert nz.sum() > 1000
    assert np.all(np.abs(drho - exact)[nz] <= 2.0 ** -24 * np.abs(exact)[nz])
    assert np.array_equal(drho == 0, ~nz)
    r0 = oracle.acc_to_rho(acc0, k, 1.0)[0].astype(np.float64)
    r1 = oracle.acc_to_rho(acc1, k, 1.0)[0].astype(np.float64)
    assert np.abs((r1 - r0) - exact)[nz].max() > 10 * np.abs(drho - exact)[nz].max()
