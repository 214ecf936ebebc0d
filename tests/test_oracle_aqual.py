"""Pins of the oracle's exact discrete AQUAL solution and of the reading R14
(the iteration of Sect. 2.1 ends in a period-2 cycle near zeros of the field).

The exact solution (``oracle.aqual_solve``) minimises the convex mesh energy
sum a0^2 Psi(|D phi|/a0) + g_N . D phi, Psi'(x) = mu(x) x, whose stationarity
condition is the discretised Eq. PDE. It is pinned three ways, none of which
compares it with itself:
  * it is a fixed point of the paper's iteration (App. Flow step 8): one more
    iteration started from its H leaves the acceleration mesh unchanged (odd
    grids, where the odd-operator convention drops no Nyquist term);
  * a brute-force minimisation of the same energy, written here with numpy
    FFTs and scipy's L-BFGS, reaches the same field;
  * in the Newtonian limit it is the closed form phi^ = A (k.kappa) phi_N^.
"""
import numpy as np
import pytest

import oracle
from paper_2312_02968_gb300 import workloads as W


def _rho(n, N, b, sigma, seed=1):
    p = W.isothermal(n, 1.0, N, b, 0.4 * n, seed=seed)
    acc, ka, _ = oracle.deposit_fixed(n, sigma, p["cell"], p["offset"], p["mass"])
    return oracle.acc_to_rho(acc, ka, 1.0)[1], p


def _mu_np(kind, x):
    return {0: x, 1: x / (1 + x), 2: x / np.sqrt(1 + x * x), 3: np.ones_like(x)}[kind]


def _spectral_grad(phi):
    """numpy: D phi with D_a = i k_a, the Nyquist term of axis a dropped."""
    n = phi.shape[0]
    k1 = np.fft.fftfreq(n) * 2 * np.pi
    if n % 2 == 0:
        k1[n // 2] = 0.0
    ph = np.fft.fftn(phi)
    out = []
    for a in range(3):
        shp = [1, 1, 1]
        shp[2 - a] = n
        out.append(np.real(np.fft.ifftn(1j * k1.reshape(shp) * ph)))
    return np.stack(out)


@pytest.mark.parametrize("kind", [oracle.MU_DEEP, oracle.MU_SIMPLE, oracle.MU_STANDARD, oracle.MU_NEWTON])
def test_exact_solution_is_a_fixed_point_of_the_iteration(kind):
    """H* = mu(|g*|/a0) g* - g_N with g* = -D phi* is divergence-free at the
    exact solution, and one iteration of App. Flow step 8 started from H*
    returns the same acceleration mesh (to rounding), two iterations nearly so
    (the iteration amplifies rounding near zeros of the field)."""
    n = 15
    rho, _ = _rho(n, 5000, 1.5, 1.0)
    ex = oracle.aqual_solve(rho, 1.0, 1.0, 1.0, kind, tol=1e-12)
    assert ex["rel_grad"] < 1e-11
    gN = oracle.solve(rho, 1.0, 1.0, 1.0, kind, 0, want=("gN",))["gN"]
    g = -_spectral_grad(ex["phi"])
    gm = np.sqrt((g ** 2).sum(0))
    Hs = _mu_np(kind, gm) * g - gN
    na = np.linalg.norm(ex["acc"])
    one = oracle.solve(rho, 1.0, 1.0, 1.0, kind, 1, H0=Hs, want=("acc",))["acc"]
    assert np.linalg.norm(one - ex["acc"]) / na < 1e-12
    two = oracle.solve(rho, 1.0, 1.0, 1.0, kind, 2, H0=Hs, want=("acc",))["acc"]
    assert np.linalg.norm(two - ex["acc"]) / na < 1e-9
    # a plausible error (the wrong interpolation function) is not a fixed point
    other = oracle.MU_SIMPLE if kind != oracle.MU_SIMPLE else oracle.MU_DEEP
    if kind != oracle.MU_NEWTON:
        wrong = oracle.aqual_solve(rho, 1.0, 1.0, 1.0, other, tol=1e-10)
        assert np.linalg.norm(wrong["acc"] - ex["acc"]) / na > 1e-2


@pytest.mark.parametrize("n,kind", [(8, oracle.MU_DEEP), (9, oracle.MU_STANDARD), (8, oracle.MU_SIMPLE)])
def test_brute_force_minimisation_agrees(n, kind):
    """scipy's L-BFGS on the energy written with numpy FFTs, from zero, on
    8^3 and 9^3 grids, lands on the oracle's minimiser."""
    so = pytest.importorskip("scipy.optimize")
    rho, _ = _rho(n, 600, 1.0, 0.75, seed=5)
    gN = oracle.solve(rho, 1.0, 1.0, 1.0, kind, 0, want=("gN",))["gN"]
    psi = {0: lambda x: x ** 3 / 3, 1: lambda x: x * x / 2 - x + np.log1p(x),
           2: lambda x: 0.5 * (x * np.sqrt(1 + x * x) - np.arcsinh(x))}[kind]

    def div_t(w):  # D^T w = -sum_a D_a w_a (D_a is skew)
        k1 = np.fft.fftfreq(n) * 2 * np.pi
        if n % 2 == 0:
            k1[n // 2] = 0.0
        tot = 0
        for a in range(3):
            shp = [1, 1, 1]
            shp[2 - a] = n
            tot = tot - 1j * k1.reshape(shp) * np.fft.fftn(w[a])
        return np.real(np.fft.ifftn(tot))

    def f(x):
        u = _spectral_grad(x.reshape(n, n, n))
        um = np.sqrt((u ** 2).sum(0))
        e = psi(um).sum() + (gN * u).sum()
        return e, div_t(_mu_np(kind, um) * u + gN).ravel()

    r = so.minimize(f, np.zeros(n ** 3), jac=True, method="L-BFGS-B",
                    options=dict(maxiter=5000, maxcor=20, ftol=1e-15, gtol=1e-13))
    bf = r.x.reshape(n, n, n)
    ex = oracle.aqual_solve(rho, 1.0, 1.0, 1.0, kind, tol=1e-12)
    gb, ge = _spectral_grad(bf), _spectral_grad(ex["phi"])
    assert np.linalg.norm(gb - ge) / np.linalg.norm(ge) < 1e-6


def test_newtonian_limit_closed_form():
    """mu = 1: the exact solution is the spectral projection of g_N, whose
    potential is phi^ = A (k.kappa) phi_N^ with kappa = sin(k s)/s (odd grid)."""
    n = 11
    rho, _ = _rho(n, 800, 1.2, 1.0, seed=6)
    ex = oracle.aqual_solve(rho, 1.0, 1.0, 1.0, oracle.MU_NEWTON, tol=1e-13)
    phiN = oracle.solve(rho, 1.0, 1.0, 1.0, oracle.MU_NEWTON, 0, want=("phi",))["phi"]
    k1 = np.fft.fftfreq(n) * 2 * np.pi
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = kx ** 2 + ky ** 2 + kz ** 2
    kkap = kx * np.sin(kx) + ky * np.sin(ky) + kz * np.sin(kz)
    A = np.where(kk > 0, 1 / np.where(kk > 0, kk, 1), 0)
    want = np.real(np.fft.ifftn(A * kkap * np.fft.fftn(phiN)))
    got = ex["phi"] - ex["phi"].mean()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-10


def test_r14_iteration_ends_in_a_two_cycle_in_fp64():
    """Reading R14, in FP64: on an isothermal sphere (32^3, b = 1 px,
    sigma 1.5 px, deep MOND) the undamped iteration does not converge. The
    iterates alternate between two states (iterates 40 and 42 agree far
    better than 40 and 41), the alternation sits at the centre, where the
    field vanishes, and its amplitude is far above 1e-4 of the acceleration
    mesh. The mean of the two states is close to the exact solution, closer
    than either state; no single iterate gets within 1e-4 of it."""
    n = 32
    rho, _ = _rho(n, 20000, 1.0, 1.5)
    a40, a41, a42 = (oracle.solve(rho, 1.0, 1.0, 1.0, oracle.MU_DEEP, K, want=("acc",))["acc"] for K in (40, 41, 42))
    ex = oracle.aqual_solve(rho, 1.0, 1.0, 1.0, oracle.MU_DEEP, tol=1e-11)
    na = np.linalg.norm(ex["acc"])
    amp = np.linalg.norm(a40 - a41) / na
    assert amp > 1e-3
    assert np.linalg.norm(a40 - a42) / na < 0.05 * amp
    d = np.sqrt(((a40 - a41) ** 2).sum(0))
    z, y, x = np.unravel_index(np.argmax(d), d.shape)
    assert max(abs(x - n // 2), abs(y - n // 2), abs(z - n // 2)) <= 2
    mean_err = np.linalg.norm(0.5 * (a40 + a41) - ex["acc"]) / na
    e40 = np.linalg.norm(a40 - ex["acc"]) / na
    e41 = np.linalg.norm(a41 - ex["acc"]) / na
    assert mean_err < 0.6 * min(e40, e41)
    assert min(e40, e41) > 1e-4
