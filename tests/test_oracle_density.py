"""Pins of the oracle's apparent-density functions (Eq. apparentdensity,
Eq. totalmass) against closed forms, numpy FFTs of the definition, the discrete
Gauss theorem and the isothermal sphere of Sect. 4.3. Nothing here compares a
function with itself."""
import math

import numpy as np
import pytest

import oracle
from paper_2312_02968_gb300 import workloads as W

FOUR_PI = 4.0 * math.pi


def test_density_of_sine_fields_closed_form():
    # g = (A sin(kx x + p), B cos(ky y), C sin(kz z)) on a 16^3 mesh of pixel
    # width s: the central difference of sin(k u) is cos(k u) sin(k s)/s and of
    # cos(k u) is -sin(k u) sin(k s)/s
    n, s, G = 16, 0.7, 2.5
    L = n * s
    u = np.arange(n) * s
    z, y, x = np.meshgrid(u, u, u, indexing="ij")
    kx, ky, kz = 2 * np.pi * 1 / L, 2 * np.pi * 3 / L, 2 * np.pi * 2 / L
    A, B, C, p = 1.3, -0.4, 0.9, 0.3
    g = np.stack([A * np.sin(kx * x + p), B * np.cos(ky * y), C * np.sin(kz * z)])
    div = (A * np.cos(kx * x + p) * np.sin(kx * s) / s - B * np.sin(ky * y) * np.sin(ky * s) / s
           + C * np.cos(kz * z) * np.sin(kz * s) / s)
    assert np.allclose(oracle.field_density(g, s, G), -div / (FOUR_PI * G), rtol=0, atol=1e-13)


def test_baryonic_density_spectral_relation():
    # rho_B = -div_FD g_N / 4 pi G with g_N = -grad_FD phi_N and
    # phi^_N = -4 pi G rho^/|k|^2: rho^_B = (|k_FD|^2/|k|^2) rho^ for k != 0, 0 at k = 0,
    # k_FD = sin(k s)/s per axis (numpy FFT, not the oracle's transform)
    n, s, G = 16, 1.3, 0.8
    rng = np.random.default_rng(11)
    rho = rng.random((n, n, n)) + 0.5
    gN = oracle.solve(rho, s, G, 1.0, oracle.MU_NEWTON, 0, want=("gN",))["gN"]
    rB = oracle.field_density(gN, s, G)
    m = np.fft.fftfreq(n, d=1.0 / n)
    k = 2 * np.pi * m / (n * s)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    kk = kx * kx + ky * ky + kz * kz
    kf = (np.sin(kx * s) ** 2 + np.sin(ky * s) ** 2 + np.sin(kz * s) ** 2) / s ** 2
    ratio = np.where(kk > 0, kf / np.where(kk > 0, kk, 1.0), 0.0)
    want = np.fft.ifftn(np.fft.fftn(rho) * ratio).real
    assert np.max(np.abs(rB - want)) < 1e-12 * np.max(np.abs(want))


def box_sum(f, lo, hi):
    n = f.shape[0]
    zi = np.arange(lo[2], hi[2] + 1) % n
    yi = np.arange(lo[1], hi[1] + 1) % n
    xi = np.arange(lo[0], hi[0] + 1) % n
    return f[np.ix_(zi, yi, xi)].sum()


def test_box_flux_mass_is_the_box_sum_of_the_density():
    # discrete Gauss theorem: the flux with face values the mean of the two
    # adjacent cells equals the sum of the central-difference divergence
    n, s, G = 12, 0.9, 1.7
    rng = np.random.default_rng(12)
    g = rng.normal(size=(3, n, n, n))
    rho = oracle.field_density(g, s, G)
    for lo, hi in [([2, 3, 1], [7, 5, 9]), ([-3, 0, 4], [2, 11, 4]), ([5, 5, 5], [5, 5, 5])]:
        got = oracle.box_flux_mass(g, s, G, lo, hi)
        assert got == pytest.approx(box_sum(rho, lo, hi) * s ** 3, rel=1e-11, abs=1e-12)
    # the whole periodic box holds no net divergence
    assert abs(oracle.box_flux_mass(g, s, G, [0, 0, 0], [n - 1, n - 1, n - 1])) < 1e-12
    assert abs(rho.sum()) < 1e-10


def test_shell_mass_brute_force():
    n, s = 8, 1.5
    rng = np.random.default_rng(13)
    rho = rng.normal(size=(n, n, n))
    c = [0.4, -2.2, 5.1]  # beyond half the box on z: the minimum image wraps it
    dr, nb = 0.8, 9
    want = np.zeros(nb)
    L = n * s
    for z in range(n):
        for y in range(n):
            for x in range(n):
                d = []
                for i, ci in zip((x, y, z), c):
                    v = (i - n / 2) * s - ci
                    v -= L * round(v / L)
                    d.append(v)
                k = int(math.floor(math.sqrt(sum(v * v for v in d)) / dr))
                if k < nb:
                    want[k] += rho[z, y, x] * s ** 3
    assert np.allclose(oracle.shell_mass(rho, s, c, dr, nb), want, rtol=1e-12, atol=1e-12)


def test_newtonian_mu_apparent_density_closed_form():
    # mu = 1: the iteration's potential is phi^ = A (k.k_FD) phi^_N (the
    # Newtonian closed form of the solve), so rho^_A = ((k.k_FD)/|k|^2) rho^_B
    # and the two agree at low k; numpy FFT of the oracle's rho_B. An odd grid
    # has no Nyquist plane, where keeping the real part after each inverse
    # transform makes the projections inexact.
    n, s, G = 15, 1.0, 1.0
    c = (np.arange(n) - n // 2) * s
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    rho = np.exp(-((x - 1.0) ** 2 + y ** 2 + (z + 0.5) ** 2) / 4.0) + 0.5 * np.exp(-(x * x + (y - 3) ** 2 + z * z))
    out = oracle.solve(rho, s, G, 1.0, oracle.MU_NEWTON, 4, want=("gN", "acc"))
    rA = oracle.field_density(out["acc"], s, G)
    rB = oracle.field_density(out["gN"], s, G)
    m = np.fft.fftfreq(n, d=1.0 / n)
    k = 2 * np.pi * m / (n * s)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    kk = kx * kx + ky * ky + kz * kz
    kkf = (kx * np.sin(kx * s) + ky * np.sin(ky * s) + kz * np.sin(kz * s)) / s
    ratio = np.where(kk > 0, kkf / np.where(kk > 0, kk, 1.0), 0.0)
    want = np.fft.ifftn(np.fft.fftn(rB) * ratio).real
    assert np.max(np.abs(rA - want)) < 1e-11 * np.max(np.abs(rB))
    # the two differ only at high k: a smooth low-pass of both agrees
    low = (np.abs(kx) < 0.5) & (np.abs(ky) < 0.5) & (np.abs(kz) < 0.5)
    la = np.fft.ifftn(np.fft.fftn(rA) * low).real
    lb = np.fft.ifftn(np.fft.fftn(rB) * low).real
    assert np.max(np.abs(la - lb)) < 0.05 * np.max(np.abs(lb))


@pytest.fixture(scope="module")
def isothermal_solution():
    n, s, b, M = 64, 1.0, 3.0, 1.0
    rho = W.isothermal_density_mesh(n, s, b, M)
    out = oracle.solve(rho, s, 1.0, 1.0, oracle.MU_DEEP, 8, want=("gN", "acc"))
    return n, s, b, M, out


def test_isothermal_apparent_density_profile(isothermal_solution):
    """Sect. 4.3: rho_A(r) = (1/4 pi) sqrt(M a0/(G b^3 r)) (5/2 + (r/b)^{3/2})
    (1 + (r/b)^{3/2})^{-2}, compared as shell means over the same cells, inside
    the radius where the periodic images stay small."""
    n, s, b, M, out = isothermal_solution
    rA = oracle.field_density(out["acc"], s, 1.0)
    c = (np.arange(n) - n / 2) * s
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    rc = np.maximum(r, 1e-9)
    q = (rc / b) ** 1.5
    closed = np.sqrt(M / (b ** 3 * rc)) * (2.5 + q) / (1 + q) ** 2 / FOUR_PI
    for k in range(2, 8):
        m = (r >= k) & (r < k + 1)
        assert abs(rA[m].mean() / closed[m].mean() - 1) < 0.03, k


def test_isothermal_enclosed_apparent_mass(isothermal_solution):
    """Sect. 4.3: M_A(r) = sqrt(M a0/G) r (1 + (b/r)^{3/2})^{-1}, against the
    shell sums of the apparent density about the centre; and M_B(r) of Eq. M
    from the Newtonian field."""
    n, s, b, M, out = isothermal_solution
    cumA = np.cumsum(oracle.shell_mass(oracle.field_density(out["acc"], s, 1.0), s, [0, 0, 0], 1.0, 16))
    cumB = np.cumsum(oracle.shell_mass(oracle.field_density(out["gN"], s, 1.0), s, [0, 0, 0], 1.0, 16))
    for R in (6, 8, 10, 12):
        MA = math.sqrt(M) * R / (1 + (b / R) ** 1.5)
        MB = M * R ** 3 / b ** 3 / (1 + (R / b) ** 1.5) ** 2
        assert abs(cumA[R - 1] / MA - 1) < 0.04, R
        assert abs(cumB[R - 1] / MB - 1) < 0.04, R
    # the phantom (apparent minus baryonic) mass grows outward: deep MOND
    assert np.all(np.diff((cumA - cumB)[4:12]) > 0)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_dipole_layer_newtonian_field(axis):
    """Sect. 5.3: a layer of mass M on the last plane and -M on the adjacent
    (periodic) first one. Gauss's law on the periodic box, whose field has
    zero mean: away from the layer the field is uniform, 4 pi G M s / L^3
    along +axis."""
    n, s, G, M = 32, 0.5, 1.3, 2.0
    rho = oracle.dipole_layer(n, s, axis, M)
    assert abs(rho.sum()) < 1e-12
    assert rho.sum(axis=tuple(a for a in range(3) if a != 2 - axis)).max() * s ** 3 == pytest.approx(M)
    gN = oracle.solve(rho, s, G, 1.0, oracle.MU_NEWTON, 0, want=("gN",))["gN"]
    want = 4 * math.pi * G * M * s / (n * s) ** 3
    # the middle third of the box along the axis, all components
    mid = [slice(None)] * 3
    mid[2 - axis] = slice(n // 3, 2 * n // 3)
    g = gN[(slice(None),) + tuple(mid)]
    assert np.max(np.abs(g[axis] / want - 1)) < 3e-3
    others = [a for a in range(3) if a != axis]
    assert np.max(np.abs(g[others])) < 1e-12
    gneg = oracle.solve(oracle.dipole_layer(n, s, axis, -M), s, G, 1.0, oracle.MU_NEWTON, 0, want=("gN",))["gN"]
    assert np.allclose(gneg, -gN, atol=1e-15)
