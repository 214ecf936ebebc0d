"""Seeded synthetic particle sets shaped like the paper's test systems.

This module holds only input generation (initial conditions); it contains none
of the method's arithmetic, and both the CUDA path and the CPU oracle consume
its output. Every generator is deterministic in its seed (numpy default_rng).

Layout of a particle set (a dict of numpy arrays):
  cell   int32   [N, 3]  FFT-domain pixel index (x, y, z) of the nearest centre
  offset float32 [N, 3]  position minus that centre, in pixels, in [-1/2, 1/2]
  vel    float32 [N, 3]  velocity in length units per time unit
  mass   float32 [N]
Physical position = (cell - n_f/2 + offset) * s, so the domain is centred on 0
(App. "Fourier transforms" grid).
"""
from __future__ import annotations

import math

import numpy as np


def to_cells(pos_px: np.ndarray, n_f: int):
    """Pixel coordinates (origin at the domain centre) -> (cell, offset)."""
    p = np.asarray(pos_px, np.float64) + n_f / 2
    cell = np.floor(p + 0.5)
    off = (p - cell).astype(np.float32)
    cell = np.mod(cell.astype(np.int64), n_f).astype(np.int32)
    return cell, off


def _pack(pos_px, vel, mass, n_f):
    cell, off = to_cells(pos_px, n_f)
    return {
        "cell": np.ascontiguousarray(cell),
        "offset": np.ascontiguousarray(off),
        "vel": np.ascontiguousarray(np.asarray(vel, np.float32).reshape(-1, 3)),
        "mass": np.ascontiguousarray(np.asarray(mass, np.float32).reshape(-1)),
    }


def displaced(p: dict, n_f: int, s: float, t: float):
    """The particle set p with every position moved along its velocity for a
    time t (vel * t / s pixels; t < 0 gives nearby earlier configurations, a
    sequence of densities for warm-started solves). Cells and offsets are
    recomputed; velocities and masses are kept."""
    pos = p["cell"].astype(np.float64) - n_f / 2 + p["offset"].astype(np.float64)
    pos = pos + p["vel"].astype(np.float64) * (t / s)
    return _pack(pos, p["vel"], p["mass"], n_f)


def uniform_random(n_f: int, N: int, seed: int, margin: int = 0, mass_range=(0.5, 1.5)):
    """Particles uniform in the domain (less a margin), random masses, small velocities."""
    rng = np.random.default_rng(seed)
    half = n_f / 2 - margin
    pos = rng.uniform(-half, half, size=(N, 3))
    mass = rng.uniform(mass_range[0], mass_range[1], size=N) / max(N, 1)
    vel = rng.normal(0.0, 0.05, size=(N, 3))
    return _pack(pos, vel, mass, n_f)


def two_body(n_f: int, s: float, sep_px: float, m1: float, m2: float, G: float = 1.0, a0: float = 1.0):
    """Two point masses on the x axis about their centre of mass, with the
    circular-orbit relative speed of Eq. twobodyvelocity (deep MOND)."""
    M = m1 + m2
    v2 = (2.0 * math.sqrt(G * M * a0) / 3.0) * (1.0 / (1.0 + math.sqrt(m1 / M)) + 1.0 / (1.0 + math.sqrt(m2 / M)))
    v = math.sqrt(v2)
    r = sep_px
    pos = np.array([[m2 * r / M, 0, 0], [-m1 * r / M, 0, 0]], np.float64)
    vel = np.array([[0, m2 * v / M, 0], [0, -m1 * v / M, 0]], np.float64)
    return _pack(pos, vel, [m1, m2], n_f), {"v_rel": v, "period": 2 * math.pi * r * s / v}


def ring(n_f: int, s: float, N: int, m0: float, ring_mass: float, r2_px: float, G: float = 1.0, a0: float = 1.0,
         with_velocity: bool = True):
    """Central mass m0 at rest at the origin plus a regular N-gon of radius r2
    (Sect. 4.2), tangential speed from Eq. ringvelocity."""
    m = ring_mass / N
    M = m0 + N * m
    v2 = (2.0 * math.sqrt(G * M * a0) / 3.0) * (1.0 / (1.0 + math.sqrt(m0 / M)) + math.sqrt(m0 / M) - math.sqrt(m / M))
    v = math.sqrt(v2) if with_velocity else 0.0
    ang = 2 * math.pi * np.arange(N) / N
    pos = np.zeros((N + 1, 3))
    vel = np.zeros((N + 1, 3))
    pos[1:, 0] = r2_px * np.cos(ang)
    pos[1:, 1] = r2_px * np.sin(ang)
    vel[1:, 0] = -v * np.sin(ang)
    vel[1:, 1] = v * np.cos(ang)
    mass = np.concatenate([[m0], np.full(N, m)])
    return _pack(pos, vel, mass, n_f), {"v": v, "m": m, "M": M}


def isothermal(n_f: int, s: float, N: int, b_px: float, r_max_px: float, seed: int, M: float = 1.0,
               G: float = 1.0, a0: float = 1.0):
    """Deep-MOND isothermal sphere (Sect. 4.3): radius by the inverse of the
    cumulative mass (1 + (b/r)^{3/2})^{-2}, isotropic direction, Maxwellian
    velocities with mean square 2 sqrt(G M a0)/3 by Box-Muller (Eq. boxmuller).
    Samples beyond r_max are redrawn. Equal masses M/N."""
    rng = np.random.default_rng(seed)
    vsq = 2.0 * math.sqrt(G * M * a0) / 3.0
    pos = np.zeros((0, 3))
    vel = np.zeros((0, 3))
    while pos.shape[0] < N:
        k = int((N - pos.shape[0]) * 1.1) + 16
        xi1 = rng.uniform(-1.0, 1.0, k)
        eta = rng.uniform(0.0, 1.0, (k, 3))
        zeta = rng.uniform(0.0, 2 * math.pi, (k, 3))
        eta = np.clip(eta, 1e-300, 1.0)
        r = b_px * (1.0 / np.sqrt(eta[:, 0]) - 1.0) ** (-2.0 / 3.0)
        sxi = np.sqrt(1.0 - xi1 ** 2)
        p = np.stack([sxi * np.cos(zeta[:, 0]), sxi * np.sin(zeta[:, 0]), xi1], 1) * r[:, None]
        a = np.sqrt(-(2.0 / 3.0) * vsq * np.log(eta[:, 1]))
        c = np.sqrt(-(2.0 / 3.0) * vsq * np.log(eta[:, 2]))
        v = np.stack([a * np.cos(zeta[:, 1]), a * np.sin(zeta[:, 1]), c * np.cos(zeta[:, 2])], 1)
        keep = np.isfinite(r) & (r <= r_max_px)
        pos = np.concatenate([pos, p[keep]])
        vel = np.concatenate([vel, v[keep]])
    pos = pos[:N]
    vel = vel[:N]
    mass = np.full(N, M / N)
    return _pack(pos, vel, mass, n_f)


def plummer(n_f: int, s: float, N: int, a_px: float, r_max_px: float, seed: int, M: float = 1.0):
    """N equal-mass particles of a Plummer sphere of scale radius a_px pixels
    centred on the domain, truncated at r_max_px (textbook inverse cumulative
    mass M(r)/M = r^3/(r^2+a^2)^{3/2}); velocities zero (a cold start)."""
    rng = np.random.default_rng(seed)
    got = np.zeros((0, 3))
    while got.shape[0] < N:
        k = int((N - got.shape[0]) * 1.2) + 16
        eta = np.clip(rng.uniform(0.0, 1.0, k), 1e-12, 1 - 1e-12)
        r = a_px / np.sqrt(eta ** (-2.0 / 3.0) - 1.0)
        u = rng.uniform(-1.0, 1.0, k)
        ph = rng.uniform(0.0, 2 * math.pi, k)
        su = np.sqrt(1 - u * u)
        p = np.stack([su * np.cos(ph), su * np.sin(ph), u], 1) * r[:, None]
        got = np.concatenate([got, p[r <= r_max_px]])
    return _pack(got[:N], np.zeros((N, 3)), np.full(N, M / N), n_f)


def mixture_spheres(n_f: int, seed: int, n_spheres=None):
    """Parameters of a mixture of 1-8 Plummer (kind 0) or Hernquist (kind 1)
    spheres: masses log-uniform over [1e-2, 1], scale radii uniform over
    [4, 32] px, centres (pixels from the domain centre) keeping three scale
    radii inside the central 0.8 of the box."""
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 9)) if n_spheres is None else int(n_spheres)
    kinds = rng.integers(0, 2, K).astype(np.int32)
    masses = np.exp(rng.uniform(math.log(1e-2), math.log(1.0), K))
    radii = rng.uniform(4.0, 32.0, K)
    centres = np.zeros((K, 3))
    for j in range(K):
        lim = max(0.0, 0.4 * n_f - 3 * radii[j])
        centres[j] = rng.uniform(-lim, lim, 3)
    return {"K": K, "kind": kinds, "mass": masses, "radius": radii, "centre": centres}


def sphere_mixture(n_f: int, N: int, seed: int, n_spheres=None):
    """N equal-mass particles drawn from mixture_spheres(n_f, seed): particles
    allotted in proportion to mass, radii truncated at 0.4 box (textbook
    inverse cumulative mass profiles); velocities zero."""
    sp = mixture_spheres(n_f, seed, n_spheres)
    rng = np.random.default_rng([seed, 1])
    K, kinds, masses, radii = sp["K"], sp["kind"], sp["mass"], sp["radius"]
    counts = np.floor(N * masses / masses.sum()).astype(np.int64)
    counts[0] += N - counts.sum()
    rmax = 0.4 * n_f
    parts = []
    for j in range(K):
        centre = sp["centre"][j]
        got = np.zeros((0, 3))
        while got.shape[0] < counts[j]:
            k = int((counts[j] - got.shape[0]) * 1.2) + 16
            eta = np.clip(rng.uniform(0.0, 1.0, k), 1e-12, 1 - 1e-12)
            if kinds[j] == 0:  # Plummer: M(r)/M = r^3/(r^2+a^2)^{3/2}
                r = radii[j] / np.sqrt(eta ** (-2.0 / 3.0) - 1.0)
            else:  # Hernquist: M(r)/M = r^2/(r+a)^2
                se = np.sqrt(eta)
                r = radii[j] * se / (1.0 - se)
            u = rng.uniform(-1.0, 1.0, k)
            ph = rng.uniform(0.0, 2 * math.pi, k)
            su = np.sqrt(1 - u * u)
            p = np.stack([su * np.cos(ph), su * np.sin(ph), u], 1) * r[:, None] + centre
            keep = (r <= rmax) & np.all(np.abs(p) < n_f / 2 - 8, axis=1)
            got = np.concatenate([got, p[keep]])
        parts.append(got[: counts[j]])
    pos = np.concatenate(parts)
    mass = np.full(N, masses.sum() / N)
    vel = np.zeros((N, 3))
    return _pack(pos, vel, mass, n_f), sp


def isothermal_density_mesh(n_f: int, s: float, b: float, M: float = 1.0):
    """Eq. rho of the isothermal sphere sampled at the mesh nodes (z, y, x),
    centred on the domain centre: 3M/(4 pi b^3) (1 + (r/b)^{3/2})^{-3}."""
    c = (np.arange(n_f) - n_f / 2) * s
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    return 3.0 * M / (4 * math.pi * b ** 3) * (1.0 + (r / b) ** 1.5) ** (-3.0)
