"""FP64 CPU oracle of the MOND particle-mesh method (Visser, Eijt & de Nijs 2023).

TEST INFRASTRUCTURE ONLY. The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The oracle shares no code
with the CUDA library under ``paper_2312_02968_gb300/``; neither imports the
other. All arithmetic lives in ``mond_oracle.c``; this module only marshals
numpy arrays into it.

What pins each function (tests in ``tests/test_oracle_*.py``):
  ball            251 taps for sigma = 1 (Sect. 3.1, Fig. 1); brute-force counts.
  axis_lut        Poisson-summation normalisation of the sampled Gaussian.
  deposit_fixed   vs the direct FP64 Eq. smooth (error bound of the rule);
                  Fourier transform of one particle = exp(-sigma^2 k^2/2)
                  (App. Fourier); mass conservation; order independence;
                  the integer rule tap by tap (a hand-worked particle, and
                  every tap of single particles recomputed from the rule).
  fft1/fft3       vs the plain DFT; round trip; Parseval; numpy.fft.
  mu/nu           mu(x) x = y <=> nu(y) y = x for every kind (Sect. 2.1).
  solve           transform count 42 for K = 4 and 2 for Newton (Sect. 5.2,
                  Sect. 6); the Newtonian closed form; the spectral Poisson
                  solve of a point mass; curl/div invariants; deep-MOND
                  point-mass field sqrt(G M a0)/r (Sect. 2); two-body force
                  (Eq. twobodyforce); ring force (Eq. ringforce); isothermal
                  field (Eq. g); the low-k residual of the discretised AQUAL
                  equation falls tenfold in three iterations; convergence
                  rate (Sect. 2.1); in FP64 the iterates end in a period-2
                  cycle at the zero of the field (reading R14).
  aqual_solve     the exact solution of the discretised AQUAL equation is a
                  fixed point of the iteration (odd grids, every kind); a
                  brute-force scipy minimisation of the same energy on 8^3
                  and 9^3 agrees; Newtonian closed form A (k.kappa) phi_N^.
  gather          particle at a node sees the node-smoothed field; constant
                  field reproduces the ball weight sum; two-body force.
  push            Eq. motion on hand-checked numbers; circular orbit period.
  particle_diag   two-body constants of motion on hand-made states.
  field_density   closed form on a sine field; the spectral relation
                  rho_B^ = (|k_FD|^2/|k|^2) rho^ (numpy FFT); Newtonian mu
                  gives rho_A = rho_B; isothermal rho_A and M_A (Sect. 4.3).
  box_flux_mass   equals the box sum of field_density (discrete Gauss
                  theorem); the total mass of a periodic box is zero.
  shell_mass      brute-force sums on small grids; enclosed M_A(r) of the
                  isothermal sphere (Sect. 4.3 closed form).
  dipole_layer    Newtonian field of the layer away from it equals the
                  closed form 4 pi G M s / L^3 (Gauss's law on the periodic
                  box); zero net mass; the field reverses with the sign.
  node_smoothed   Eq. gi at pixel centres: the spectrum of the smoothing of
                  one mode equals the ball sum of the Gaussian (numpy).
  interp_gather   reproduces linear (order 1) and quadratic (order 3)
                  fields exactly; node values at zero offset; convergence
                  orders 2 and 3 against Eq. gi on smooth fields.
  linearised      central differences of v -> nu(|v|/a0) v and
                  v -> mu(|v|/a0) v for every kind; y nu'(y), x mu'(x)
                  against central differences of nu and mu.
  solve_increment Newtonian kind: equals the difference of two full solves;
                  linear in the density increment; about a converged base,
                  the central difference of the full iteration with error
                  falling fourfold as the step halves (Sect. 5.2 (v)).
  delta_rho       the integer difference of two deposits is the deposit of
                  the moved particles' new minus old positions, exactly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mond_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmondoracle.so")
_lock = threading.Lock()
_lib = None

MU_DEEP, MU_SIMPLE, MU_STANDARD, MU_NEWTON = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
            L.ora_mu.restype = f64
            L.ora_mu.argtypes = [i32, f64]
            L.ora_nu.restype = f64
            L.ora_nu.argtypes = [i32, f64]
            L.ora_ball_reach.restype = i32
            L.ora_ball_reach.argtypes = [f64]
            L.ora_ball.restype = i32
            L.ora_ball.argtypes = [f64, P, i32]
            L.ora_axis_lut.argtypes = [f64, P]
            L.ora_kacc.restype = i32
            L.ora_kacc.argtypes = [i64, P]
            L.ora_deposit_fixed.restype = i64
            L.ora_deposit_fixed.argtypes = [i32, f64, i64, P, P, P, i32, P]
            L.ora_acc_to_rho.argtypes = [i32, P, i32, f64, P, P]
            L.ora_deposit_exact.argtypes = [i32, f64, f64, i64, P, P, P, P]
            L.ora_dft1.argtypes = [i32, P, P, i32]
            L.ora_fft1.argtypes = [i32, P, i32]
            L.ora_fft3_raw.argtypes = [i32, P, i32]
            L.ora_solve.restype = i32
            L.ora_solve.argtypes = [i32, f64, f64, f64, i32, i32, P, P, i32, P, P, P, P, P, P]
            L.ora_solve_ex.restype = i32
            L.ora_solve_ex.argtypes = [i32, f64, f64, f64, i32, i32, P, P, i32, i32, P, P, P, P, P, P]
            L.ora_solve_increment.restype = i32
            L.ora_solve_increment.argtypes = [i32, f64, f64, f64, i32, i32, P, P, P, P, P, P, P, P]
            L.ora_linearised.argtypes = [i32, i32, f64, P, P, P]
            L.ora_ynu_prime.restype = f64
            L.ora_ynu_prime.argtypes = [i32, f64]
            L.ora_xmu_prime.restype = f64
            L.ora_xmu_prime.argtypes = [i32, f64]
            L.ora_gather.argtypes = [i32, f64, P, i64, P, P, P]
            L.ora_push.argtypes = [i32, f64, f64, i64, P, P, P, P, i32]
            L.ora_particle_diag.argtypes = [i32, f64, i64, P, P, P, P, P]
            L.ora_transform_count.restype = ctypes.c_longlong
            L.ora_num_threads.restype = i32
            L.ora_set_num_threads.restype = i32
            L.ora_set_num_threads.argtypes = [i32]
            L.ora_project_div.argtypes = [i32, f64, P, P]
            L.ora_field_density.argtypes = [i32, f64, f64, P, P]
            L.ora_box_flux_mass.restype = f64
            L.ora_box_flux_mass.argtypes = [i32, f64, f64, P, P, P]
            L.ora_shell_mass.argtypes = [i32, f64, P, P, f64, i32, P]
            L.ora_interp_gather.argtypes = [i32, i32, P, i64, P, P, P]
            L.ora_aqual_solve.restype = i32
            L.ora_aqual_solve.argtypes = [i32, f64, f64, f64, i32, P, P, f64, i32, P, P, P]
            _lib = L
        return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return lib().ora_num_threads()


def set_num_threads(t: int) -> int:
    """Threads of the oracle's parallel loops from now on; returns the count."""
    return lib().ora_set_num_threads(int(t))


def mu(kind: int, x: float) -> float:
    return lib().ora_mu(kind, float(x))


def nu(kind: int, y: float) -> float:
    return lib().ora_nu(kind, float(y))


def ball_reach(sigma: float) -> int:
    return lib().ora_ball_reach(float(sigma))


def ball(sigma: float) -> np.ndarray:
    n = lib().ora_ball(float(sigma), None, 0)
    d = np.zeros((n, 3), np.int32)
    lib().ora_ball(float(sigma), _p(d), n)
    return d


def axis_lut(sigma: float) -> np.ndarray:
    r = ball_reach(sigma)
    t = np.zeros((65537, 2 * r + 1), np.uint32)
    lib().ora_axis_lut(float(sigma), _p(t))
    return t


def kacc(mass) -> int:
    m = _c(mass, np.float32)
    return lib().ora_kacc(m.size, _p(m))


def deposit_fixed(n: int, sigma: float, cell, off, mass, kacc_val: int | None = None):
    """Fixed-point deposit. Returns (acc uint64 [n,n,n] in z,y,x order, kacc, skipped)."""
    cell = _c(cell, np.int32).reshape(-1, 3)
    off = _c(off, np.float32).reshape(-1, 3)
    mass = _c(mass, np.float32).reshape(-1)
    if kacc_val is None:
        kacc_val = kacc(mass)
    acc = np.zeros((n, n, n), np.uint64)
    sk = lib().ora_deposit_fixed(n, float(sigma), mass.size, _p(cell), _p(off), _p(mass), int(kacc_val), _p(acc))
    return acc, int(kacc_val), int(sk)


def acc_to_rho(acc, kacc_val: int, s: float):
    acc = _c(acc, np.uint64)
    n = acc.shape[0]
    r32 = np.zeros(acc.shape, np.float32)
    r64 = np.zeros(acc.shape, np.float64)
    lib().ora_acc_to_rho(n, _p(acc), int(kacc_val), float(s), _p(r32), _p(r64))
    return r32, r64


def deposit_exact(n: int, sigma: float, s: float, cell, off, mass):
    cell = _c(cell, np.int32).reshape(-1, 3)
    off = _c(off, np.float32).reshape(-1, 3)
    mass = _c(mass, np.float32).reshape(-1)
    rho = np.zeros((n, n, n), np.float64)
    lib().ora_deposit_exact(n, float(sigma), float(s), mass.size, _p(cell), _p(off), _p(mass), _p(rho))
    return rho


def dft1(x, sign: int = -1):
    x = _c(x, np.complex128)
    X = np.zeros_like(x)
    lib().ora_dft1(x.size, _p(x), _p(X), int(sign))
    return X


def fft1(x, sign: int = -1):
    x = _c(x, np.complex128).copy()
    lib().ora_fft1(x.size, _p(x), int(sign))
    return x


def fft3_raw(a, sign: int = -1):
    a = _c(a, np.complex128).copy()
    lib().ora_fft3_raw(a.shape[0], _p(a), int(sign))
    return a


def transform_count() -> int:
    return int(lib().ora_transform_count())


def reset_transform_count() -> None:
    lib().ora_reset_transform_count()


def solve(rho, s: float, G: float, a0: float, mu_kind: int, n_iter: int, H0=None,
          finish_h: bool = False, want=("gN", "H", "phi", "acc", "dH"), mean_last2: bool = False):
    """Field solve (App. Flow steps 3-9). rho: [n,n,n] float64 (z,y,x).
    Returns a dict of the requested outputs (vector fields as [3,n,n,n]);
    "gM" (not in the default) is the curl-free g_M of the last iteration.
    mean_last2: the potential is the mean of the last two iterations' (the
    midpoint of the period-2 cycle of reading R14; n_iter >= 2)."""
    rho = _c(rho, np.float64)
    n = rho.shape[0]
    out = {}
    gN = np.zeros((3, n, n, n)) if "gN" in want else None
    H = np.zeros((3, n, n, n)) if "H" in want else None
    phi = np.zeros((n, n, n)) if "phi" in want else None
    acc = np.zeros((3, n, n, n)) if "acc" in want else None
    dH = np.zeros(max(n_iter, 1)) if "dH" in want else None
    gM = np.zeros((3, n, n, n)) if ("gM" in want and n_iter > 0) else None
    H0a = None if H0 is None else _c(H0, np.float64)
    rc = lib().ora_solve_ex(n, float(s), float(G), float(a0), int(mu_kind), int(n_iter), _p(rho), _p(H0a),
                            int(bool(finish_h)), int(bool(mean_last2)), _p(gN), _p(H), _p(phi), _p(acc), _p(dH),
                            _p(gM))
    if rc != 0:
        raise RuntimeError(f"oracle solve failed: {rc}")
    for k, v in (("gN", gN), ("H", H), ("phi", phi), ("acc", acc), ("dH", dH), ("gM", gM)):
        if v is not None:
            out[k] = v
    return out


def aqual_solve(rho, s: float, G: float, a0: float, mu_kind: int, phi0=None, tol: float = 1e-9,
                max_iter: int = 400):
    """The exact solution of the discretised AQUAL equation (the field the
    iteration of Sect. 2.1 would reach if it converged): the minimiser of the
    convex mesh energy sum a0^2 Psi(|D phi|/a0) + g_N . D phi (Psi' = mu(x) x),
    by preconditioned L-BFGS from phi0 (default zero). Returns dict phi,
    acc = -grad_FD phi ([3,n,n,n]), iterations, rel_grad (|grad E| over
    |D^T g_N| at the end) and evals."""
    rho = _c(rho, np.float64)
    n = rho.shape[0]
    phi = np.zeros((n, n, n))
    acc = np.zeros((3, n, n, n))
    info = np.zeros(3)
    p0 = None if phi0 is None else _c(phi0, np.float64)
    rc = lib().ora_aqual_solve(n, float(s), float(G), float(a0), int(mu_kind), _p(rho), _p(p0), float(tol),
                               int(max_iter), _p(phi), _p(acc), _p(info))
    if rc != 0:
        raise RuntimeError(f"oracle AQUAL solve failed: {rc}")
    return {"phi": phi, "acc": acc, "iterations": int(info[0]), "rel_grad": float(info[1]), "evals": int(info[2])}


def solve_increment(drho, s: float, G: float, a0: float, mu_kind: int, n_iter: int, gN0, H0, gM0):
    """Incremental solve (Sect. 5.2 (v)): field increments for the density
    increment drho [n,n,n] about the base (g_N0, H0, g_M0), each [3,n,n,n],
    with the nu and mu steps linearised about F0 = g_N0 + H0 and g_M0.
    Returns dict dgN, dH, dgM, dacc ([3,n,n,n] each)."""
    drho = _c(drho, np.float64)
    n = drho.shape[0]
    gN0, H0, gM0 = (_c(a, np.float64) for a in (gN0, H0, gM0))
    out = {k: np.zeros((3, n, n, n)) for k in ("dgN", "dH", "dgM", "dacc")}
    rc = lib().ora_solve_increment(n, float(s), float(G), float(a0), int(mu_kind), int(n_iter), _p(drho),
                                   _p(gN0), _p(H0), _p(gM0), _p(out["dgN"]), _p(out["dH"]), _p(out["dgM"]),
                                   _p(out["dacc"]))
    if rc != 0:
        raise RuntimeError(f"oracle incremental solve failed: {rc}")
    return out


def linearised(kind: int, which: int, a0: float, P, dv):
    """The linearised nu (which = 0) or mu (which = 1) step of Sect. 5.2 (v)
    about the point P applied to dv (3-vectors)."""
    P = _c(P, np.float64)
    dv = _c(dv, np.float64)
    out = np.zeros(3)
    lib().ora_linearised(int(kind), int(which), float(a0), _p(P), _p(dv), _p(out))
    return out


def delta_rho(acc1, acc0, kacc_val: int, s: float):
    """Density increment of two fixed-point deposits with the same Kacc
    (rule R1): float(double(acc1 - acc0) * 2^-Kacc / s^3), the integer
    difference taken first so that it is exact."""
    d = np.asarray(acc1).astype(np.int64) - np.asarray(acc0).astype(np.int64)
    sc = np.ldexp(1.0, -int(kacc_val)) / (s * s * s)
    return (d.astype(np.float64) * sc).astype(np.float32)


def project_div(field, s: float):
    """Divergence-free part of a vector field [3, n, n, n] (Eq. divH)."""
    f = _c(field, np.float64)
    out = np.zeros_like(f)
    lib().ora_project_div(f.shape[1], float(s), _p(f), _p(out))
    return out


def field_density(g, s: float, G: float):
    """Eq. apparentdensity: -(div_FD g) / (4 pi G) for a field [3, n, n, n]
    (g_N gives rho_B, the MOND acceleration rho_A)."""
    g = _c(g, np.float64)
    out = np.zeros(g.shape[1:])
    lib().ora_field_density(g.shape[1], float(s), float(G), _p(g), _p(out))
    return out


def box_flux_mass(g, s: float, G: float, lo, hi) -> float:
    """Eq. totalmass: -(1/(4 pi G)) times the flux of g out of the box of
    cells lo..hi (inclusive, (x, y, z) order, periodic)."""
    g = _c(g, np.float64)
    lo = np.ascontiguousarray(lo, np.int32)
    hi = np.ascontiguousarray(hi, np.int32)
    return float(lib().ora_box_flux_mass(g.shape[1], float(s), float(G), _p(g), _p(lo), _p(hi)))


def shell_mass(rho, s: float, center, dr: float, nbins: int):
    """Mass rho s^3 in shells [k dr, (k+1) dr) about center (physical (x, y, z),
    cell i at (i - n/2) s, minimum image)."""
    rho = _c(rho, np.float64)
    c = np.ascontiguousarray(center, np.float64)
    out = np.zeros(nbins)
    lib().ora_shell_mass(rho.shape[0], float(s), _p(rho), _p(c), float(dr), int(nbins), _p(out))
    return out


def dipole_layer(n: int, s: float, axis: int, mass: float):
    """Density of the external-field dipole layer (Sect. 5.3): +mass spread
    over the last plane along axis (0, 1, 2 = x, y, z) and -mass over the
    first, as mass per s^3 on [n, n, n] (z, y, x)."""
    rho = np.zeros((n, n, n))
    sl_hi = [slice(None)] * 3
    sl_lo = [slice(None)] * 3
    sl_hi[2 - axis] = n - 1
    sl_lo[2 - axis] = 0
    rho[tuple(sl_hi)] += mass / (n * n * s ** 3)
    rho[tuple(sl_lo)] -= mass / (n * n * s ** 3)
    return rho


def node_smoothed(sigma: float, acc):
    """The force Eq. gi gives a particle sitting on every pixel centre: the
    acceleration mesh [3, n, n, n] smoothed with the ball-truncated Gaussian."""
    acc = _c(acc, np.float64)
    n = acc.shape[1]
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cell = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.int32)
    g = gather(sigma, acc, cell, np.zeros((n ** 3, 3)))
    return np.ascontiguousarray(g.T.reshape(3, n, n, n))


def interp_gather(order: int, S, cell, off):
    """Force at the particles by linear (order 1) or Keys cubic (order 3)
    interpolation of a node field S [3, n, n, n]; returns [N][3]."""
    S = _c(S, np.float64)
    cell = _c(cell, np.int32)
    off = _c(off, np.float64)
    N = cell.shape[0]
    out = np.zeros((N, 3))
    lib().ora_interp_gather(S.shape[1], int(order), _p(S), N, _p(cell), _p(off), _p(out))
    return out


def gather(sigma: float, acc, cell, off):
    acc = _c(acc, np.float64)
    n = acc.shape[1]
    cell = _c(cell, np.int32).reshape(-1, 3)
    off = _c(off, np.float32).reshape(-1, 3)
    g = np.zeros((cell.shape[0], 3))
    lib().ora_gather(n, float(sigma), _p(acc), cell.shape[0], _p(cell), _p(off), _p(g))
    return g


def push(n: int, s: float, dt: float, g, cell, off, vel, drift: bool = True):
    """Kick (and drift). Returns new (cell int32, offset float64, vel float64)."""
    g = _c(g, np.float64).reshape(-1, 3)
    cell = _c(cell, np.int32).reshape(-1, 3).copy()
    off = _c(off, np.float64).reshape(-1, 3).copy()
    vel = _c(vel, np.float64).reshape(-1, 3).copy()
    lib().ora_push(n, float(s), float(dt), cell.shape[0], _p(g), _p(cell), _p(off), _p(vel), int(bool(drift)))
    return cell, off, vel


def particle_diag(n: int, s: float, cell, off, vel, mass):
    cell = _c(cell, np.int32).reshape(-1, 3)
    off = _c(off, np.float64).reshape(-1, 3)
    vel = _c(vel, np.float64).reshape(-1, 3)
    mass = _c(mass, np.float32).reshape(-1)
    out = np.zeros(11)
    lib().ora_particle_diag(n, float(s), mass.size, _p(cell), _p(off), _p(vel), _p(mass), _p(out))
    return {"mass": out[0], "P": out[1:4].copy(), "R": out[4:7].copy(), "L": out[7:10].copy(), "Ekin": out[10]}


def step(n: int, s: float, G: float, a0: float, mu_kind: int, sigma: float, n_iter: int, dt: float,
         cell, off, vel, mass, H0=None, finish_h: bool = False, mean_last2: bool = False):
    """One time step in the order deposit -> solve -> gather -> kick -> drift.
    Returns (cell, off float64, vel float64, g, fields dict, kacc)."""
    acc, ka, _ = deposit_fixed(n, sigma, cell, off, mass)
    _, rho64 = acc_to_rho(acc, ka, s)
    f = solve(rho64, s, G, a0, mu_kind, n_iter, H0=H0, finish_h=finish_h, mean_last2=mean_last2)
    g = gather(sigma, f["acc"], cell, off)
    c2, o2, v2 = push(n, s, dt, g, cell, np.asarray(off, np.float64), vel)
    return c2, o2, v2, g, f, ka
