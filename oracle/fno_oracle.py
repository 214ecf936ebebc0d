"""FP64 CPU oracle of the learned warm start (Fourier neural operator).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
leg of ``bench.py`` are its only callers. It shares no code with the CUDA
library and imports nothing from it.

The paper seeds its iteration with the previous step's H (Sect. 5.2, item iv)
and has no network; the network and its parameter layout are fixed by the
library's C header for the surrogate and restated here from that definition:

  x (4 channels) -> v_0 = P x + p
  z_l = W_l v_l + b_l + K_l v_l,   v_{l+1} = gelu(z_l)  (l < L-1),  v_L = z_{L-1}
  y = Q v_L + q (3 channels)
  K_l v = (1/V) sum_k a(k_x) Re( t(k) e^{+2 pi i k.x/n} ),
  t_c(k) = sum_j R_l[k][j][c] s_j(k),  s_j(k) = sum_x v_j(x) e^{-2 pi i k.x/n}
over the kept modes k_x in [0, M), k_y, k_z in {0..M-1, -M..-1}; a(0) = 1,
a(k_x > 0) = 2 (the conjugate half of a real field); gelu is the tanh form.

numpy's FFTs serve as library primitives for the truncated transforms; the
backward pass is the chain rule of the definition above, written out, and is
pinned by central finite differences of the forward pass.

Pins (tests/test_fno_oracle.py): the truncated transform against a brute-force
DFT sum; the spectral layer as the identity on band-limited fields; gradients
against central differences; bfloat16 rounding on hand-worked values and
against torch's conversion; GELU against the erf form; Adam's first step in
closed form; block means and cubic-convolution upsampling on constant,
linear and quadratic fields; the sphere-mixture density against the
closed-form enclosed masses.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------- parameters
class Shape:
    def __init__(self, n: int, width: int, modes: int, layers: int):
        self.n, self.C, self.M, self.L = n, width, modes, layers
        self.V = n ** 3
        self.K = modes * (2 * modes) * (2 * modes)

    def layer_size(self):
        return self.C * self.C + self.C + 2 * self.K * self.C * self.C

    def count(self):
        return 5 * self.C + self.L * self.layer_size() + 3 * self.C + 3


def unpack(flat: np.ndarray, sh: Shape) -> dict:
    """Views of the flat parameter array: P [C][4], p [C], per layer W [C][C],
    b [C], R [K][C][C] complex (R[k][j][c]: input j -> output c), Q [3][C], q [3]."""
    flat = np.asarray(flat, np.float64)
    C, K = sh.C, sh.K
    o = 0

    def take(cnt):
        nonlocal o
        a = flat[o:o + cnt]
        o += cnt
        return a

    d = {"P": take(4 * C).reshape(C, 4), "p": take(C), "W": [], "b": [], "R": []}
    for _ in range(sh.L):
        d["W"].append(take(C * C).reshape(C, C))
        d["b"].append(take(C))
        r = take(2 * K * C * C).reshape(K, C, C, 2)
        d["R"].append(r[..., 0] + 1j * r[..., 1])
    d["Q"] = take(3 * C).reshape(3, C)
    d["q"] = take(3)
    assert o == sh.count()
    return d


def pack(d: dict, sh: Shape) -> np.ndarray:
    parts = [d["P"].ravel(), d["p"].ravel()]
    for l in range(sh.L):
        r = np.stack([d["R"][l].real, d["R"][l].imag], -1)
        parts += [d["W"][l].ravel(), d["b"][l].ravel(), r.ravel()]
    parts += [d["Q"].ravel(), d["q"].ravel()]
    return np.concatenate(parts).astype(np.float64)


def bf16_round(a: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float64.
    Finite inputs only."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ------------------------------------------------------- truncated transforms
def _mode_index(n: int, M: int):
    f = np.concatenate([np.arange(M), np.arange(-M, 0)])
    return np.mod(f, n)  # numpy FFT index of each kept frequency


def spec_fwd(v: np.ndarray, M: int) -> np.ndarray:
    """s_j(k) for the kept modes: v [C][n][n][n] (z, y, x) -> [C][K] with
    k = (kz 2M + ky) M + kx."""
    C, n = v.shape[0], v.shape[1]
    f = np.fft.rfftn(v, axes=(1, 2, 3))  # e^{-2 pi i k.x/n}, no scaling
    idx = _mode_index(n, M)
    sub = f[:, idx][:, :, idx][:, :, :, :M]  # [C][2M][2M][M]
    return sub.reshape(C, -1)


def spec_inv(t: np.ndarray, n: int, M: int) -> np.ndarray:
    """(1/V) sum_k a(kx) Re(t(k) e^{+2 pi i k.x/n}) over the kept modes:
    [C][K] -> [C][n][n][n]."""
    C = t.shape[0]
    full = np.zeros((C, n, n, n // 2 + 1), np.complex128)
    idx = _mode_index(n, M)
    tt = t.reshape(C, 2 * M, 2 * M, M)
    for a, iz in enumerate(idx):
        for b, iy in enumerate(idx):
            full[:, iz, iy, :M] = tt[:, a, b, :]
    return np.fft.irfftn(full, s=(n, n, n), axes=(1, 2, 3))


def spec_inv_adjoint(g: np.ndarray, n: int, M: int) -> np.ndarray:
    """Adjoint of spec_fwd as a map into real fields: sum_k Re(g(k) e^{+2 pi i k.x/n})
    (weight 1, no 1/V)."""
    C = g.shape[0]
    gg = g.reshape(C, 2 * M, 2 * M, M)
    out = np.zeros((C, n, n, n))
    idx = _mode_index(n, M)
    full = np.zeros((C, n, n, n), np.complex128)
    for a, iz in enumerate(idx):
        for b, iy in enumerate(idx):
            full[:, iz, iy, :M] = gg[:, a, b, :]
    out = np.real(np.fft.ifftn(full, axes=(1, 2, 3))) * (n ** 3)
    return out


def mix(s: np.ndarray, R: np.ndarray) -> np.ndarray:
    """t_c(k) = sum_j R[k][j][c] s_j(k)."""
    return np.einsum("kjc,jk->ck", R, s)


# ---------------------------------------------------------------- activation
_K0 = math.sqrt(2.0 / math.pi)
_K1 = 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(_K0 * (z + _K1 * z ** 3)))


def gelu_grad(z):
    th = np.tanh(_K0 * (z + _K1 * z ** 3))
    return 0.5 * (1.0 + th) + 0.5 * z * (1.0 - th * th) * _K0 * (1.0 + 3.0 * _K1 * z * z)


# ------------------------------------------------------------ forward/backward
def _pw(Wm, bvec, v):
    """Pointwise channel map: out[o] = sum_i W[o][i] v[i] + b[o]; v [Cin][...]."""
    out = np.tensordot(Wm, v, axes=([1], [0]))
    if bvec is not None:
        out += bvec.reshape((-1,) + (1,) * (v.ndim - 1))
    return out


def forward(flat: np.ndarray, x: np.ndarray, sh: Shape):
    """x [4][n][n][n] -> y [3][n][n][n], and the cache for backward."""
    d = unpack(flat, sh)
    x = np.asarray(x, np.float64)
    v = _pw(d["P"], d["p"], x)
    cache = {"x": x, "v": [v], "z": [], "s": []}
    for l in range(sh.L):
        s = spec_fwd(v, sh.M)
        z = _pw(d["W"][l], d["b"][l], v) + spec_inv(mix(s, d["R"][l]), sh.n, sh.M)
        cache["s"].append(s)
        cache["z"].append(z)
        v = gelu(z) if l + 1 < sh.L else z
        cache["v"].append(v)
    y = _pw(d["Q"], d["q"], v)
    return y, cache


def backward(flat: np.ndarray, cache: dict, dy: np.ndarray, sh: Shape) -> np.ndarray:
    """d loss / d params (flat layout) from dy = d loss / d y."""
    d = unpack(flat, sh)
    n, M, V = sh.n, sh.M, sh.V
    g = {"P": None, "p": None, "W": [None] * sh.L, "b": [None] * sh.L, "R": [None] * sh.L}
    dy = np.asarray(dy, np.float64)
    vL = cache["v"][sh.L]
    g["Q"] = np.tensordot(dy, vL, axes=([1, 2, 3], [1, 2, 3]))
    g["q"] = dy.sum(axis=(1, 2, 3))
    dv = np.tensordot(d["Q"].T, dy, axes=([1], [0]))
    kx = np.arange(sh.K) % M
    alpha = np.where(kx == 0, 1.0, 2.0)
    for l in range(sh.L - 1, -1, -1):
        z = cache["z"][l]
        vl = cache["v"][l]
        dz = dv * gelu_grad(z) if l + 1 < sh.L else dv
        g["W"][l] = np.tensordot(dz, vl, axes=([1, 2, 3], [1, 2, 3]))
        g["b"][l] = dz.sum(axis=(1, 2, 3))
        dv = np.tensordot(d["W"][l].T, dz, axes=([1], [0]))
        # spectral part: G_t(k) = a(kx)/V * DFT(dz)(k) is dL/dRe t + i dL/dIm t
        Gt = spec_fwd(dz, M) * (alpha / V)[None, :]
        s = cache["s"][l]
        g["R"][l] = np.einsum("jk,ck->kjc", np.conj(s), Gt)
        Gs = np.einsum("kjc,ck->jk", np.conj(d["R"][l]), Gt)
        dv = dv + spec_inv_adjoint(Gs, n, M)
    g["P"] = np.tensordot(dv, cache["x"], axes=([1, 2, 3], [1, 2, 3]))
    g["p"] = dv.sum(axis=(1, 2, 3))
    return pack(g, sh)


# ---------------------------------------------------------- loss and optimiser
def loss(y: np.ndarray, t: np.ndarray, weight: float = 1.0):
    """weight * |y - t|^2 / |t|^2 and its gradient."""
    y = np.asarray(y, np.float64)
    t = np.asarray(t, np.float64)
    tn = float(np.sum(t * t))
    r = y - t
    return weight * float(np.sum(r * r)) / tn, 2.0 * weight * r / tn


def adam(p, g, m, v, lr, b1, b2, eps, step):
    """One Adam step (bias-corrected moments); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ----------------------------------------------- mesh <-> network grid maps
def coarsen(fine: np.ndarray, n: int) -> np.ndarray:
    """Means over f^3 blocks: [c][N][N][N] -> [c][n][n][n], f = N / n."""
    c, N = fine.shape[0], fine.shape[1]
    f = N // n
    return np.asarray(fine, np.float64).reshape(c, n, f, n, f, n, f).mean(axis=(2, 4, 6))


def features(gN_fine: np.ndarray, n: int, a0: float):
    """Network input from the fine Newtonian field: block means, scaled by
    their RMS s, plus log10(|g_N|/a0)/4 of the coarse field."""
    g = coarsen(gN_fine, n)
    s = math.sqrt(float(np.mean(g * g)))
    mag = np.sqrt(np.sum(g * g, axis=0))
    x = np.concatenate([g / s, (0.25 * np.log10(mag / a0 + 1e-12))[None]], 0)
    return x, s


def cubic_weights(u):
    """Cubic convolution (Keys, a = -1/2) weights of the taps -1, 0, 1, 2 at
    fraction u in [0, 1); they sum to 1 and reproduce quadratics."""
    u = np.asarray(u, np.float64)
    return np.stack([((-u + 2) * u - 1) * u / 2, ((3 * u - 5) * u * u + 2) / 2, ((-3 * u + 4) * u + 1) * u / 2,
                     (u - 1) * u * u / 2])


def upsample(y: np.ndarray, N: int, scale: float) -> np.ndarray:
    """Periodic cubic-convolution interpolation of a cell-centred coarse field
    onto the fine cell centres, times scale: [c][n]^3 -> [c][N]^3."""
    c, n = y.shape[0], y.shape[1]
    f = N // n
    u = (np.arange(N) + 0.5) / f - 0.5
    i0 = np.floor(u).astype(np.int64)
    w = cubic_weights(u - i0)  # [4][N]
    out = np.zeros((c, N, N, N))
    for a in range(4):
        iz = np.mod(i0 + a - 1, n)
        for b in range(4):
            iy = np.mod(i0 + b - 1, n)
            for d in range(4):
                ix = np.mod(i0 + d - 1, n)
                wt = w[a][:, None, None] * w[b][None, :, None] * w[d][None, None, :]
                out += y[:, iz][:, :, iy][:, :, :, ix] * wt[None]
    return scale * out


def mixture_density(N: int, s: float, centre, mass, radius, kind, rmax: float) -> np.ndarray:
    """Plummer (kind 0): 3M/(4 pi a^3) (1 + r^2/a^2)^{-5/2}; Hernquist (kind 1):
    M a / (2 pi r (r + a)^3) with r >= 1/2; both zero beyond rmax; radii and
    positions in pixels from the domain centre, density per s^3; [z][y][x]."""
    c = np.arange(N) - N // 2
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    rho = np.zeros((N, N, N))
    for j in range(len(mass)):
        r = np.sqrt((X - centre[j][0]) ** 2 + (Y - centre[j][1]) ** 2 + (Z - centre[j][2]) ** 2)
        a, m = float(radius[j]), float(mass[j])
        if int(kind[j]) == 0:
            prof = 3.0 * m / (4 * math.pi * a ** 3) * (1.0 + r * r / (a * a)) ** -2.5
        else:
            rr = np.maximum(r, 0.5)
            prof = m * a / (2 * math.pi * rr * (rr + a) ** 3)
        rho += np.where(r <= rmax, prof, 0.0)
    return rho / s ** 3
