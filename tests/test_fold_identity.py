"""The folded form of the curl-free, final and Newton steps (MOND_OPT_FOLD) is
an exact restatement of the three-component operators: FP64 numpy model of
the pass sequence, index logic as the kernels have it (y blocks of 8 columns,
z blocks of 16 at n = 32; the block holding kx = n/2 and the row ky = n/2
unfolded), against the projection written out component by component.

Curl-free projection (Eq. rotg): P_ab = k_a k_b A, the off-diagonal terms
dropped where exactly one of a, b lies on its Nyquist plane; final step
(App. Flow step 9): phi^ = i A sum_b k'_b g_b (k'_b = 0 on b's Nyquist plane),
a^ = -i kappa phi^ with kappa = sin(k s)/s.
"""
import numpy as np
import pytest

N = 32
H = N // 2
PY, PZ = 8, 16  # columns per folded y tile and per z tile at this size


def kvecs(n, s=1.0):
    f = np.array([i if i < (n + 1) // 2 else i - n for i in range(n)])
    k = 2 * np.pi * f / (n * s)
    kap = np.where(np.arange(n) * 2 == n, 0.0, np.sin(2 * np.pi * f / n) / s)
    return k, kap


K, KAP = kvecs(N)
KX, KY, KZ = K[None, None, :H + 1], K[None, :, None], K[:, None, None]
NX = (np.arange(H + 1) == H)[None, None, :]
NY = (np.arange(N) == H)[None, :, None]
NZ = (np.arange(N) == H)[:, None, None]
KK = KX ** 2 + KY ** 2 + KZ ** 2
A = np.where(KK > 0, 1.0 / np.where(KK > 0, KK, 1.0), 0.0)
NORM = 1.0 / N ** 3


def yf(a):
    return np.fft.fft(a, axis=1)


def yi(a):
    return np.fft.ifft(a, axis=1) * N


def zf(a):
    return np.fft.fft(a, axis=0)


def zi(a):
    return np.fft.ifft(a, axis=0) * N


def spectra(seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((N, N, H + 1)) + 1j * rng.standard_normal((N, N, H + 1)) for _ in range(3)]


def curl_three(g):
    gs = [zf(yf(c)) for c in g]
    k3, n3 = [KX, KY, KZ], [NX, NY, NZ]
    out = []
    for a in range(3):
        acc = 0
        for b in range(3):
            acc = acc + np.where(n3[a] == n3[b], gs[b] * k3[a] * k3[b] * A, 0)
        out.append(yi(zi(acc * NORM)))
    return out


def final_three(g):
    gs = [zf(yf(c)) for c in g]
    k3, n3 = [KX, KY, KZ], [NX, NY, NZ]
    S = sum(np.where(~n3[b], gs[b] * k3[b], 0) for b in range(3))
    aS = S * A * NORM
    return [yi(zi(aS * kk)) for kk in (KAP[None, None, :H + 1], KAP[None, :, None], KAP[:, None, None])]


def fold(g):
    """Folded y-pass: s = kx gx^ + ky gy^ into component 0 except in the
    block holding kx = N/2 and on the row ky = N/2 (there gx^ stays, and gy^
    goes to component 1)."""
    gx, gy, gz = [yf(c) for c in g]
    s0, s1 = gx.copy(), gy.copy()
    nb = (H + 1 + PY - 1) // PY
    for blk in range(nb - 1):
        cols = slice(blk * PY, (blk + 1) * PY)
        rows = np.arange(N) != H
        s0[:, rows, cols] = KX[0, 0, cols] * gx[:, rows, cols] + K[rows][None, :, None] * gy[:, rows, cols]
    return [s0, s1, gz]


def zpass(w, mode):
    """Folded z-pass: the tiles holding kx = N/2 or ky = N/2 as three
    components (outputs unfolded, as the three-component pass writes them),
    the others from (s, gz^) to (u, z output)."""
    nbz = (H + 1 + PZ - 1) // PZ
    ws = [zf(c) for c in w]
    out = [np.zeros_like(w[0]) for _ in range(3)]
    for blk in range(nbz):
        cols = slice(blk * PZ, min(H + 1, (blk + 1) * PZ))
        for y in range(N):
            if y == H or blk == nbz - 1:
                gg = [c[:, y, cols] for c in ws]
                kx, ky, kz = KX[0, 0, cols][None, :], K[y], KZ[:, 0, :]
                nx, ny, nz = NX[0, 0, cols][None, :], y == H, NZ[:, 0, :]
                a = A[:, y, cols]
                k3, n3 = [kx, ky, kz], [nx, ny, nz]
                if mode == "curl":
                    for c in range(3):
                        acc = 0
                        for b in range(3):
                            acc = acc + np.where(n3[c] == n3[b], gg[b] * k3[c] * k3[b] * a, 0)
                        out[c][:, y, cols] = zi(acc * NORM)
                else:
                    S = sum(np.where(~np.broadcast_to(n3[b], a.shape), gg[b] * k3[b], 0) for b in range(3))
                    aS = S * a * NORM
                    for c, kap in enumerate((KAP[:H + 1][cols][None, :], KAP[y], KAP[:, None])):
                        out[c][:, y, cols] = zi(aS * kap)
            else:
                s, gz = ws[0][:, y, cols], ws[2][:, y, cols]
                kz, nz, a = KZ[:, 0, :], NZ[:, 0, :], A[:, y, cols]
                if mode == "curl":
                    u = np.where(nz, s * a, (s + gz * kz) * a) * NORM
                    v = np.where(nz, gz * kz * kz * a, (s + gz * kz) * a * kz) * NORM
                else:
                    u = np.where(nz, s, s + gz * kz) * a * NORM
                    v = u * KAP[:, None]
                out[0][:, y, cols] = zi(u)
                out[2][:, y, cols] = zi(v)
    return out


def unfold(w, mode):
    """Unfolding y-pass: kx u and ky u (k for the curl-free step, kappa for
    the gradients) before the inverse, the unfolded block and row as they are."""
    kt = K if mode == "curl" else KAP
    nb = (H + 1 + PY - 1) // PY
    o0, o1 = w[0].copy(), w[1].copy()
    for blk in range(nb - 1):
        cols = slice(blk * PY, (blk + 1) * PY)
        rows = np.arange(N) != H
        u = w[0][:, rows, cols]
        o1[:, rows, cols] = u * kt[rows][None, :, None]
        o0[:, rows, cols] = u * kt[:H + 1][cols][None, None, :]
    return [yi(o0), yi(o1), yi(w[2])]


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("mode", ["curl", "final"])
def test_folded_passes_equal_three_component_operators(mode, seed):
    g = spectra(seed)
    ref = curl_three(g) if mode == "curl" else final_three(g)
    got = unfold(zpass(fold(g), mode), mode)
    for a in range(3):
        assert np.abs(got[a] - ref[a]).max() <= 1e-12 * np.abs(ref[a]).max()


def test_fold_without_the_nyquist_split_is_wrong():
    """Folding the Nyquist block and row as well (a plausible mistake) breaks
    the curl-free projection there, so the comparison above can fail."""
    g = spectra(2)
    ref = curl_three(g)
    gx, gy, gz = [yf(c) for c in g]
    s = KX * gx + KY * gy
    ws = [zf(s), None, zf(gz)]
    u = (ws[0] + ws[2] * KZ) * A * NORM
    got = [yi(zi(u) * KX), yi(zi(u) * KY), yi(zi(u * KZ))]
    assert max(np.abs(got[a] - ref[a]).max() / np.abs(ref[a]).max() for a in range(3)) > 1e-6
