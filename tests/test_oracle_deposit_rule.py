"""Pins of the deposit's integer rule (reading R1) in the oracle.

The paper fixes the Gaussian of Eq. smooth and a lookup table for the
exponential (Sect. 3.1); where the products of the per-axis weights and the
mass are rounded is a reading. These tests pin that reading tap by tap: a
hand-worked particle (tests/golden/deposit_rule_R1.json), and single particles
whose every tap is recomputed here with Python integers from the stated rule.
Moving a rounding point to another factor (the mass into the y or z word,
or one rounding for the whole product) fails them.
"""
import json
import math
import os
import struct

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "deposit_rule_R1.json")))


def _reach(sigma):
    r = 0
    while (r + 1) * (r + 1) < 16 * sigma * sigma:
        r += 1
    return r


def _word(sigma, u):
    """round_half_even(2^24 g1(u)), g1(u) = exp(-u^2/2 sigma^2)/(sigma sqrt(2 pi))."""
    return round(math.exp(-(u * u) / (2.0 * sigma * sigma)) / (sigma * math.sqrt(2.0 * math.pi)) * 16777216.0)


def _mass_parts(m):
    b = struct.unpack("<I", struct.pack("<f", m))[0]
    e = (b >> 23) & 0xFF
    sig = ((b & 0x7FFFFF) | 0x800000) if e else (b & 0x7FFFFF)
    return sig, (e - 150 if e else -149), b >> 31, max(e, 1)


def _taps(sigma, off, m, N, variant="R1"):
    """{(dx, dy, dz): int64 contribution} of one particle by the rule."""
    r = _reach(sigma)
    q = [round(float(np.float32(o)) * 65536.0) for o in off]
    Wd = [[_word(sigma, (j - r) - q[a] / 65536.0) for j in range(2 * r + 1)] for a in range(3)]
    msig, e2, neg, emax = _mass_parts(m)
    kacc = 62 - (emax - 126) - (N - 1).bit_length()
    sh = 40 - kacc - e2
    out = {}
    for dz in range(-r, r + 1):
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                if dx * dx + dy * dy + dz * dz >= 16 * sigma * sigma:
                    continue
                wx, wy, wz = Wd[0][dx + r], Wd[1][dy + r], Wd[2][dz + r]
                if variant == "R1":  # mass into x, y and z joined
                    P = ((wy * wz + 2 ** 15) >> 16) * ((wx * msig + 2 ** 15) >> 16)
                elif variant == "mass_in_y":
                    P = ((wx * wz + 2 ** 15) >> 16) * ((wy * msig + 2 ** 15) >> 16)
                elif variant == "mass_in_z":
                    P = ((wx * wy + 2 ** 15) >> 16) * ((wz * msig + 2 ** 15) >> 16)
                else:  # one rounding of the whole product
                    P = (wx * wy * wz * msig + 2 ** 31) >> 32
                c = (P + (1 << (sh - 1))) >> sh if sh > 0 else P << (-sh)
                out[(dx, dy, dz)] = -c if neg else c
    return out


def _oracle_single(n, sigma, cell, off, m):
    acc, ka, _ = oracle.deposit_fixed(n, sigma, np.array([cell], np.int32), np.array([off], np.float32),
                                      np.array([m], np.float32))
    return acc.view(np.int64), ka


def test_hand_worked_particle():
    c = GOLD["case"]
    acc, ka = _oracle_single(c["n"], c["sigma"], c["cell"], c["offset"], c["mass"])
    assert ka == 61
    x, y, z = c["cell"]
    a = GOLD["acc"]
    assert int(acc[z, y, x]) == a["centre (0,0,0)"]
    assert int(acc[z, y, x + 1]) == a["x neighbour (1,0,0)"]
    assert int(acc[z, y + 1, x]) == a["y neighbour (0,1,0)"]
    assert int(acc[z + 1, y, x]) == a["z neighbour (0,0,1)"]
    assert abs(int(acc[z, y, x]) * 2.0 ** -61 - (2 * math.pi) ** -1.5) < 1e-8


@pytest.mark.parametrize("sigma,off,m", [
    (0.75, (0.5, -0.5, 0.0), 1.0),
    (1.0, (0.123456, -0.37, 0.49), 3.7e-6),
    (1.5, (-0.25, 2.0 ** -17, -3 * 2.0 ** -17), -0.8125),  # half-way offsets: ties to even
    (2.0, (0.3141, 0.0, -0.2718), 1e-6),
])
def test_every_tap_follows_the_rule(sigma, off, m):
    n = 32
    cell = (16, 15, 17)
    acc, _ = _oracle_single(n, sigma, cell, off, m)
    want = _taps(sigma, off, m, 1)
    seen = np.zeros_like(acc, dtype=bool)
    for (dx, dy, dz), c in want.items():
        j = ((cell[2] + dz) % n, (cell[1] + dy) % n, (cell[0] + dx) % n)
        assert int(acc[j]) == c, (dx, dy, dz)
        seen[j] = True
    assert not acc[~seen].any()
    # each moved rounding point gives other integers somewhere in the ball
    for variant in ("mass_in_y", "mass_in_z", "single"):
        alt = _taps(sigma, off, m, 1, variant)
        assert any(alt[k] != want[k] for k in want), variant


def test_kacc_follows_particle_count_and_largest_mass():
    # Kacc = 62 - (emax - 126) - ceil(log2 N): the total of N particles of the largest mass fits below 2^62
    for N, m, want in ((1, 1.0, 61), (2, 1.0, 60), (3, 1.0, 59), (1000, 1e-3, 62 - (117 - 126) - 10)):
        assert oracle.kacc(np.full(N, m, np.float32)) == want
