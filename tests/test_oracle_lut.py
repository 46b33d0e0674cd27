"""Pins for the oracle's restatement of the paper's lookup-table random bits
(section 3.2): the table against its closed form in 80-digit arithmetic;
the generated bits' frequency (p = exp(-4J/T)), pairwise independence and
the two-word AND (p^2 = exp(-8J/T)); the dynamics against Kaufman's exact
energy of the 64 x 64 torus and Onsager below Tc; the exact +-flip symmetry.
"""
import math

import mpmath
import numpy as np
import pytest

import physics as ph

mpmath.mp.dps = 80
TC = ph.TC


@pytest.mark.parametrize("J,T", [(1.0, TC), (1.0, 0.9 * TC), (1.0, 1.3 * TC), (0.5, 1.0), (1.0, 0.3), (1.0, 50.0)])
def test_table_closed_form(orc, J, T):
    tbl = orc.lut_table(J, T)
    p = mpmath.exp(-4 * mpmath.mpf(J) / mpmath.mpf(T))
    cum = mpmath.mpf(0)
    for j in range(16):
        exact = int(mpmath.floor(mpmath.ldexp(cum, 32)))
        assert abs(int(tbl[j]) - min(exact, 2**32 - 1)) <= 1, (j, int(tbl[j]), exact)
        k = bin(j).count("1")
        cum += p**k * (1 - p) ** (4 - k)
    assert tbl[0] == 0 and all(tbl[i] <= tbl[i + 1] for i in range(15))


def test_bits_have_the_stated_distribution(orc):
    J, T = 1.0, TC
    tbl = orc.lut_table(J, T)
    p = math.exp(-4 * J / T)
    n = 3000
    w0 = np.array([orc.lut_word(11, tbl, w, 5, 1, 0) for w in range(n)], dtype=np.uint64)
    w1 = np.array([orc.lut_word(11, tbl, w, 5, 1, 1) for w in range(n)], dtype=np.uint64)
    bits0 = ((w0[:, None] >> np.arange(32, dtype=np.uint64)) & 1).astype(np.float64)
    bits1 = ((w1[:, None] >> np.arange(32, dtype=np.uint64)) & 1).astype(np.float64)
    N = bits0.size
    for f, q in [(bits0.mean(), p), (bits1.mean(), p), ((bits0 * bits1).mean(), p * p)]:
        assert abs(f - q) < 4 * math.sqrt(q * (1 - q) / N), (f, q)
    # bits of one lookup (k, k+1) and of different lookups (k, k+4) are independent
    for a, b in [(0, 1), (2, 3), (1, 5), (30, 31)]:
        f = (bits0[:, a] * bits0[:, b]).mean()
        assert abs(f - p * p) < 4 * math.sqrt(p * p / n), (a, b, f)


def _energy(orc, L, T, seed, sweeps, discard, ordered):
    tbl = orc.lut_table(1.0, T)
    s = np.ones((L, L), dtype=np.int8) if ordered else orc.init(0, L, seed)
    obs = orc.run_lut(s, seed, tbl, 0, sweeps)[discard:]
    return ph.binned(-obs[:, 1].astype(np.float64) / (L * L), 30)


@pytest.mark.parametrize("T,ordered", [(0.9 * TC, True), (1.3 * TC, False)])
def test_energy_matches_kaufman_on_the_64_torus(orc, T, ordered):
    L = 64
    mean, err = _energy(orc, L, T, 17, 3000, 300, ordered)
    u = ph.kaufman_u(L, T)
    assert err < 3e-3
    assert abs(mean - u) < 4 * err + 1e-4, (mean, u, err)
    if T < TC:
        assert abs(u - ph.onsager_u(T)) < 1e-6  # far below Tc the 64-torus is at the thermodynamic limit


def test_flip_symmetry(orc):
    L, seed = 128, 4
    tbl = orc.lut_table(1.0, TC)
    a = orc.init(0, L, seed)
    b = (-a).astype(np.int8)
    for t in range(12):
        orc.sweep_lut(a, seed, tbl, t)
        orc.sweep_lut(b, seed, tbl, t)
        assert np.array_equal(a, -b)


def test_strip_form_equals_full_sweep(orc):
    L, seed, t = 128, 21, 5
    tbl = orc.lut_table(1.0, TC)
    s = orc.init(0, L, seed)
    for i in range(t):
        orc.sweep_lut(s, seed, tbl, i)
    full = orc.sweep_lut(s.copy(), seed, tbl, t)
    for y0, H in [(0, 8), (60, 5), (126, 4)]:
        strip = np.ascontiguousarray(s[[(y0 - 2 + i) % L for i in range(H + 4)]])
        orc.sweep_strip_lut(L, seed, tbl, t, y0, strip)
        assert np.array_equal(strip[2:H + 2], full[[(y0 + i) % L for i in range(H)]])
