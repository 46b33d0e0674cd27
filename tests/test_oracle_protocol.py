"""Pins of the oracle's section 3.3 correlation protocol.

The protocol's integers come from floating-point formulas (r_c(t), the
log-spaced distances floor(2^(x/32)), the measurement times
floor(2^(x/8) + 0.5)).  Each is checked here against arithmetic that owes
nothing to FP64: 60-digit decimal for r_c, exact integer roots for the two
power-of-two sequences.  The downsampled sums are checked against the
all-sites correlation at R = 1 and against a numpy array form (strided
sources, rolled targets).
"""
from decimal import Decimal, getcontext

import numpy as np
import pytest

getcontext().prec = 60

LS = [64, 128, 192, 256, 320, 1024, 4096, 1 << 14, 3 << 13, 1 << 16, 1 << 17, 1 << 19, 1 << 20]


def _exact_rc(L: int, t: int) -> int:
    g = 6 * ((Decimal(L) / Decimal(65536)).ln() / (Decimal("3.3") ** 2) + 1).sqrt()
    v = int((g * Decimal(t).sqrt() + Decimal("0.5")).to_integral_value(rounding="ROUND_FLOOR"))
    return max(256, v)


def _iroot(n: int, k: int) -> int:
    """floor(n^(1/k)) for integers, by bisection on exact integer powers."""
    lo, hi = 0, 1 << (n.bit_length() // k + 1)
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if mid ** k <= n:
            lo = mid
        else:
            hi = mid - 1
    return lo


def _exact_distances(L: int, t: int, R: int) -> list[int]:
    rc = _exact_rc(L, t)
    half = L // 2
    out = list(range(2 * R + 1, min(rc, half) + 1))
    last = out[-1] if out else 0
    x = 1
    while True:
        r = _iroot(1 << x, 32)  # floor(2^(x/32))
        if r > half:
            break
        if r > rc and r > last:
            out.append(r)
            last = r
        x += 1
    return out


def _exact_times(tmax: int) -> list[int]:
    out, x = [], 1
    while True:
        # floor(2^(x/8) + 1/2) = floor((floor(2^((x+8)/8)) + 1) / 2)
        t = (_iroot(1 << (x + 8), 8) + 1) // 2
        if t > tmax:
            break
        if not out or t != out[-1]:
            out.append(t)
        x += 1
    return out


def test_rc_matches_decimal_arithmetic(orc):
    ts = list(range(1, 1500)) + [int(v) for v in _exact_times(1 << 34)] + [10**6 + 7, 524288, 10**9]
    for L in LS:
        for t in ts:
            assert orc.protocol_rc(L, t) == _exact_rc(L, t), (L, t)


def test_rc_special_values(orc):
    # g(2^16) = 6: r_c = max(256, floor(6 sqrt(t) + 1/2))
    assert orc.protocol_rc(1 << 16, 1) == 256
    assert orc.protocol_rc(1 << 16, 10000) == 600
    assert orc.protocol_rc(1 << 16, 1822) == 256  # 6 sqrt(1822) + 0.5 = 256.6
    assert orc.protocol_rc(1 << 16, 1823) == 256  # 256.68
    assert orc.protocol_rc(1 << 16, 1850) == 258  # 258.57
    # g grows with L, slowly: g(2^22) = 6 sqrt(1 + 6 ln2 / 3.3^2)
    g22 = 6 * np.sqrt(1 + 6 * np.log(2) / 3.3**2)
    assert orc.protocol_rc(1 << 20, 1 << 20) == max(256, int(np.floor(6 * np.sqrt(1 + 4 * np.log(2) / 3.3**2) * 1024 + 0.5)))
    assert 6.0 < g22 < 7.3


@pytest.mark.parametrize("L", LS)
@pytest.mark.parametrize("t", [1, 2, 100, 1000, 1850, 10**5, 10**7])
def test_distances_match_exact_integers(orc, L, t):
    got = orc.protocol_distances(L, t, 16).tolist()
    assert got == _exact_distances(L, t, 16)


@pytest.mark.parametrize("L,t", [(1 << 17, 1000), (1 << 20, 1), (1 << 16, 10**6), (4096, 10), (1 << 19, 7 * 10**6)])
def test_distance_set_structure(orc, L, t):
    R = 16
    d = orc.protocol_distances(L, t, R).astype(np.int64)
    rc = orc.protocol_rc(L, t)
    assert np.all(np.diff(d) > 0) and d[0] == 2 * R + 1 and d[-1] == L // 2
    dense = d[d <= rc]
    assert np.array_equal(dense, np.arange(2 * R + 1, min(rc, L // 2) + 1))
    # beyond r_c: 32 distances per octave (2^k, 2^(k+1)] once the octave lies above r_c
    for k in range(int(np.log2(rc)) + 1, int(np.log2(L)) - 1):
        sel = d[(d > (1 << k)) & (d <= (1 << (k + 1)))]
        assert sel.size == 32, (k, sel.size)
        assert sel[-1] == 1 << (k + 1)


def test_small_lattice_has_only_the_dense_part(orc):
    # r_c >= 256 >= L/2: every r in (2R, L/2]
    for L in (128, 256, 320, 512):
        assert orc.protocol_distances(L, 50, 16).tolist() == list(range(33, L // 2 + 1))
    assert orc.protocol_distances(64, 50, 16).size == 0  # L/2 = 32 = 2R


def test_times_match_exact_integers(orc):
    for tmax in (1, 2, 13, 100, 1000, 524288, 1 << 40):
        assert orc.protocol_times(tmax).tolist() == _exact_times(tmax)
    t = orc.protocol_times(1 << 20).astype(np.int64)
    # 8 times per octave once they are distinct; powers of two are hit exactly
    assert np.sum((t > 1 << 10) & (t <= 1 << 11)) == 8
    assert all((1 << k) in set(t.tolist()) for k in range(21))
    assert t[:13].tolist() == list(range(1, 14))


def _numpy_sampled(s, R, rs):
    src = s[::R, ::R].astype(np.int64)
    cx = [int(np.sum(src * np.roll(s, -r, axis=1)[::R, ::R])) for r in rs]
    cy = [int(np.sum(src * np.roll(s, -r, axis=0)[::R, ::R])) for r in rs]
    return np.array(cx, dtype=np.int64), np.array(cy, dtype=np.int64)


@pytest.mark.parametrize("vals", [(-1, 1), (-1, 0, 1)])
@pytest.mark.parametrize("L,R", [(64, 16), (64, 4), (96, 16), (128, 32), (64, 64), (80, 8)])
def test_sampled_matches_numpy(orc, vals, L, R):
    rng = np.random.default_rng(L * 7 + R)
    s = np.asarray(vals, dtype=np.int8)[rng.integers(0, len(vals), size=(L, L))]
    rs = list(range(0, L // 2 + 1)) + [L - 1, 1, 17]
    cx, cy = orc.correlation_sampled(s, R, rs)
    ex, ey = _numpy_sampled(s, R, rs)
    assert np.array_equal(cx, ex) and np.array_equal(cy, ey)


def test_sampled_at_R1_is_the_full_correlation(orc):
    rng = np.random.default_rng(3)
    s = np.asarray((-1, 0, 1), dtype=np.int8)[rng.integers(0, 3, size=(48, 48))]
    fx, fy = orc.correlation(s, 24)
    cx, cy = orc.correlation_sampled(s, 1, range(25))
    assert np.array_equal(cx, fx) and np.array_equal(cy, fy)


def test_sampled_special_cases(orc):
    L, R = 128, 16
    ones = np.ones((L, L), dtype=np.int8)
    cx, cy = orc.correlation_sampled(ones, R, [0, 5, 64])
    assert np.all(cx == (L // R) ** 2) and np.all(cy == (L // R) ** 2)
    # a stripe pattern s = (-1)^x: C_x(r) = (L/R)^2 (-1)^r, C_y(r) = (L/R)^2
    stripes = np.where(np.arange(L)[None, :] % 2 == 0, 1, -1).astype(np.int8).repeat(L, 0)
    cx, cy = orc.correlation_sampled(stripes, R, [1, 2, 33])
    assert cx.tolist() == [-(L // R) ** 2, (L // R) ** 2, -(L // R) ** 2]
    assert np.all(cy == (L // R) ** 2)
