"""Pin the oracle's integer acceptance tables.

Each entry is checked three independent ways:
  * dE is recomputed by brute force from the Hamiltonians of Eqs. (1) and (2)
    on a 5-site star (centre + 4 neighbours whose values give the entry's h),
    so a wrong sign, index or dropped term in the table's dE fails;
  * the integer equals floor(2^32 exp(-dE/T)) evaluated with 80 significant
    digits (mpmath), T being the exact binary value of the double;
  * detailed balance: for every move s->s' and its reverse the ratio of
    acceptance probabilities is exp(-dE/T) to within one unit in 2^32.
"""
import itertools

import mpmath
import numpy as np
import pytest

mpmath.mp.dps = 80
TC = 2.0 / np.log(1.0 + np.sqrt(2.0))
ALWAYS = 1 << 32


def _star_energy(model, centre, nbrs, J, Delta):
    # Eq. (1)/(2) restricted to the bonds and sites that a centre move changes.
    e = -J * sum(centre * n for n in nbrs)
    if model == 1:
        e += Delta * centre * centre
    return e


def _nbrs_for_h(model, h):
    # Some neighbour values with sum h (the energy change depends only on h).
    vals = (-1, 1) if model == 0 else (-1, 0, 1)
    for n in itertools.product(vals, repeat=4):
        if sum(n) == h:
            return n
    return None


def _exact_thr(dE, T):
    if dE <= 0:
        return ALWAYS
    v = int(mpmath.floor(mpmath.ldexp(mpmath.exp(-mpmath.mpf(dE) / mpmath.mpf(T)), 32)))
    return min(v, ALWAYS)


ISING_CASES = [(1.0, TC), (1.0, 0.9 * TC), (1.0, 0.8 * TC), (1.0, 1.2 * TC), (1.0, 2.269185),
               (0.5, 1.0), (1.0, 0.05), (1.0, 1e12)]
BC_CASES = [(1.0, 1.0, 1.398), (1.0, 0.5, 1.69), (1.0, 1.5, 1.69), (1.0, 0.0, 1.69),
            (1.0, 1.966, 0.608), (1.0, 1.0, 1.2), (1.0, 1.0, 1.6), (1.0, 1.0, 0.9786),
            (1.0, -1.0, 3.0), (1.0, 1.0, 0.05)]


@pytest.mark.parametrize("J,T", ISING_CASES)
def test_ising_table(orc, J, T):
    thr = orc.thresholds(0, J, T)
    assert thr.shape == (5,)
    for i in range(5):
        k = 2 * i - 4
        for s in (-1, 1):
            if k % s:
                continue
            h = k // s
            nb = _nbrs_for_h(0, h)
            dE = _star_energy(0, -s, nb, J, 0) - _star_energy(0, s, nb, J, 0)
            assert dE == pytest.approx(2 * J * s * h)
            assert int(thr[i]) == _exact_thr(dE, T), (i, s, h)


@pytest.mark.parametrize("J,Delta,T", BC_CASES)
def test_bc_table(orc, J, Delta, T):
    thr = orc.thresholds(1, J, T, Delta)
    assert thr.shape == (54,)
    others = {-1: (0, 1), 0: (-1, 1), 1: (-1, 0)}
    for s in (-1, 0, 1):
        assert others[s][0] < others[s][1] and s not in others[s]
        for b in (0, 1):
            sp = others[s][b]
            for h in range(-4, 5):
                nb = _nbrs_for_h(1, h)
                dE = _star_energy(1, sp, nb, J, Delta) - _star_energy(1, s, nb, J, Delta)
                idx = ((s + 1) * 2 + b) * 9 + (h + 4)
                assert int(thr[idx]) == _exact_thr(dE, T), (s, sp, h)


@pytest.mark.parametrize("J,Delta,T", BC_CASES)
def test_bc_detailed_balance(orc, J, Delta, T):
    thr = orc.thresholds(1, J, T, Delta)
    others = {-1: (0, 1), 0: (-1, 1), 1: (-1, 0)}
    beta = mpmath.mpf(1) / mpmath.mpf(T)
    for s in (-1, 0, 1):
        for b in (0, 1):
            sp = others[s][b]
            bb = others[sp].index(s)          # the reverse proposal, also probability 1/2
            for h in range(-4, 5):
                a = int(thr[((s + 1) * 2 + b) * 9 + h + 4])
                r = int(thr[((sp + 1) * 2 + bb) * 9 + h + 4])
                nb = _nbrs_for_h(1, h)
                dE = _star_energy(1, sp, nb, J, Delta) - _star_energy(1, s, nb, J, Delta)
                # One direction is always accepted (dE <= 0 or its reverse).
                assert a == ALWAYS or r == ALWAYS
                ratio = mpmath.exp(-beta * dE)      # pi(s')/pi(s)
                if a == ALWAYS and r == ALWAYS:
                    assert dE == 0
                elif a == ALWAYS:
                    # pi(s) * 1 = pi(s') * r/2^32  =>  r/2^32 = 1/ratio
                    assert abs(mpmath.mpf(r) / 2**32 - 1 / ratio) <= mpmath.mpf(2) ** -32
                else:
                    assert abs(mpmath.mpf(a) / 2**32 - ratio) <= mpmath.mpf(2) ** -32


def test_ising_detailed_balance_and_limits(orc):
    thr = orc.thresholds(0, 1.0, TC)
    assert all(int(t) == ALWAYS for t in thr[:3])       # s*h <= 0: downhill or flat
    e4, e8 = int(thr[3]) / 2**32, int(thr[4]) / 2**32
    assert e4 == pytest.approx(np.exp(-4 / TC), abs=2**-32)
    assert e8 == pytest.approx(np.exp(-8 / TC), abs=2**-32)
    # T -> 0 forbids every uphill move.  As T -> infinity an uphill entry
    # tends to 2^32 from below: floor(2^32 (1 - dE/T)) = 2^32 - 1, never ALWAYS.
    assert list(orc.thresholds(0, 1.0, 0.01)[3:]) == [0, 0]
    assert list(orc.thresholds(0, 1.0, 1e15)) == [ALWAYS] * 3 + [ALWAYS - 1] * 2
