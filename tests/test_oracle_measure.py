"""Pin the oracle's observables, correlation, packing and hash.

* (M, B, Q) of random states equal a numpy restatement over rolled arrays
  (independent code path: array rolls instead of index loops).
* C(r) equals the circular autocorrelation computed with numpy's FFT in
  float64 and rounded; C(0) = L^2 (Ising) or Q (Blume-Capel); the sums are
  symmetric under r -> L - r; and the nearest-neighbour bond sum obeys
  B = Cx(1) + Cy(1) exactly (each bond is a distance-1 pair along one axis).
* Canonical packing equals numpy.packbits with little bit order.
"""
import numpy as np
import pytest

import physics as ph


def _random_state(model, L, seed):
    rng = np.random.default_rng(seed)
    vals = np.array([-1, 1] if model == 0 else [-1, 0, 1], dtype=np.int8)
    return vals[rng.integers(0, vals.size, size=(L, L))]


@pytest.mark.parametrize("model,L", [(0, 8), (0, 64), (1, 64), (1, 5), (0, 128)])
def test_measure_matches_array_form(orc, model, L):
    s = _random_state(model, L, L + model)
    M, B, Q = orc.measure(model, s)
    assert M == int(s.astype(np.int64).sum())
    assert Q == int((s.astype(np.int64) ** 2).sum())
    assert B == int(ph.bonds(s.astype(np.int64)))


def _fft_corr(s, axis):
    f = np.fft.fft(s.astype(np.float64), axis=axis)
    ac = np.fft.ifft(f * np.conj(f), axis=axis).real
    return np.rint(ac.sum(axis=1 - axis)).astype(np.int64)


@pytest.mark.parametrize("model,L", [(0, 64), (1, 64), (0, 128), (1, 96), (0, 6)])
def test_correlation_equals_fft(orc, model, L):
    s = _random_state(model, L, 3 * L + model)
    rmax = L - 1
    cx, cy = orc.correlation(s, rmax)
    assert np.array_equal(cx, _fft_corr(s, 1)[: rmax + 1])
    assert np.array_equal(cy, _fft_corr(s, 0)[: rmax + 1])
    M, B, Q = orc.measure(model, s)
    assert cx[0] == cy[0] == (L * L if model == 0 else Q)
    assert np.array_equal(cx[1:], cx[1:][::-1]) and np.array_equal(cy[1:], cy[1:][::-1])
    assert B == cx[1] + cy[1]


def test_correlation_after_dynamics(orc):
    L, seed = 64, 11
    thr = orc.thresholds(0, 1.0, ph.TC)
    s = orc.init(0, L, seed)
    orc.run(0, s, seed, thr, 0, 30, record=False)
    cx, cy = orc.correlation(s, 32)
    assert np.array_equal(cx, _fft_corr(s, 1)[:33]) and np.array_equal(cy, _fft_corr(s, 0)[:33])
    assert orc.measure(0, s)[1] == cx[1] + cy[1]


@pytest.mark.parametrize("model,L", [(0, 64), (0, 192), (1, 64), (1, 128)])
def test_pack_matches_packbits(orc, model, L):
    s = _random_state(model, L, 17 + L)
    w = orc.pack(model, s)
    plane0 = (s == 1) if model == 0 else (s != 0)
    ref = np.packbits(plane0.astype(np.uint8), axis=1, bitorder="little").reshape(-1).view(np.uint64)
    n = L * L // 64
    assert np.array_equal(w[:n], ref)
    if model == 1:
        ref1 = np.packbits((s == -1).astype(np.uint8), axis=1, bitorder="little").reshape(-1).view(np.uint64)
        assert np.array_equal(w[n:], ref1)
    assert orc.lattice_hash(model, s) == orc.hash_words(w)


def test_hash_separates_single_spin_changes(orc):
    s = _random_state(0, 64, 1)
    h0 = orc.lattice_hash(0, s)
    seen = {h0}
    for (y, x) in [(0, 0), (5, 63), (63, 1), (31, 32)]:
        t = s.copy()
        t[y, x] = -t[y, x]
        seen.add(orc.lattice_hash(0, t))
    assert len(seen) == 5


@pytest.mark.parametrize("model,L", [(0, 64), (1, 64)])
def test_init_distribution(orc, model, L):
    # The quench draws each spin uniformly: +-1 with p = 1/2 (Ising) or each of
    # -1, 0, +1 with p = 1/3 (Blume-Capel), independently per site.
    s = orc.init(model, 256, 12345 + model)
    vals = (-1, 1) if model == 0 else (-1, 0, 1)
    counts = np.array([(s == v).sum() for v in vals], dtype=np.float64)
    expect = s.size / len(vals)
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < 20.0 and counts.sum() == s.size
    # Neighbouring spins are uncorrelated at t = 0: C(1) / L^2 is O(1/L).
    cx, cy = orc.correlation(s, 1)
    norm = float(cx[0])
    assert abs(cx[1]) / norm < 0.02 and abs(cy[1]) / norm < 0.02


@pytest.mark.parametrize("model,Delta", [(0, 0.0), (1, 1.0)])
def test_strip_sweep_equals_full_sweep(orc, model, Delta):
    L, seed, t = 64, 21, 7
    thr = orc.thresholds(model, 1.0, 1.5, Delta)
    s = orc.init(model, L, seed)
    orc.run(model, s, seed, thr, 0, t, record=False)
    full = orc.sweep(model, s.copy(), seed, thr, t)
    for y0, H in [(0, 8), (30, 5), (60, 4), (17, 1)]:
        rows = [(y0 - 2 + i) % L for i in range(H + 4)]
        strip = np.ascontiguousarray(s[rows])
        orc.sweep_strip(model, L, seed, thr, t, y0, strip)
        assert np.array_equal(strip[2:H + 2], full[[(y0 + i) % L for i in range(H)]])


@pytest.mark.parametrize("model", [0, 1])
def test_init_rows_equals_full_init(orc, model):
    L, seed = 128, 77
    full = orc.init(model, L, seed)
    for y0, n in [(0, 5), (100, 40), (127, 1)]:
        part = orc.init_rows(model, L, seed, y0, n)
        assert np.array_equal(part, full[[(y0 + i) % L for i in range(n)]])
