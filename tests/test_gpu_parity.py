"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Everything here is integer work, so the bar is bit-exactness: the lattice
after every sweep, the exact int64 (M, B, Q) per sweep (fused and separate
reductions), the C(r) sums, the Schwinger-Dyson histogram and the canonical
hash.  The only floating point is the host-side normalisation e = E/L^2,
checked at relative tolerance 1e-12.  Lattice sizes span one to many
sweep-kernel chunks per row and ragged word counts (L/64 odd, strips of
the correlation kernel that end mid-tile); temperatures cover every
acceptance mode (draw, always, never).
"""
import numpy as np
import pytest

from paper_2502_18624_gb300 import binding as b

pytestmark = pytest.mark.gpu

TC = b.TC_ISING


def _compare_run(orc, model, L, T, seed, Delta=0.0, nsweeps=8, rmax=None, every=1):
    lat = b.Lattice(model, L, T, seed, Delta=Delta)
    thr = orc.thresholds(model, 1.0, T, Delta)
    assert np.array_equal(lat.thresholds(), thr)
    s = orc.init(model, L, seed)
    assert np.array_equal(lat.spins(), s), "quench differs"
    for t in range(nsweeps):
        obs = lat.sweep(1)
        orc.sweep(model, s, seed, thr, t)
        if t % every == 0 or t == nsweeps - 1:
            g = lat.spins()
            if not np.array_equal(g, s):
                bad = np.argwhere(g != s)
                raise AssertionError("sweep %d: %d sites differ, first %s" % (t, len(bad), bad[:4].tolist()))
        M, B, Q = orc.measure(model, s)
        assert (int(obs["M"][0]), int(obs["B"][0]), int(obs["Q"][0]), int(obs["sweep"][0])) == (M, B, Q, t + 1)
        if rmax is not None:
            cx, cy = lat.correlation(rmax)
            ox, oy = orc.correlation(s, rmax)
            assert np.array_equal(cx, ox) and np.array_equal(cy, oy)
    assert lat.measure()[:3] == orc.measure(model, s)
    lat.close()
    return s


def test_ising_reference_workload_L256(gpu, orc):
    """L=256, T=Tc, seed 1234, 100 sweeps; lattice, E, M and C(r<=128) after every sweep."""
    L, seed, n = 256, 1234, 100
    lat = b.Lattice(0, L, TC, seed)
    thr = orc.thresholds(0, 1.0, TC)
    s = orc.init(0, L, seed)
    assert np.array_equal(lat.spins(), s)
    for t in range(n):
        obs = lat.sweep(1)
        orc.sweep(0, s, seed, thr, t)
        assert np.array_equal(lat.spins(), s), "sweep %d" % t
        M, B, Q = orc.measure(0, s)
        assert (int(obs["M"][0]), int(obs["B"][0])) == (M, B)
        e_gpu = -1.0 * float(obs["B"][0]) / (L * L)
        e_ref = orc.energy(0, (M, B, Q)) / (L * L)
        assert e_gpu == pytest.approx(e_ref, rel=1e-12, abs=0)
        cx, cy = lat.correlation(128)
        ox, oy = orc.correlation(s, 128)
        assert np.array_equal(cx, ox) and np.array_equal(cy, oy), "C(r) at sweep %d" % t
        assert int(cx[1] + cy[1]) == B
    assert lat.hash() == orc.lattice_hash(0, s)
    lat.close()


@pytest.mark.parametrize("L", [64, 128, 192, 320, 512])
@pytest.mark.parametrize("T", [TC, 0.9 * TC, 5.0, 1e-3, 1e15])
def test_ising_sizes_and_modes(gpu, orc, L, T):
    _compare_run(orc, 0, L, T, seed=L * 31 + int(T * 7) % 1000, nsweeps=6)


@pytest.mark.parametrize("L", [64, 128, 192, 256])
@pytest.mark.parametrize("Delta,T", [(1.0, 1.398), (0.5, 1.69), (1.5, 1.69), (-1.0, 3.0), (1.0, 1e-3),
                                     (0.0, 1e15), (1.966, 0.608)])
def test_blume_capel_sizes_and_modes(gpu, orc, L, Delta, T):
    _compare_run(orc, 1, L, T, seed=99 + L, Delta=Delta, nsweeps=6)


def test_multi_sweep_call_records_every_sweep(gpu, orc):
    for model, Delta, T in [(0, 0.0, TC), (1, 1.0, 1.398)]:
        L, seed, n = 192, 5, 37
        lat = b.Lattice(model, L, T, seed, Delta=Delta)
        obs = lat.sweep(n)
        s = orc.init(model, L, seed)
        ref = orc.run(model, s, seed, orc.thresholds(model, 1.0, T, Delta), 0, n)
        assert np.array_equal(np.stack([obs["M"], obs["B"], obs["Q"]], 1), ref)
        assert list(obs["sweep"]) == list(range(1, n + 1))
        assert np.array_equal(lat.spins(), s)
        # without recording, the lattice advances identically
        lat2 = b.Lattice(model, L, T, seed, Delta=Delta)
        assert lat2.sweep(n, record=False) is None
        assert lat2.hash() == lat.hash() == orc.lattice_hash(model, s)
        lat.close(); lat2.close()


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("L,rmax", [(64, 32), (64, 0), (64, 31), (128, 1), (128, 33), (192, 96), (192, 63),
                                    (256, 128), (256, 64), (320, 7), (320, 160), (512, 256), (512, 95),
                                    (1024, 512), (1024, 100)])
def test_correlation_parity(gpu, orc, model, L, rmax):
    T, Delta = (TC, 0.0) if model == 0 else (1.398, 1.0)
    lat = b.Lattice(model, L, T, 11, Delta=Delta)
    lat.sweep(5, record=False)
    s = lat.spins()
    cx, cy = lat.correlation(rmax)
    ox, oy = orc.correlation(s, rmax)
    assert np.array_equal(cx, ox) and np.array_equal(cy, oy)
    M, B, Q = lat.measure()[:3]
    assert cx[0] == cy[0] == (L * L if model == 0 else Q)
    if rmax >= 1:
        assert cx[1] + cy[1] == B
    lat.close()


@pytest.mark.parametrize("model", [0, 1])
def test_sd_histogram_and_hash_parity(gpu, orc, model):
    T, Delta = (TC, 0.0) if model == 0 else (1.398, 1.0)
    for L in (64, 192, 256):
        lat = b.Lattice(model, L, T, 3, Delta=Delta)
        lat.sweep(9, record=False)
        s = lat.spins()
        assert np.array_equal(lat.sd_hist(), orc.sd_hist(s))
        assert lat.hash() == orc.lattice_hash(model, s)
        lat.close()


@pytest.mark.parametrize("model", [0, 1])
def test_set_get_spins_and_invalid_values(gpu, orc, model):
    L = 192
    lat = b.Lattice(model, L, 2.0, 1, Delta=0.5)
    rng = np.random.default_rng(4)
    vals = np.array([-1, 1] if model == 0 else [-1, 0, 1], dtype=np.int8)
    s = vals[rng.integers(0, vals.size, size=(L, L))]
    lat.set_spins(s)
    assert np.array_equal(lat.spins(), s)
    assert np.array_equal(lat.rows(L - 3, 7), s[[(L - 3 + i) % L for i in range(7)]])
    assert lat.measure()[:3] == orc.measure(model, s)
    bad = s.copy()
    bad[5, 7] = 0 if model == 0 else 2
    with pytest.raises(b.LatError) as e:
        lat.set_spins(bad)
    assert e.value.code == b.LAT_EINVAL
    lat.close()


@pytest.mark.parametrize("model", [0, 1])
def test_checkpoint_resume_is_bit_exact(gpu, orc, model):
    L, seed, T, Delta = 256, 42, (TC if model == 0 else 1.398), (0.0 if model == 0 else 1.0)
    a = b.Lattice(model, L, T, seed, Delta=Delta)
    a.sweep(30, record=False)
    ref_hash = a.hash()
    c = b.Lattice(model, L, T, seed, Delta=Delta)
    c.sweep(15, record=False)
    state, t = c.state(), c.sweep_index
    c.close()
    d = b.Lattice(model, L, T, seed, Delta=Delta)
    d.set_state(state)
    d.sweep_index = t
    d.sweep(15, record=False)
    assert d.sweep_index == 30 and d.hash() == ref_hash
    a.close(); d.close()


def test_ising_flip_symmetry_on_gpu(gpu):
    L, seed = 256, 8
    a = b.Lattice(0, L, TC, seed)
    s0 = a.spins()
    m = b.Lattice(0, L, TC, seed)
    m.set_spins(-s0)
    for _ in range(10):
        oa, om = a.sweep(1), m.sweep(1)
        assert np.array_equal(a.spins(), -m.spins())
        assert oa["M"][0] == -om["M"][0] and oa["B"][0] == om["B"][0]
    assert np.array_equal(a.correlation(64)[0], m.correlation(64)[0])
    a.close(); m.close()


def _transition_check(orc, lat, model, L, seed, thr, windows, H=6):
    """One sweep of the device lattice against the oracle's strip sweep on windows."""
    t = lat.sweep_index
    before = {y0: lat.rows((y0 - 2) % L, H + 4) for y0 in windows}
    obs = lat.sweep(1)
    for y0 in windows:
        strip = np.ascontiguousarray(before[y0])
        orc.sweep_strip(model, L, seed, thr, t, y0, strip)
        after = lat.rows(y0, H)
        assert np.array_equal(after, strip[2:H + 2]), "window at row %d, sweep %d" % (y0, t)
    return obs


@pytest.mark.parametrize("model,L,T,Delta", [(0, 1 << 17, TC, 0.0), (0, 1 << 17, 0.9 * TC, 0.0),
                                             (1, 1 << 16, 1.398, 1.0)])
def test_large_lattice_windows(gpu, orc, model, L, T, Delta):
    """Full-size lattices: quench rows, one-sweep transitions on windows that
    include the periodic seam and sites above 2^32, and whole-lattice
    invariants (fused = separate reduction, B = Cx(1) + Cy(1), C(0))."""
    seed = 7 if model == 0 else 99
    lat = b.Lattice(model, L, T, seed, Delta=Delta)
    thr = orc.thresholds(model, 1.0, T, Delta)
    for y0 in (0, L // 2 + 5, L - 2):
        assert np.array_equal(lat.rows(y0, 4), orc.init_rows(model, L, seed, y0, 4))
    lat.sweep(2, record=False)
    windows = [0, 12345, L - 3, (1 << 15) + 1 if model == 0 else L // 2]
    obs = _transition_check(orc, lat, model, L, seed, thr, windows)
    M, B, Q, _ = lat.measure()
    assert (int(obs["M"][0]), int(obs["B"][0]), int(obs["Q"][0])) == (M, B, Q)
    cx, cy = lat.correlation(2)
    assert cx[0] == cy[0] == (L * L if model == 0 else Q)
    assert cx[1] + cy[1] == B
    if model == 0:
        assert (M - L * L) % 2 == 0
    lat.close()


def test_capacity_point_L2p19(gpu, orc):
    """L = 2^19 Ising (2^38 spins, 32 GiB packed): quench rows and a one-sweep
    transition on windows at the top, the seam and site indices near 2^38."""
    L, seed = 1 << 19, 7
    lat = b.Lattice(0, L, TC, seed)
    thr = orc.thresholds(0, 1.0, TC)
    assert np.array_equal(lat.rows(L - 1, 2), orc.init_rows(0, L, seed, L - 1, 2))
    obs = _transition_check(orc, lat, 0, L, seed, thr, [0, L - 4, 300000], H=4)
    M, B, Q, _ = lat.measure()
    assert (int(obs["M"][0]), int(obs["B"][0]), Q) == (M, B, L * L)
    lat.close()


@pytest.mark.parametrize("model", [0, 1])
def test_spin_counts_and_invalid_codes(gpu, orc, model):
    """The spin-count consistency check: per-value counts against the
    oracle's lattice, their sum L^2, and (Blume-Capel) a 2-bit code that is
    not a spin, planted in the raw state, is counted and nothing else moves."""
    T, Delta = (TC, 0.0) if model == 0 else (1.398, 1.0)
    L = 192
    lat = b.Lattice(model, L, T, 21, Delta=Delta)
    lat.sweep(7, record=False)
    s = lat.spins()
    counts = lat.spin_counts()
    assert counts.tolist() == [int((s == -1).sum()), int((s == 0).sum()), int((s == 1).sum()), 0]
    M, B, Q, _ = lat.measure()
    assert counts[:3].sum() == L * L and M == counts[2] - counts[0] and Q == counts[0] + counts[2]
    if model == 1:
        st = lat.state().view(np.uint64).copy()
        n0, g0 = int(st[0]), int(st[1])          # word pair (row 0, word 0): n plane, g plane
        zero_bit = next(i for i in range(64) if not (n0 >> i) & 1)
        st[1] = np.uint64(g0 | (1 << zero_bit))  # g without n at a zero site
        lat.set_state(st.view(np.uint8))
        bad = lat.spin_counts()
        assert bad[3] == 1 and bad[1] == counts[1] - 1 and bad[0] == counts[0] and bad[2] == counts[2]
    lat.close()


@pytest.mark.parametrize("model,L", [(0, 1 << 17), (1, 1 << 16)])
def test_spin_counts_full_size(gpu, model, L):
    T, Delta = (TC, 0.0) if model == 0 else (1.398, 1.0)
    lat = b.Lattice(model, L, T, 5, Delta=Delta)
    obs = lat.sweep(2)
    counts = lat.spin_counts()
    assert counts[:3].sum() == L * L and counts[3] == 0
    assert int(obs["M"][-1]) == counts[2] - counts[0] and int(obs["Q"][-1]) == counts[0] + counts[2]
    lat.close()


@pytest.mark.parametrize("model,L", [(0, 1 << 20), (1, 1 << 19)])
def test_maximum_sizes(gpu, orc, model, L):
    """The largest lattices the library accepts: Ising L = 2^20 (2^40 spins,
    128 GiB packed) and Blume-Capel L = 2^19 (2^38 spins, 64 GiB).  Quench
    rows at both ends, one-sweep transitions on windows at the top, the
    periodic seam and the last rows (site indices near L^2), and whole-lattice
    invariants."""
    T, Delta = (TC, 0.0) if model == 0 else (1.398, 1.0)
    seed = 13
    lat = b.Lattice(model, L, T, seed, Delta=Delta)
    thr = orc.thresholds(model, 1.0, T, Delta)
    for y0 in (0, L - 2):
        assert np.array_equal(lat.rows(y0, 2), orc.init_rows(model, L, seed, y0, 2))
    obs = _transition_check(orc, lat, model, L, seed, thr, [0, L - 4, L // 3], H=4)
    M, B, Q, _ = lat.measure()
    assert (int(obs["M"][0]), int(obs["B"][0]), int(obs["Q"][0])) == (M, B, Q)
    counts = lat.spin_counts()
    assert counts[:3].sum() == L * L and counts[3] == 0 and M == counts[2] - counts[0]
    cx, cy = lat.correlation(1)
    assert cx[1] + cy[1] == B
    lat.close()
    import torch
    torch.cuda.empty_cache()  # return the 64-128 GiB to the device for the tests that follow


@pytest.mark.parametrize("model", [0, 1])
def test_empty_calls_change_nothing(gpu, model):
    T, Delta = (TC, 0.0) if model == 0 else (1.398, 1.0)
    lat = b.Lattice(model, 128, T, 3, Delta=Delta)
    lat.sweep(3, record=False)
    h0, t0 = lat.hash(), lat.sweep_index
    assert lat.sweep(0).size == 0 and lat.sweep(0, record=False) is None
    cx, cy = lat.correlation(0)
    assert cx[0] == cy[0] == lat.spin_counts()[[0, 2]].sum()
    assert lat.correlation_sampled(16, [])[0].size == 0
    r = b.Runner(2, 4)
    assert r.run([lat], [0]) is not None
    r.close()
    assert lat.hash() == h0 and lat.sweep_index == t0
    lat.close()


def _phase_rule(s, colour, flip_if_agree_at_most):
    """One colour phase of a deterministic Ising rule, in numpy."""
    L = s.shape[0]
    y, x = np.indices((L, L))
    agree = sum((np.roll(s, d, axis=a) == s).astype(int) for a in (0, 1) for d in (1, -1))
    act = ((x + y) % 2 == colour) & (agree <= flip_if_agree_at_most)
    return np.where(act, -s, s).astype(np.int8)


@pytest.mark.parametrize("L", [64, 192])
def test_ising_zero_and_infinite_temperature_rules(gpu, L):
    """Textbook limits of the Metropolis rule, independent of the oracle:
    at T -> 0 a site flips iff at most two of its four neighbours agree with
    it (dE = 2Js*h <= 0), which exercises every one of the 16 neighbour
    patterns of the kernel's classification; at T -> infinity every site
    flips, so one sweep negates the lattice."""
    cold = b.Lattice(0, L, 1e-6, 5)
    s = cold.spins()
    for _ in range(3):
        s = _phase_rule(_phase_rule(s, 0, 2), 1, 2)
        obs = cold.sweep(1)
        assert np.array_equal(cold.spins(), s)
        assert int(obs["draws"][0]) == 0  # thresholds 0: no site draws
    cold.close()
    hot = b.Lattice(0, L, 1e15, 6)
    s = hot.spins()
    obs = hot.sweep(1)
    # at T = 1e15 the bound is 2^32 - 1, not 2^32: uphill sites still draw, and this seed's draws all accept
    assert np.array_equal(hot.spins(), -s) and int(obs["draws"][0]) > 0
    hot.close()
