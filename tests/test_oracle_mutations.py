"""Show that the oracle's pins have power: plant a plausible mistake in a copy
of oracle.c (compiled on the CPU, never on a GPU), and require that the pin
meant to catch it fails.  Each entry names the mistake, the exact text it
changes and the pin that must detect it.
"""
import contextlib
import ctypes

import numpy as np
import pytest

import physics as ph


@contextlib.contextmanager
def _variant(orc, tmp_path, old, new):
    src = orc.source()
    assert src.count(old) == 1, old
    lib = orc._bind(ctypes.CDLL(orc.compile_variant(src.replace(old, new), str(tmp_path))))
    saved = orc._lib
    orc._lib = lib
    try:
        yield orc
    finally:
        orc._lib = saved


def _ising_enum_fails(orc):
    st = ph.ising_states(4)
    exact, _ = ph.boltzmann_averages(st, 1.0, 0.0, ph.TC, 0)
    thr = orc.thresholds(0, 1.0, ph.TC)
    s = orc.init(0, 4, 5)
    obs = orc.run(0, s, 5, thr, 0, 100_000)[1000:]
    mean, err = ph.binned(-obs[:, 1].astype(np.float64))
    return abs(mean - exact["E"]) > 4 * err


def _bc_enum_fails(orc):
    st = ph.bc_states(3)
    exact, _ = ph.boltzmann_averages(st, 1.0, 1.0, 1.398, 1)
    thr = orc.thresholds(1, 1.0, 1.398, 1.0)
    s = orc.init(1, 3, 5)
    obs = orc.run(1, s, 5, thr, 0, 100_000)[1000:]
    E = -obs[:, 1].astype(np.float64) + obs[:, 2]
    mean, err = ph.binned(E)
    return abs(mean - exact["E"]) > 4 * err


def _philox_fails(orc):
    import test_oracle_philox as tp
    lib = tp._curand()
    ref = tp._host_stream(lib, 1234, 0, 4 * 64).reshape(64, 4)
    ctr = np.stack([np.zeros(64), np.zeros(64), np.arange(64), np.zeros(64)], 1).astype(np.uint32)
    return not np.array_equal(orc.philox(ctr, [1234, 0]), ref)


def _measure_fails(orc):
    s = np.where(np.random.default_rng(1).random((16, 16)) < 0.5, -1, 1).astype(np.int8)
    return orc.measure(0, s)[1] != int(ph.bonds(s.astype(np.int64)))


def _sd_fails(orc):
    st = ph.ising_states(4)
    _, w = ph.boltzmann_averages(st, 1.0, 0.0, ph.TC, 0)
    rhs = np.array([orc.sd_value(orc.sd_hist(np.ascontiguousarray(x)), 1.0, ph.TC) for x in st])
    return abs(float(w @ rhs) - 1.0) > 1e-9


def _corr_fails(orc):
    s = np.where(np.random.default_rng(2).random((32, 32)) < 0.5, -1, 1).astype(np.int8)
    cx, cy = orc.correlation(s, 31)
    f = np.fft.fft(s.astype(np.float64), axis=0)
    ref = np.rint(np.fft.ifft(f * np.conj(f), axis=0).real.sum(axis=1)).astype(np.int64)
    return not np.array_equal(cy, ref)


def _thr_fails(orc):
    import test_oracle_thresholds as tt
    thr = orc.thresholds(0, 1.0, ph.TC)
    return int(thr[3]) != tt._exact_thr(4.0, ph.TC) or int(thr[4]) != tt._exact_thr(8.0, ph.TC)


def _init_fails(orc):
    s = orc.init(1, 256, 9)
    frac = np.array([(s == v).mean() for v in (-1, 0, 1)])
    return np.max(np.abs(frac - 1 / 3)) > 0.01


def _lut_energy_fails(orc):
    import test_oracle_lut as tl
    mean, err = tl._energy(orc, 64, 0.9 * ph.TC, 17, 1500, 300, True)
    return abs(mean - ph.kaufman_u(64, 0.9 * ph.TC)) > 4 * err + 1e-4


def _lut_table_fails(orc):
    import mpmath
    p = mpmath.exp(-4 / mpmath.mpf(ph.TC))
    tbl = orc.lut_table(1.0, ph.TC)
    cum = p**0 * (1 - p) ** 4  # probability of pattern 0
    return abs(int(tbl[1]) - int(mpmath.floor(mpmath.ldexp(cum, 32)))) > 1 or int(tbl[0]) != 0


def _rc_fails(orc):
    import test_oracle_protocol as tp
    return any(orc.protocol_rc(L, t) != tp._exact_rc(L, t) for L in (1 << 17, 1 << 20, 4096) for t in (10**5, 10**7))


def _distances_fails(orc):
    import test_oracle_protocol as tp
    return orc.protocol_distances(1 << 17, 1000, 16).tolist() != tp._exact_distances(1 << 17, 1000, 16)


def _times_fails(orc):
    import test_oracle_protocol as tp
    return orc.protocol_times(1 << 20).tolist() != tp._exact_times(1 << 20)


def _sampled_fails(orc):
    import test_oracle_protocol as tp
    s = np.where(np.random.default_rng(4).random((64, 64)) < 0.5, -1, 1).astype(np.int8)
    rs = [0, 1, 7, 33]
    got = orc.correlation_sampled(s, 16, rs)
    ref = tp._numpy_sampled(s, 16, rs)
    return not (np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]))


def _fails(fn, *a):
    try:
        fn(*a)
    except AssertionError:
        return True
    return False


def _hash_position_fails(orc):
    import test_oracle_hash as th
    return _fails(th.test_exchanging_two_unequal_words_changes_the_hash, orc, 0)


def _hash_avalanche_fails(orc):
    import test_oracle_hash as th
    return _fails(th.test_mixer_avalanche, orc)


def _pack_planes_fail(orc):
    import test_oracle_measure as tm
    return _fails(tm.test_pack_matches_packbits, orc, 1, 64)


def _window_fails(orc):
    import test_oracle_window as tw
    return _fails(tw.test_window_interior_equals_periodic_run, orc, 0, ph.TC, 0.0)


def _window_lut_fails(orc):
    import test_oracle_window as tw
    return _fails(tw.test_lut_window_interior_equals_periodic_run, orc)


def _par_fails(orc):
    import test_oracle_threads as tt
    return _fails(tt.test_parallel_sweep_equals_sequential, orc, 0, ph.TC, 0.0)


def _par_strip_fails(orc):
    import test_oracle_threads as tt
    return _fails(tt.test_parallel_strip_sweep_equals_sequential, orc, 1)


def _strip_fails(orc):
    import test_oracle_measure as tm
    return _fails(tm.test_strip_sweep_equals_full_sweep, orc, 0, 0.0)


def _init_rows_fail(orc):
    import test_oracle_measure as tm
    return _fails(tm.test_init_rows_equals_full_init, orc, 1)


def _corr_x_fails(orc):
    import test_oracle_measure as tm
    return _fails(tm.test_correlation_equals_fft, orc, 0, 64)


def _magnetisation_fails(orc):
    import test_oracle_measure as tm
    return _fails(tm.test_measure_matches_array_form, orc, 1, 5)


MUTATIONS = [
    ("sweep drops the east neighbour",
     "s[y * L + (x + L - 1) % L] + s[y * L + (x + 1) % L];\n                s[site] = or_update_site",
     "s[y * L + (x + L - 1) % L];\n                s[site] = or_update_site", _ising_enum_fails),
    ("Ising table indexed with the wrong sign", "thr[(sv * h + 4) / 2]", "thr[(-sv * h + 4) / 2]",
     _ising_enum_fails),
    ("Blume-Capel crystal-field term with the wrong sign",
     "+ Delta * (double)(sp * sp - s * s)", "- Delta * (double)(sp * sp - s * s)", _bc_enum_fails),
    ("Blume-Capel neighbour sum missing from dE",
     "double dE = -J * (double)(sp - s) * (double)h +", "double dE = 0.0 * (double)h +", _bc_enum_fails),
    ("Philox multipliers swapped", "#define OR_PHILOX_M0 0xD2511F53u", "#define OR_PHILOX_M0 0xCD9E8D57u",
     _philox_fails),
    ("Philox second key word never bumped", "k1 += OR_PHILOX_W1;", "k1 += 0;", _philox_fails),
    ("Philox words 1 and 3 swapped", "c0 = n0; c1 = n1; c2 = n2; c3 = n3;", "c0 = n0; c1 = n3; c2 = n2; c3 = n1;",
     _philox_fails),
    ("bond sum misses vertical bonds", "B += v * s[((y + 1) % L) * L + x];", "", _measure_fails),
    ("Schwinger-Dyson histogram with the wrong sign", "hist[s[y * L + x] * h + 4] += 1;",
     "hist[-s[y * L + x] * h + 4] += 1;", _sd_fails),
    ("correlation shifted by one extra row", "ay += v * s[((y + r) % L) * L + x];",
     "ay += v * s[((y + r + 1) % L) * L + x];", _corr_fails),
    ("threshold rounded up", "double v = floor(ldexp(exp(-dE / T), 32));",
     "double v = ceil(ldexp(exp(-dE / T), 32));", _thr_fails),
    ("lookup-table 4-agree flip uses one word instead of two",
     "                    flip = or_lut_bit(seed, tbl, w, (uint32_t)sweep, colour, 0, k) &\n                           or_lut_bit(seed, tbl, w, (uint32_t)sweep, colour, 1, k);",
     "                    flip = or_lut_bit(seed, tbl, w, (uint32_t)sweep, colour, 0, k);", _lut_energy_fails),
    ("lookup table built from the next pattern's cumulative probability",
     "        double v = floor(ldexp(cum, 32));\n        tbl[j]",
     "        int kk = __builtin_popcount((unsigned)j);\n        double v = floor(ldexp(cum + pow(exp(-4.0 * J / T), kk) * pow(1.0 - exp(-4.0 * J / T), 4 - kk), 32));\n        tbl[j]",
     _lut_table_fails),
    ("Blume-Capel quench not uniform over three values",
     "s[site] = (int8_t)((int)(((uint64_t)w[0] * 3u) >> 32) - 1);",
     "s[site] = (int8_t)((int)(((uint64_t)w[0] * 2u) >> 32) - 1);", _init_fails),
    ("r_c with a base-2 logarithm in g(L)", "sqrt(log((double)L / 65536.0)", "sqrt(log2((double)L / 65536.0)",
     _rc_fails),
    ("log-spaced distances at 16 per octave", "floor(exp2((double)x / 32.0))", "floor(exp2((double)x / 16.0))",
     _distances_fails),
    ("measurement times rounded down", "floor(exp2((double)x / 8.0) + 0.5)", "floor(exp2((double)x / 8.0))",
     _times_fails),
    ("downsampled sources on every column",
     "            for (uint64_t x = 0; x < L; x += R) {\n                int v = s[y * L + x];\n                ax += v * s[y * L + (x + r[i]) % L];",
     "            for (uint64_t x = 0; x < L; x += 1) {\n                int v = s[y * L + x];\n                ax += v * s[y * L + (x + r[i]) % L];",
     _sampled_fails),
    ("hash blind to word positions (i ^ dropped)", "h += or_mix64(i ^ words[i]);", "h += or_mix64(words[i]);",
     _hash_position_fails),
    ("hash mixer missing its second multiply", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;",
     "z = (z ^ (z >> 27));", _hash_avalanche_fails),
    ("Blume-Capel planes swapped in the canonical packing",
     "                if (v != 0) words[i] |= bit;\n                if (v == -1) words[n + i] |= bit;",
     "                if (v != 0) words[n + i] |= bit;\n                if (v == -1) words[i] |= bit;",
     _pack_planes_fail),
    ("window sweep draws with the unwrapped site index",
     "                *c = or_update_site(model, *c, h, y * L + x, sweep, colour, seed, thr);",
     "                *c = or_update_site(model, *c, h, (y0 + i) * L + (x0 + j), sweep, colour, seed, thr);",
     _window_fails),
    ("lookup-table window sweep takes the word index from the window, not the lattice",
     "                uint64_t w = y * (L / 64) + x / 64;\n                int k = (int)((x % 64) / 2);\n                int flip;\n                if (agree == 4)\n                    flip = or_lut_bit(seed, tbl, w, sweep, colour, 0, k) & or_lut_bit(seed, tbl, w, sweep, colour, 1, k);\n                else if (agree == 3)\n                    flip = or_lut_bit(seed, tbl, w, sweep, colour, 0, k);\n                else\n                    flip = 1;\n                if (flip) *c",
     "                uint64_t w = i * (L / 64) + j / 64;\n                int k = (int)((x % 64) / 2);\n                int flip;\n                if (agree == 4)\n                    flip = or_lut_bit(seed, tbl, w, sweep, colour, 0, k) & or_lut_bit(seed, tbl, w, sweep, colour, 1, k);\n                else if (agree == 3)\n                    flip = or_lut_bit(seed, tbl, w, sweep, colour, 0, k);\n                else\n                    flip = 1;\n                if (flip) *c",
     _window_lut_fails),
    ("row-parallel sweep skips the last row", "        for (int64_t y = 0; y < (int64_t)L; ++y)\n            or_phase_rows(",
     "        for (int64_t y = 0; y < (int64_t)L - 1; ++y)\n            or_phase_rows(", _par_fails),
    ("row-parallel strip sweep starts colour 1 one row early", "        int64_t r_lo = colour == 0 ? 1 : 2;",
     "        int64_t r_lo = 1;", _par_strip_fails),
    ("strip sweep draws with the strip row instead of the lattice row",
     "                row[x] = or_update_site(model, row[x], h, y * L + x, sweep, colour, seed, thr);",
     "                row[x] = or_update_site(model, row[x], h, r * L + x, sweep, colour, seed, thr);", _strip_fails),
    ("quench rows start one row late", "uint64_t y = (y0 + r) % L;", "uint64_t y = (y0 + r + 1) % L;",
     _init_rows_fail),
    ("correlation along x shifted by one extra column", "ax += v * s[y * L + (x + r) % L];",
     "ax += v * s[y * L + (x + r + 1) % L];", _corr_x_fails),
    ("magnetisation sums squares", "            M += v;", "            M += v * v;", _magnetisation_fails),
]


@pytest.mark.parametrize("name,old,new,detect", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(orc, tmp_path, name, old, new, detect):
    assert not detect(orc), "the detector must pass on the unmodified oracle"
    with _variant(orc, tmp_path, old, new) as bad:
        assert detect(bad), f"planted mistake not detected: {name}"
