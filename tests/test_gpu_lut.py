"""The lookup-table random-bit mode (section 3.2) on the GPU against the
oracle's restatement: bit-exact lattice and (M, B, Q) after every sweep,
full-size windows, the runner, and the +-flip symmetry."""
import numpy as np
import pytest

from paper_2502_18624_gb300 import binding as b

pytestmark = pytest.mark.gpu
TC = b.TC_ISING
LUT = b.LAT_RNG_TABLE


@pytest.mark.parametrize("L", [64, 128, 192, 320, 512])
# T = 1.0 and 0.5 put two to seven steps of the index into single 2^17-wide
# buckets of the kernel's bucket table (the uniforms landing there take the
# four-step search); near Tc every step sits alone in its bucket.
@pytest.mark.parametrize("T", [TC, 0.9 * TC, 5.0, 1.0, 0.5, 0.05, 1e12])
def test_lut_mode_matches_oracle(gpu, orc, L, T):
    seed = 17 * L + 3
    lat = b.Lattice(0, L, T, seed, rng=LUT)
    tbl = orc.lut_table(1.0, T)
    s = orc.init(0, L, seed)
    assert np.array_equal(lat.spins(), s)
    for t in range(6):
        obs = lat.sweep(1)
        orc.sweep_lut(s, seed, tbl, t)
        assert np.array_equal(lat.spins(), s), "sweep %d" % t
        M, B, Q = orc.measure(0, s)
        assert (int(obs["M"][0]), int(obs["B"][0]), int(obs["Q"][0])) == (M, B, Q)
        assert int(obs["draws"][0]) == 2 * 4 * (L * L // 64)  # 4 Philox blocks per word per phase
    lat.close()


def test_lut_mode_full_size_windows(gpu, orc):
    L, seed = 1 << 17, 7
    lat = b.Lattice(0, L, TC, seed, rng=LUT)
    tbl = orc.lut_table(1.0, TC)
    lat.sweep(2, record=False)
    H = 6
    for y0 in (0, L - 3, (1 << 15) + 9):
        pre = lat.rows((y0 - 2) % L, H + 4)
        t = lat.sweep_index
        strip = np.ascontiguousarray(pre)
        orc.sweep_strip_lut(L, seed, tbl, t, y0, strip)
        lat.sweep(1, record=False)
        assert np.array_equal(lat.rows(y0, H), strip[2:H + 2]), y0
    M, B, Q, _ = lat.measure()
    cx, cy = lat.correlation(1)
    assert cx[1] + cy[1] == B and Q == L * L
    lat.close()


def test_lut_mode_in_the_runner_and_flip_symmetry(gpu):
    jobs = [(0, 256, TC, 1), (0, 192, 0.9 * TC, 2), (0, 1024, 1.2 * TC, 3)]
    lats = [b.Lattice(0, L, T, s, rng=LUT) for (_, L, T, s) in jobs]
    refs = [b.Lattice(0, L, T, s, rng=LUT) for (_, L, T, s) in jobs]
    runner = b.Runner(4, 16)
    obs = runner.run(lats, [7, 5, 9])
    for a, r, o, k in zip(lats, refs, obs, [7, 5, 9]):
        assert np.array_equal(o, r.sweep(k)) and a.hash() == r.hash()
    runner.close()
    a = b.Lattice(0, 256, TC, 5, rng=LUT)
    m = b.Lattice(0, 256, TC, 5, rng=LUT)
    m.set_spins(-a.spins())
    a.sweep(10, record=False)
    m.sweep(10, record=False)
    assert np.array_equal(a.spins(), -m.spins())
