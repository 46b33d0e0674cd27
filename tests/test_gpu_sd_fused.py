"""The Schwinger-Dyson histogram of Eq. (3) fused into the sweep kernels
(lat_sweep_sd) against the oracle's histogram of the lattice after every
sweep, for both models, both Ising random-number modes and several
acceptance regimes; across the 1024-sweep record batches; and at full size
against the separate histogram kernel."""
import numpy as np
import pytest

from paper_2502_18624_gb300 import binding as b

pytestmark = pytest.mark.gpu
TC = b.TC_ISING

CASES = [  # model, L, T, Delta, rng
    (0, 64, TC, 0.0, b.LAT_RNG_SITE), (0, 192, 0.9 * TC, 0.0, b.LAT_RNG_SITE), (0, 128, 1e-3, 0.0, b.LAT_RNG_SITE),
    (0, 256, 5.0, 0.0, b.LAT_RNG_SITE), (0, 128, TC, 0.0, b.LAT_RNG_TABLE), (0, 320, 1.2 * TC, 0.0, b.LAT_RNG_TABLE),
    (1, 64, 1.398, 1.0, b.LAT_RNG_SITE), (1, 192, 1.69, 0.5, b.LAT_RNG_SITE), (1, 128, 0.5, 1.5, b.LAT_RNG_SITE),
]


@pytest.mark.parametrize("model,L,T,Delta,rng", CASES)
def test_fused_sd_histogram_matches_oracle_every_sweep(gpu, orc, model, L, T, Delta, rng):
    seed = 300 + L + model
    lat = b.Lattice(model, L, T, seed, Delta=Delta, rng=rng)
    s = orc.init(model, L, seed)
    thr = orc.thresholds(model, 1.0, T, Delta)
    tbl = orc.lut_table(1.0, T) if rng == b.LAT_RNG_TABLE else None
    t = 0
    for n in (1, 5, 3):   # calls of different lengths: every call ends with its own colour-0 pass
        obs, sd = lat.sweep_sd(n)
        for i in range(n):
            if tbl is not None:
                orc.sweep_lut(s, seed, tbl, t)
            else:
                orc.sweep(model, s, seed, thr, t)
            t += 1
            assert np.array_equal(sd[i], orc.sd_hist(s)), "sweep %d" % (t - 1)
            M, B, Q = orc.measure(model, s)
            assert (int(obs["M"][i]), int(obs["B"][i]), int(obs["Q"][i])) == (M, B, Q)
        assert sd[-1].sum() == L * L
    assert np.array_equal(lat.spins(), s)
    lat.close()


def test_fused_sd_histogram_across_record_batches(gpu, orc):
    """1030 sweeps in one call: the records come in batches of 1024, each
    closed by its own colour-0 pass."""
    L, seed, T = 64, 77, TC
    lat = b.Lattice(0, L, T, seed)
    s = orc.init(0, L, seed)
    thr = orc.thresholds(0, 1.0, T)
    _, sd = lat.sweep_sd(1030, record=False)
    for t in range(1030):
        orc.sweep(0, s, seed, thr, t)
        if t in (0, 1, 1022, 1023, 1024, 1025, 1029):
            assert np.array_equal(sd[t], orc.sd_hist(s)), t
    lat.close()


@pytest.mark.parametrize("model,L,T,Delta", [(0, 1 << 17, TC, 0.0), (1, 1 << 16, 1.398, 1.0)])
def test_fused_sd_histogram_full_size(gpu, model, L, T, Delta):
    lat = b.Lattice(model, L, T, 9, Delta=Delta)
    for n in (1, 2):
        _, sd = lat.sweep_sd(n, record=False)
        assert np.array_equal(sd[-1], lat.sd_hist())
        assert sd[-1].sum() == L * L
    lat.close()
