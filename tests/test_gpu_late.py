"""Full-size parity late in the headline jobs, and by light cones.

The lattices of the bench workloads (Ising L = 2^17 in both random-number
modes, Blume-Capel L = 2^16) are too large for the oracle to run whole.
Two checks still reach deep into their trajectories:

* light cone: after t sweeps from the quench, a W x W block depends only on
  the quench inside the (W + 4t)^2 window around it (each colour phase reads
  nearest neighbours only), so the oracle recomputes 64 x 64 blocks at
  t = 128 from the quench alone, on windows across the periodic seams and at
  site indices above 2^32;
* late transitions: at sweeps 511 and 999 of the same job, one device sweep
  of strips at the top, at the seam and above row 2^16 equals the oracle's
  strip sweep applied to the device's own state before it.
"""
import numpy as np
import pytest

from paper_2502_18624_gb300 import binding as b

pytestmark = pytest.mark.gpu
TC = b.TC_ISING

MODES = {  # name: (model, L, T, Delta, seed, rng)
    "ising-site": (0, 1 << 17, TC, 0.0, 7, b.LAT_RNG_SITE),
    "ising-lut": (0, 1 << 17, TC, 0.0, 7, b.LAT_RNG_TABLE),
    "bc": (1, 1 << 16, 1.398, 1.0, 99, b.LAT_RNG_SITE),
}


def _block(lat, L, y0, x0, W):
    rows = lat.rows(y0, W)
    return np.ascontiguousarray(rows[:, [(x0 + j) % L for j in range(W)]])


@pytest.mark.parametrize("mode", sorted(MODES))
def test_light_cone_and_late_transitions(gpu, orc, mode):
    model, L, T, Delta, seed, rng = MODES[mode]
    lut = rng == b.LAT_RNG_TABLE
    lat = b.Lattice(model, L, T, seed, Delta=Delta, rng=rng)
    t_cone, W = 128, 64
    lat.sweep(t_cone, record=False)
    blocks = [(L - 20, L - 30), (L // 2 + 11, 5), ((1 << 16) + 3 if model == 0 else L // 3, L // 2 - 17)]
    for (y0, x0) in blocks:
        ref = orc.light_cone(model, L, seed, T, t_cone, y0, x0, W, Delta=Delta, lut=lut)
        assert np.array_equal(_block(lat, L, y0, x0, W), ref), "light cone at (%d, %d), t = %d" % (y0, x0, t_cone)

    H = 6
    thr = orc.thresholds(model, 1.0, T, Delta)
    tbl = orc.lut_table(1.0, T) if lut else None
    windows = [0, L - 3, (1 << 16) + 7 if model == 0 else L // 2 + 5]
    for t_late in (511, 999):
        lat.sweep(t_late - lat.sweep_index, record=False)
        assert lat.sweep_index == t_late
        before = {y0: np.ascontiguousarray(lat.rows((y0 - 2) % L, H + 4)) for y0 in windows}
        obs = lat.sweep(1)
        for y0 in windows:
            strip = before[y0]
            if lut:
                orc.sweep_strip_lut(L, seed, tbl, t_late, y0, strip)
            else:
                orc.sweep_strip(model, L, seed, thr, t_late, y0, strip)
            assert np.array_equal(lat.rows(y0, H), strip[2:H + 2]), "strip at row %d, sweep %d" % (y0, t_late)
        M, B, Q, _ = lat.measure()
        assert (int(obs["M"][0]), int(obs["B"][0]), int(obs["Q"][0])) == (M, B, Q)
        counts = lat.spin_counts()
        assert counts[:3].sum() == L * L and counts[3] == 0
    lat.close()
