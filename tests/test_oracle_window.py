"""Pin the oracle's light-cone windows (or_init_window, or_sweep_window,
or_sweep_window_lut): a window that is not periodic, swept t times, must
hold the periodic lattice's values after t sweeps on its interior (each
colour phase reads only nearest neighbours, section 3.1), for windows that
cross both seams of the torus, both models and the lookup-table stream.
"""
import numpy as np
import pytest

import physics as ph


@pytest.mark.parametrize("model,T,Delta", [(0, ph.TC, 0.0), (0, 1.2, 0.0), (1, 1.398, 1.0), (1, 0.9, 0.5)])
def test_window_interior_equals_periodic_run(orc, model, T, Delta):
    L, seed, t = 128, 31 + model, 6
    thr = orc.thresholds(model, 1.0, T, Delta)
    s = orc.init(model, L, seed)
    full = [s.copy()]
    for k in range(t):
        orc.sweep(model, s, seed, thr, k)
        full.append(s.copy())
    for (y0, x0, H, Wd) in [(0, 0, 40, 40), (120, 3, 44, 30), (50, 110, 30, 52), (127, 127, 26, 26)]:
        win = orc.init_window(model, L, seed, y0, x0, H, Wd)
        rows, cols = [(y0 + i) % L for i in range(H)], [(x0 + j) % L for j in range(Wd)]
        assert np.array_equal(win, full[0][np.ix_(rows, cols)])
        for k in range(t):
            orc.sweep_window(model, L, seed, thr, k, y0, x0, win)
            m = 2 * (k + 1)
            if H - 2 * m <= 0 or Wd - 2 * m <= 0:
                break
            ref = full[k + 1][np.ix_(rows[m:H - m], cols[m:Wd - m])]
            assert np.array_equal(win[m:H - m, m:Wd - m], ref), (y0, x0, k)


def test_lut_window_interior_equals_periodic_run(orc):
    L, seed, t = 128, 41, 5
    tbl = orc.lut_table(1.0, ph.TC)
    s = orc.init(0, L, seed)
    full = [s.copy()]
    for k in range(t):
        orc.sweep_lut(s, seed, tbl, k)
        full.append(s.copy())
    for (y0, x0, H, Wd) in [(100, 90, 40, 60), (5, 126, 36, 36)]:
        win = orc.init_window(0, L, seed, y0, x0, H, Wd)
        rows, cols = [(y0 + i) % L for i in range(H)], [(x0 + j) % L for j in range(Wd)]
        for k in range(t):
            orc.sweep_window_lut(L, seed, tbl, k, y0, x0, win)
            m = 2 * (k + 1)
            ref = full[k + 1][np.ix_(rows[m:H - m], cols[m:Wd - m])]
            assert np.array_equal(win[m:H - m, m:Wd - m], ref), (y0, x0, k)


def test_light_cone_helper(orc):
    L, seed, t, W = 128, 9, 7, 12
    thr = orc.thresholds(0, 1.0, ph.TC)
    s = orc.init(0, L, seed)
    orc.run(0, s, seed, thr, 0, t, record=False)
    for (y0, x0) in [(0, 0), (120, 70), (60, 125)]:
        got = orc.light_cone(0, L, seed, ph.TC, t, y0, x0, W)
        rows, cols = [(y0 + i) % L for i in range(W)], [(x0 + j) % L for j in range(W)]
        assert np.array_equal(got, s[np.ix_(rows, cols)])
