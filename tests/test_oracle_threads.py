"""The oracle's multi-threaded sweeps (used only to time the oracle on all
host cores) equal its sequential sweeps exactly, for every thread count, on
both models, odd strip heights and windows across the periodic seam."""
import numpy as np
import pytest

import physics as ph


@pytest.mark.parametrize("model,T,Delta", [(0, ph.TC, 0.0), (0, 0.5, 0.0), (1, 1.398, 1.0)])
def test_parallel_sweep_equals_sequential(orc, model, T, Delta):
    L, seed = 128, 5 + model
    thr = orc.thresholds(model, 1.0, T, Delta)
    ref = orc.init(model, L, seed)
    for nth in (1, 2, 3, 8, 16):
        a = orc.init(model, L, seed)
        r = ref.copy()
        for t in range(4):
            orc.sweep_par(model, a, seed, thr, t, nth)
            orc.sweep(model, r, seed, thr, t)
            assert np.array_equal(a, r), (nth, t)


@pytest.mark.parametrize("model", [0, 1])
def test_parallel_strip_sweep_equals_sequential(orc, model):
    L, seed, t = 256, 9, 3
    T, Delta = (ph.TC, 0.0) if model == 0 else (1.398, 1.0)
    thr = orc.thresholds(model, 1.0, T, Delta)
    for y0, H in [(0, 7), (250, 16), (100, 1)]:
        base = orc.init_rows(model, L, seed, (y0 - 2) % L, H + 4)
        ref = orc.sweep_strip(model, L, seed, thr, t, y0, base.copy())
        for nth in (1, 4, 7):
            got = orc.sweep_strip_par(model, L, seed, thr, t, y0, base.copy(), nth)
            assert np.array_equal(got, ref), (y0, H, nth)


def test_threads_available(orc):
    assert orc.threads_available() >= 1
