"""Pin the oracle's dynamics to what the physics fixes.

* Exact enumeration: long oracle Metropolis runs on a 4x4 Ising torus
  (2^16 states) and a 3x3 Blume-Capel torus (3^9 states) reproduce the
  Boltzmann averages of Eqs. (1)-(2) within 4 binned standard errors.  A
  dropped neighbour, a wrong sign in dE, a wrong proposal or a wrong table
  index breaks detailed balance or the energy and moves these averages far
  beyond the stated error.
* Onsager's internal energy at 0.9 Tc (ordered start) and Kaufman's exact
  finite-torus energy at Tc; Kaufman itself is pinned to enumeration and to
  u(Tc) = -sqrt(2) as L grows.
* The +-flip symmetry of the Ising dynamics (dE = 2 J s h is flip invariant
  and the random stream does not depend on the spins).
* T -> 0: no uphill move is ever accepted, so E never increases.
* The Schwinger-Dyson identity, Eq. (3), holds exactly under the enumerated
  weights and approximately along equilibrium runs.
"""
import numpy as np
import pytest

import physics as ph

TC = ph.TC


@pytest.fixture(scope="module")
def ising4():
    return ph.ising_states(4)


@pytest.fixture(scope="module")
def bc3():
    return ph.bc_states(3)


def _run_series(orc, model, L, seed, J, T, Delta, nsweeps, burn, s0=None):
    thr = orc.thresholds(model, J, T, Delta)
    s = orc.init(model, L, seed) if s0 is None else s0.copy()
    obs = orc.run(model, s, seed, thr, 0, nsweeps)[burn:]
    M, B, Q = obs[:, 0].astype(np.float64), obs[:, 1].astype(np.float64), obs[:, 2].astype(np.float64)
    E = -J * B + (Delta * Q if model == 1 else 0.0)
    return {"E": E, "M2": M * M, "absM": np.abs(M), "Q": Q}


@pytest.mark.parametrize("T", [1.5, TC, 3.0])
def test_ising_4x4_matches_enumeration(orc, ising4, T):
    exact, _ = ph.boltzmann_averages(ising4, 1.0, 0.0, T, 0)
    series = _run_series(orc, 0, 4, 1000 + int(T * 100), 1.0, T, 0.0, 400_000, 2_000)
    for key in ("E", "M2", "absM"):
        mean, err = ph.binned(series[key])
        assert err < 0.02 * max(1.0, abs(exact[key])), (key, err)
        assert abs(mean - exact[key]) < 4 * err + 1e-9, (key, mean, exact[key], err)


@pytest.mark.parametrize("T,Delta", [(1.398, 1.0), (1.69, 0.5), (0.9, 1.5)])
def test_bc_3x3_matches_enumeration(orc, bc3, T, Delta):
    # L = 3 is odd, so (x+y) parity is not a proper two-colouring of the torus;
    # the oracle's sequential in-place sweep is still a product of single-site
    # Metropolis updates, each of which keeps the Boltzmann weights stationary.
    exact, _ = ph.boltzmann_averages(bc3, 1.0, Delta, T, 1)
    series = _run_series(orc, 1, 3, 77, 1.0, T, Delta, 400_000, 2_000)
    for key in ("E", "Q", "M2"):
        mean, err = ph.binned(series[key])
        assert err < 0.02 * max(1.0, abs(exact[key])), (key, err)
        assert abs(mean - exact[key]) < 4 * err + 1e-9, (key, mean, exact[key], err)


def test_kaufman_formula_is_exact_on_4x4(ising4):
    for T in (1.5, TC, 3.0):
        K = 1.0 / T
        B = ph.bonds(ising4).astype(np.float64)
        lnZ = np.log(np.sum(np.exp(K * B - K * 32))) + K * 32
        assert float(ph.kaufman_lnZ(4, 4, K)) == pytest.approx(lnZ, rel=1e-13)
        exact, _ = ph.boltzmann_averages(ising4, 1.0, 0.0, T, 0)
        assert ph.kaufman_u(4, T) == pytest.approx(exact["E"] / 16, rel=1e-10)


def test_kaufman_tends_to_onsager_at_tc():
    # u(Tc) = -sqrt(2) in the thermodynamic limit (Onsager); finite-L energies approach it.
    us = [ph.kaufman_u(L, TC) for L in (32, 128, 512)]
    gaps = [abs(u + np.sqrt(2.0)) for u in us]
    assert gaps[0] > gaps[1] > gaps[2]
    assert gaps[2] < 2e-3
    assert ph.onsager_u(TC) == pytest.approx(-np.sqrt(2.0), abs=1e-12)


def test_onsager_energy_below_tc(orc):
    T, L = 0.9 * TC, 64
    s0 = np.ones((L, L), dtype=np.int8)
    series = _run_series(orc, 0, L, 31, 1.0, T, 0.0, 3000, 300, s0=s0)
    mean, err = ph.binned(series["E"] / (L * L), 30)
    u = ph.onsager_u(T)
    assert err < 2e-3
    assert abs(mean - u) < 4 * err + 1e-4, (mean, u, err)


def test_kaufman_energy_at_tc(orc):
    L = 32
    s0 = np.ones((L, L), dtype=np.int8)
    series = _run_series(orc, 0, L, 4242, 1.0, TC, 0.0, 40_000, 2_000, s0=s0)
    mean, err = ph.binned(series["E"] / (L * L), 40)
    u = ph.kaufman_u(L, TC)
    assert err < 5e-3
    assert abs(mean - u) < 4 * err, (mean, u, err)


@pytest.mark.parametrize("L,T", [(16, TC), (64, 0.9 * TC), (32, 5.0)])
def test_ising_flip_symmetry(orc, L, T):
    seed = 99
    thr = orc.thresholds(0, 1.0, T)
    a = orc.init(0, L, seed)
    b = (-a).astype(np.int8)
    for t in range(40):
        orc.sweep(0, a, seed, thr, t)
        orc.sweep(0, b, seed, thr, t)
        assert np.array_equal(a, -b)
        ma, mb = orc.measure(0, a), orc.measure(0, b)
        assert ma[0] == -mb[0] and ma[1] == mb[1] and ma[2] == mb[2]
        ca, cb = orc.correlation(a, 8), orc.correlation(b, 8)
        assert np.array_equal(ca[0], cb[0]) and np.array_equal(ca[1], cb[1])


@pytest.mark.parametrize("model,Delta", [(0, 0.0), (1, 1.0), (1, -0.5)])
def test_zero_temperature_energy_never_increases(orc, model, Delta):
    L, seed = 32, 5
    thr = orc.thresholds(model, 1.0, 1e-3, Delta)
    assert all(int(t) in (0, 1 << 32) for t in thr)
    s = orc.init(model, L, seed)
    e_prev = orc.energy(model, orc.measure(model, s), 1.0, Delta)
    for t in range(60):
        orc.sweep(model, s, seed, thr, t)
        e = orc.energy(model, orc.measure(model, s), 1.0, Delta)
        assert e <= e_prev
        e_prev = e


def test_spin_values_stay_valid(orc):
    # The spin count is conserved and every spin keeps a legal value (Table 3's
    # consistency check): L^2 spins, each in {-1, 0, +1} (BC) or {-1, +1} (Ising).
    for model, vals in ((0, {-1, 1}), (1, {-1, 0, 1})):
        s = orc.init(model, 32, 3)
        thr = orc.thresholds(model, 1.0, 1.5, 1.0)
        orc.run(model, s, 3, thr, 0, 20, record=False)
        assert s.size == 32 * 32 and set(np.unique(s)) <= vals


@pytest.mark.parametrize("model,L,T,Delta", [(0, 4, TC, 0.0), (0, 4, 1.5, 0.0), (1, 3, 1.398, 1.0)])
def test_schwinger_dyson_exact_under_enumeration(orc, ising4, bc3, model, L, T, Delta):
    states = ising4 if model == 0 else bc3
    _, w = ph.boltzmann_averages(states, 1.0, Delta, T, model)
    rhs = np.array([orc.sd_value(orc.sd_hist(np.ascontiguousarray(st)), 1.0, T) for st in states])
    assert float(w @ rhs) == pytest.approx(1.0, abs=1e-12)


def test_schwinger_dyson_along_an_equilibrium_run(orc):
    L, T, seed = 32, TC, 8
    thr = orc.thresholds(0, 1.0, T)
    s = np.ones((L, L), dtype=np.int8)
    orc.run(0, s, seed, thr, 0, 500, record=False)
    vals = []
    for t in range(500, 4500):
        orc.sweep(0, s, seed, thr, t)
        vals.append(orc.sd_value(orc.sd_hist(s), 1.0, T))
    mean, err = ph.binned(np.array(vals), 40)
    assert abs(mean - 1.0) < 4 * err + 1e-4, (mean, err)
