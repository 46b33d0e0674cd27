"""Exact results that pin the oracle's dynamics, written from the physics.

Nothing here calls the oracle: these are brute-force enumerations of the
Hamiltonians of Eqs. (1)-(2), Onsager's closed-form internal energy and
Kaufman's exact partition function of a finite torus.
"""
from __future__ import annotations

import mpmath
import numpy as np
from scipy.special import ellipk

TC = 2.0 / np.log(1.0 + np.sqrt(2.0))


def ising_states(L: int) -> np.ndarray:
    """All 2^(L*L) Ising configurations, shape (2^n, L, L), int8."""
    n = L * L
    idx = np.arange(2**n, dtype=np.uint32)
    bits = ((idx[:, None] >> np.arange(n, dtype=np.uint32)) & 1).astype(np.int8)
    return (2 * bits - 1).reshape(-1, L, L)


def bc_states(L: int) -> np.ndarray:
    """All 3^(L*L) Blume-Capel configurations, shape (3^n, L, L), int8."""
    n = L * L
    idx = np.arange(3**n, dtype=np.int64)
    digits = np.empty((idx.size, n), dtype=np.int8)
    rest = idx.copy()
    for i in range(n):
        digits[:, i] = rest % 3
        rest //= 3
    return (digits - 1).reshape(-1, L, L)


def bonds(s: np.ndarray) -> np.ndarray:
    """Sum over nearest-neighbour pairs (each once) of s_x s_y, periodic."""
    return (s * np.roll(s, -1, axis=-1)).sum((-1, -2)) + (s * np.roll(s, -1, axis=-2)).sum((-1, -2))


def boltzmann_averages(states: np.ndarray, J: float, Delta: float, T: float, model: int):
    """Exact <E>, <M^2>, <|M|>, <Q> and the Boltzmann weights."""
    B = bonds(states).astype(np.float64)
    Q = (states.astype(np.int64) ** 2).sum((1, 2)).astype(np.float64)
    M = states.sum((1, 2)).astype(np.float64)
    E = -J * B + (Delta * Q if model == 1 else 0.0)
    w = np.exp(-(E - E.min()) / T)
    w /= w.sum()
    return {"E": float(w @ E), "M2": float(w @ (M * M)), "absM": float(w @ np.abs(M)),
            "Q": float(w @ Q)}, w


def onsager_u(T: float, J: float = 1.0) -> float:
    """Onsager's internal energy per site of the infinite square lattice."""
    K = J / T
    k = 2.0 * np.sinh(2 * K) / np.cosh(2 * K) ** 2
    a = 2 * np.tanh(2 * K) ** 2 - 1
    # At Tc, k = 1 and K(k) diverges only logarithmically while a -> 0: the product's limit is 0.
    term = 0.0 if k * k >= 1.0 else a * ellipk(k * k)
    return float(-J / np.tanh(2 * K) * (1 + (2 / np.pi) * term))


def kaufman_lnZ(m: int, n: int, K):
    """ln Z of the m x n periodic Ising lattice (Kaufman 1949), mpmath precision."""
    K = mpmath.mpf(K)
    c2 = mpmath.cosh(2 * K) / mpmath.tanh(2 * K)
    gam = []
    for l in range(2 * n):
        if l == 0:
            gam.append(2 * K + mpmath.log(mpmath.tanh(K)))
        else:
            gam.append(mpmath.acosh(c2 - mpmath.cos(mpmath.pi * l / n)))
    odd, even = gam[1::2], gam[0::2]
    p1 = mpmath.fprod(2 * mpmath.cosh(m * g / 2) for g in odd)
    p2 = mpmath.fprod(2 * mpmath.sinh(m * g / 2) for g in odd)
    p3 = mpmath.fprod(2 * mpmath.cosh(m * g / 2) for g in even)
    p4 = mpmath.fprod(2 * mpmath.sinh(m * g / 2) for g in even)
    return mpmath.log(mpmath.mpf(1) / 2) + mpmath.mpf(m * n) / 2 * mpmath.log(2 * mpmath.sinh(2 * K)) \
        + mpmath.log(p1 + p2 + p3 + p4)


def kaufman_u(L: int, T: float, J: float = 1.0) -> float:
    """Exact internal energy per site of the L x L periodic Ising lattice."""
    with mpmath.workdps(40):
        K = mpmath.mpf(J) / mpmath.mpf(T)
        d = mpmath.diff(lambda k: kaufman_lnZ(L, L, k), K)
        return float(-J * d / (L * L))


def binned(x: np.ndarray, nbins: int = 64):
    """Mean and standard error of a correlated series by non-overlapping bins."""
    n = (x.size // nbins) * nbins
    b = x[x.size - n:].reshape(nbins, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(nbins))
