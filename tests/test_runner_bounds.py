"""The runner's tile counters on the CPU: the host bound that lat_runner_run
applies before every launch (csrc/runner_bounds.h), compiled here with the
host compiler and checked against exact integer arithmetic.

A lattice with ntiles tiles per colour phase and nsweeps sweeps counts its
finished tiles up to base + 2 nsweeps ntiles; the bound must accept exactly
the runs in which that stays below 2^64 - 1 (the wait target of a stalled
lattice), and in particular every run that a 32-bit count could not hold.
"""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_18624_gb300", "csrc")
TOP = (1 << 64) - 1


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("bounds") / "runner_bounds_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC,
                           os.path.join(ROOT, "tests", "cpp", "runner_bounds_check.cpp"), "-o", exe])

    def run(cases):
        text = "".join("%d %d %d\n" % c for c in cases)
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split()
        return [o == "1" for o in out]
    return run


def _exact(base, ns, nt):
    return base < TOP and base + 2 * ns * nt < TOP


def test_bound_equals_exact_arithmetic(checker):
    rng = np.random.default_rng(11)
    cases = [(0, 1 << 20, 1 << 23), (0, 4100, 1 << 19), (0, (1 << 32) - 1, (1 << 32) - 1),
             (0, 1 << 31, 1 << 31), (0, 1 << 31, 1 << 32), (0, 1 << 32, 1 << 31), (TOP, 0, 0), (TOP - 1, 0, 5),
             (TOP - 1, 1, 1), (TOP - 2, 1, 1), (TOP - 3, 1, 1), (TOP - 71, 5, 7), (TOP - 70, 5, 7),
             (TOP - 71, 5, 8), (TOP - 71, 6, 7), (0, 0, 1 << 40), (5, 1 << 40, 0)]
    for _ in range(4000):
        kind = rng.integers(0, 3)
        if kind == 0:
            base = int(rng.integers(0, 1 << 62)) * int(rng.integers(1, 4))
            ns, nt = int(rng.integers(0, 1 << 33)), int(rng.integers(0, 1 << 33))
        elif kind == 1:   # near the edge: base + 2 ns nt within a few units of 2^64 - 1
            ns, nt = int(rng.integers(1, 1 << 20)), int(rng.integers(1, 1 << 20))
            base = TOP - 2 * ns * nt + int(rng.integers(-3, 4))
            base = min(max(base, 0), TOP)
        else:
            base = int(rng.integers(0, 1 << 33))
            ns, nt = int(rng.integers(0, 1 << 32)), int(rng.integers(0, 1 << 32))
        cases.append((base, ns, nt))
    got = checker(cases)
    assert len(got) == len(cases)
    bad = [c for c, g in zip(cases, got) if g != _exact(*c)]
    assert not bad, bad[:5]


def test_runs_beyond_32_bit_counts_are_accepted(checker):
    # Ising L = 2^19 with the default 4096-item tiles has 2^19 tiles per phase;
    # a 2^20-sweep run reaches 2^40 finished tiles, far past 2^32.
    assert checker([(0, 1 << 20, 1 << 19), (0, 1 << 20, 1 << 23), ((1 << 32) - 5, 8, 1 << 17)]) == [True] * 3
