"""Seeded synthetic workloads: lists of simulation jobs (model, size,
temperature, seed, sweeps).  Nothing here touches the method's arithmetic;
both the tests and bench.py draw their inputs from these generators.

- batched_replicas(): 512 independent replicas of uneven sizes
  L in {64, ..., 4096} with weights proportional to 1/L; 384 Ising with T
  uniform in [0.8 Tc, 1.2 Tc], 128 Blume-Capel with Delta = 1 and T uniform
  in [1.2, 1.6]; replica seed = 2025 + replica id; 500 sweeps each.
- served_jobs(): a Poisson stream of jobs (mean rate 200 jobs/s), Ising with
  p = 0.7 or Blume-Capel with Delta in {0.5, 1.0, 1.5}; L = 2^k, k uniform in
  8..14; T uniform in [0.7, 1.3] x the model's reference Tc (2.269185 for
  Ising; 1.398 for Delta = 1.0, 1.69 for Delta = 0.5 and 1.5); sweeps
  log-uniform in [10, 10000]; job seed = base + job id.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

TC_ISING = 2.0 / math.log(1.0 + math.sqrt(2.0))
SERVED_TC = {("ising", 0.0): 2.269185, ("bc", 0.5): 1.69, ("bc", 1.0): 1.398, ("bc", 1.5): 1.69}


@dataclass(frozen=True)
class Job:
    id: int
    model: int        # 0 Ising, 1 Blume-Capel
    L: int
    T: float
    Delta: float
    seed: int
    sweeps: int
    arrival: float = 0.0  # seconds after the stream starts (served jobs)


def batched_replicas(n: int = 512, n_ising: int = 384, sweeps: int = 500, seed: int = 2025,
                     sizes=(64, 128, 256, 512, 1024, 2048, 4096)) -> list[Job]:
    rng = np.random.default_rng(seed)
    w = np.array([1.0 / L for L in sizes])
    w /= w.sum()
    Ls = rng.choice(np.array(sizes), size=n, p=w)
    jobs = []
    for i in range(n):
        if i < n_ising:
            T = float(rng.uniform(0.8 * TC_ISING, 1.2 * TC_ISING))
            jobs.append(Job(i, 0, int(Ls[i]), T, 0.0, seed + i, sweeps))
        else:
            T = float(rng.uniform(1.2, 1.6))
            jobs.append(Job(i, 1, int(Ls[i]), T, 1.0, seed + i, sweeps))
    return jobs


def served_jobs(n: int = 10000, rate: float = 200.0, seed: int = 20250, kmin: int = 8, kmax: int = 14,
                smin: int = 10, smax: int = 10000) -> list[Job]:
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        if rng.random() < 0.7:
            model, Delta, tc = 0, 0.0, SERVED_TC[("ising", 0.0)]
        else:
            Delta = float(rng.choice([0.5, 1.0, 1.5]))
            model, tc = 1, SERVED_TC[("bc", Delta)]
        L = 2 ** int(rng.integers(kmin, kmax + 1))
        T = float(rng.uniform(0.7, 1.3)) * tc
        sw = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        jobs.append(Job(i, model, L, T, Delta, seed + i, sw, t))
    return jobs


def footprint_bytes(job: Job) -> int:
    """Packed lattice bytes of a job (the device workspace adds a few MiB)."""
    return job.L * job.L // (8 if job.model == 0 else 4)
