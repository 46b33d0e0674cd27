#!/usr/bin/env python
"""Throughput of the checkerboard Metropolis hot path on GB300.

Workload (default): Ising, L = 2^17 (1.7e10 spins, 2 GiB packed), J = 1,
T = Tc = 2/ln(1+sqrt 2), quench from seed 7, K sweeps (default 1000) with the
exact (M, B, Q) after every sweep and C(r <= 1024) along both axes after
sweeps 2^k.  A step is one sweep (two colour phases with the fused E/M
reduction) plus its share of the correlation measurements.  The metric is
attempted spin updates per nanosecond ("flips/ns", L^2 per sweep) over the
whole job; the lattice is far larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                  [--workload ising-tc|ising-0.9tc|ising-capacity|bc]

N > 1 (torchrun, one process per GPU) runs independent replicas (seed + rank):
the path has no exchange step, so there is no collective beyond the timing
barrier and the max-over-ranks reduction.  --impl reference times the CPU
oracle on the host (every core) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spin flips/ns on 1 GB300 (Ising L=2^17) + % of roofline; batched vs plain flips/ns"
UNIT = "flips/ns"
TC = 2.0 / math.log(1.0 + math.sqrt(2.0))
# The sweep is bound by integer multiplies (Philox4x32-10).  The integer
# multiply-add pipe of an SM retires 64 32-bit IMAD lane-ops per clock (16
# lanes on each of the 4 schedulers' FMA-heavy pipe), so the peak is
# 152 SMs x 64 x 2070 MHz = 20.1 T IMAD-ops/s.
SMS, IMAD_LANES_PER_SM, SM_MAX_MHZ = 152, 64, 2070.0
ALU_PEAK_TOPS = SMS * IMAD_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
# Algorithmic multiply work of one Philox4x32-10 block by its definition:
# 10 rounds x 2 widening 32x32->64 multiplies, each two 32-bit IMAD-ops
# (high and low halves).
OPS_PER_DRAW = 40

WORKLOADS = {
    "ising-tc": dict(model=0, L=1 << 17, T=TC, Delta=0.0, seed=7, rmax=1024,
                     name="ising-2d L=131072 T=Tc seed=7: K sweeps, E/M every sweep, C(r<=1024) x/y at sweeps 2^k"),
    "ising-0.9tc": dict(model=0, L=1 << 17, T=0.9 * TC, Delta=0.0, seed=7, rmax=1024,
                        name="ising-2d L=131072 T=0.9Tc seed=7: K sweeps, E/M every sweep, C(r<=1024) at sweeps 2^k"),
    "ising-capacity": dict(model=0, L=1 << 19, T=TC, Delta=0.0, seed=7, rmax=1024,
                           name="ising-2d L=524288 (2^38 spins, 32 GiB) T=Tc seed=7: K sweeps, E/M every sweep, "
                                "C(r<=1024) x/y at sweeps 2^k"),
    "ising-lut": dict(model=0, L=1 << 17, T=TC, Delta=0.0, seed=7, rmax=1024, rng=1,
                      name="ising-2d L=131072 T=Tc seed=7, the paper's lookup-table random bits: K sweeps, E/M every "
                           "sweep, C(r<=1024) x/y at sweeps 2^k"),
    "ising-protocol": dict(model=0, L=1 << 17, T=TC, Delta=0.0, seed=7, rmax=32, protocol=16,
                           name="ising-2d L=131072 T=Tc seed=7: K sweeps, E/M every sweep, C(r) by the section 3.3 "
                                "protocol (all sites r<=32, one source per 16x16 square beyond, r_c(t), log-spaced r) "
                                "at t=floor(2^(x/8)+0.5)"),
    "bc": dict(model=1, L=1 << 16, T=1.398, Delta=1.0, seed=99, rmax=512,
               name="blume-capel L=65536 Delta=1 T=1.398 seed=99: K sweeps, E/M/Q every sweep, C(r<=512) at sweeps 2^k"),
}


# ---------------------------------------------------------------- distributed
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def reduce_max(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job(updates_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job flips/ns: all ranks' updates over the slowest rank's time."""
    return updates_per_rank * world / (max_seconds * 1e9)


# ------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.rows: list[list[str]] = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self

        def reader():
            for line in self.proc.stdout:
                self.rows.append([x.strip() for x in line.split(",")])

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        return self

    def stop(self) -> dict:
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def gpu_id_for(device_index: int) -> str:
    import torch
    try:
        u = torch.cuda.get_device_properties(device_index).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            return vis.split(",")[device_index]
        return str(device_index)


# ------------------------------------------------------------ native arm
def powers_of_two_upto(k: int):
    out, p = set(), 1
    while p <= k:
        out.add(p)
        p *= 2
    return out


def run_job(lat, K: int, wl, stream, with_corr: bool = True):
    """K sweeps with per-sweep E/M and C(r) at the workload's measurement times.

    Measurement times are the sweeps 2^k (C(r <= rmax) from every site), or,
    for the protocol workload, t = floor(2^(x/8) + 0.5) with the section 3.3
    protocol.  Returns (sweep_ms_total, n_sweep_launches, total_draws,
    n_corr_points, obs_count, corr_rows, corr_seconds, n_corr_launches).  CUDA events bracket
    every lat_sweep and every correlation call on the lattice's stream, so the
    kernel times are measured on the stream the kernels run on (each call
    returns host data, so its interval is its kernels plus one small copy)."""
    import numpy as np
    import torch

    from paper_2502_18624_gb300 import binding as b
    R = wl.get("protocol", 0)
    if not with_corr:
        meas = set()
    elif R:
        meas = set(int(t) for t in b.lat_protocol_times(K))
    else:
        meas = powers_of_two_upto(K)
    done, sweep_ms, draws, nlaunch_corr, nobs, rows, corr_s, npts = 0, 0.0, 0, 0, 0, 0, 0.0, 0
    while done < K:
        nxt = min([m for m in meas if m > done], default=K)
        n = min(nxt, K) - done
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        obs = lat.sweep(n)
        e1.record(stream)
        e1.synchronize()
        sweep_ms += e0.elapsed_time(e1)
        draws += int(obs["draws"].sum())
        nobs += len(obs)
        done += n
        if done in meas:
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            if R:
                out = lat.correlation_protocol(done, R)
                nds = int(np.sum(out["r"] > 2 * R))
                rows += len(out["r"])
                # near kernel, source-column copy, x and y launches per 2048 distances
                nlaunch_corr += 1 + (1 if R >= 16 and nds else 0) + 2 * ((nds + 2047) // 2048)
            else:
                lat.correlation(wl["rmax"])
                rows += wl["rmax"] + 1
                nlaunch_corr += 1 if wl["rmax"] <= 32 else 2
            c1.record(stream)
            c1.synchronize()
            corr_s += c0.elapsed_time(c1) / 1e3
            npts += 1
    return sweep_ms, 2 * K, draws, npts, nobs, rows, corr_s, nlaunch_corr


def native(args, wl):
    import torch

    from paper_2502_18624_gb300 import binding as b

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = dist_init(world, "nccl")
    b.load()
    stream = torch.cuda.current_stream(device)
    seed = wl["seed"] + rank
    K, W = args.steps, args.warmup
    mk = lambda: b.Lattice(wl["model"], wl["L"], wl["T"], seed, Delta=wl["Delta"], stream=stream, device=device,
                           rng=wl.get("rng", 0))

    # warm-up sweeps (kernels, module load, clocks), then a fresh quench for the timed job
    lat = mk()
    lat.sweep(W)
    lat.close()
    lat = mk()
    torch.cuda.synchronize(device)
    barrier(dist, device)
    sampler = ClockSampler(gpu_id_for(local)).start()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    t_start.record(stream)
    sweep_ms, nlaunch, draws, ncorr, _, _, corr_s, corr_launches = run_job(lat, K, wl, stream)
    t_end.record(stream)
    torch.cuda.synchronize(device)
    clocks = sampler.stop()
    barrier(dist, device)
    secs = t_start.elapsed_time(t_end) / 1e3
    max_secs = reduce_max(dist, secs, device)
    L2 = float(wl["L"]) ** 2
    value = whole_job(L2 * K, world, max_secs)
    thresholds = [int(x) for x in lat.thresholds()]
    counts = lat.spin_counts()  # consistency check: every site holds a spin, L^2 in total
    assert counts[3] == 0 and int(counts[:3].sum()) == wl["L"] ** 2, "spin counts inconsistent: %s" % counts
    final_hash = lat.hash()
    lat.close()

    # end to end through the C ABI with host buffers: upload a quench from pinned
    # memory, run the same job, download the final lattice.
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(b, mk, stream, device, dist, wl, K, world, final_hash)
    line_e2e = e2e
    batched = None if args.no_batched else batched_leg(b, stream, device, dist, world)

    # measured issue rates of the integer pipes (the roofline denominators)
    psampler = ClockSampler(gpu_id_for(local)).start()
    rates = b.lat_probe_rates()
    rates["clocks"] = psampler.stop()

    # roofline of the dominant kernel (the colour-phase sweep kernel)
    launch_s = (sweep_ms / 1e3) / nlaunch
    draws_per_launch = draws / nlaunch
    achieved = OPS_PER_DRAW * draws_per_launch / launch_s / 1e12
    # peak: the measured rate of full Philox4x32-10 blocks (ten rounds, the
    # algorithmic unit of the sweep) at 40 IMAD-ops each
    imad_peak = OPS_PER_DRAW * rates["philox_blocks_per_s"] / 1e12
    traffic, inst = None, None
    prof = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if os.path.exists(prof) and not args.L:
        try:
            with open(prof) as f:
                # the protocol workload runs the same sweep launches as ising-tc
                tr = json.load(f).get({"ising-protocol": "ising-tc"}.get(args.workload, args.workload), {})
            if tr.get("kernel_rev") == kernel_rev():
                traffic = tr.get("bytes_per_launch")
                inst = tr.get("warp_inst_per_launch")
        except Exception:
            traffic, inst = None, None
    roofline = {"bound": "alu", "achieved": achieved, "peak": imad_peak, "unit": "T IMAD-ops/s",
                "frac": achieved / imad_peak, "traffic": traffic,
                "kernel": ("k_ising_phase_lut" if wl.get("rng") else "k_ising_phase") if wl["model"] == 0
                          else "k_bc_phase",
                "launch_ms": launch_s * 1e3, "draws_per_launch": draws_per_launch,
                "ops_per_draw": OPS_PER_DRAW,
                "peak_note": "measured on this GPU after the timed job (lat_probe_rates): full Philox4x32-10 "
                             "blocks per second from a register-only microkernel, x 40 IMAD-ops (10 rounds x 2 "
                             "widening multiplies x 2 halves); achieved counts 40 IMAD-ops per needed block",
                "peak_mad_wide": rates["imad_ops_per_s"] / 1e12, "frac_of_mad_wide": achieved * 1e12 /
                rates["imad_ops_per_s"],
                "peak_derived": ALU_PEAK_TOPS, "frac_of_derived": achieved / ALU_PEAK_TOPS,
                "probe": rates,
                "hbm_frac_of_measured": (L2 / (4.0 if wl["model"] == 0 else 2.0)) / launch_s / 1e9 /
                measured_hbm_gbs()}
    if inst:
        # issue slots: 4 schedulers per SM, one warp instruction each per clock
        issue_peak = SMS * 4 * (rates["clocks"].get("sm_mhz") or SM_MAX_MHZ) * 1e6
        roofline["issue_frac"] = inst / launch_s / issue_peak
        roofline["warp_inst_per_launch"] = inst
    if ncorr and not wl.get("protocol"):
        roofline["corr"] = corr_roofline(wl, ncorr, corr_s, rates)
    wl = dict(wl, corr_launches=corr_launches, corr_share=corr_s / max_secs, thresholds=thresholds)
    return finish(args, wl, rank, world, K, W, value, max_secs, ncorr, nlaunch, roofline, line_e2e, clocks, dist,
                  batched)


def corr_roofline(wl, npts: int, corr_s: float, rates: dict) -> dict:
    """Roofline of C(r <= rmax) from every site (k_corr_x + k_corr_y).

    Algorithmic work per measurement: 2 (rmax + 1) L^2 / 32 pairs of 32-bit
    words (both axes, every distance; one XOR and one population count per
    pair by the definition, Ising).  The kernels pair two word pairs per
    population count (a carry-save step: sum bit and carry of two XOR words
    and the running sum, two 3-input logic operations), so per pair they need
    2 LOP3 on the ALU pipe and 1/2 POPC: the bound is the slower of
    LOP3 rate / 2 and POPC rate / (1/2), with both rates measured."""
    L, rmax = wl["L"], wl["rmax"]
    per = (2 if wl["model"] == 0 else 4) * (rmax + 1) * float(L) * L / 32   # Blume-Capel: two planes
    achieved = per * npts / corr_s / 1e12
    lop3, popc = rates["lop3_per_s"] / 1e12, rates["popc_per_s"] / 1e12
    peak = min(lop3 / 2.0, popc / 0.5)
    return {"bound": "alu", "kernel": "k_corr_x + k_corr_y", "achieved": achieved, "peak": peak,
            "unit": "T word-pairs/s", "frac": achieved / peak, "frac_of_popc_one_per_pair": achieved / popc,
            "pairs_per_measurement": per, "measurements": npts, "ms_per_measurement": corr_s * 1e3 / npts,
            "peak_note": "carry-save pairing: 2 LOP3 + 1/2 POPC per 32-bit word pair; min(LOP3 rate/2, POPC "
                         "rate x 2) from lat_probe_rates (measured on this GPU)"}


def batched_leg(b, stream, device, dist, world):
    """The 512-replica mixed workload: one runner launch against the plain path.

    Both legs start from the replicas' quenches and run 500 sweeps with the
    exact (M, B, Q) after every sweep; the plain leg runs lat_sweep on one
    replica after another.  Every replica must end bit-identical in both."""
    import torch

    from paper_2502_18624_gb300 import autotune, workloads
    jobs = workloads.batched_replicas()
    sweeps = jobs[0].sweeps
    sched = autotune.tune(jobs, use_cache=False)
    mk = lambda: [b.Lattice(j.model, j.L, j.T, j.seed, Delta=j.Delta, stream=stream, device=device) for j in jobs]
    updates = float(sum(j.L * j.L for j in jobs)) * sweeps

    runner = b.Runner(len(jobs), sweeps, stream=stream, device=device)
    autotune.apply(runner, sched)
    lats = mk()
    torch.cuda.synchronize(device)
    barrier(dist, device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    runner.run(lats, [sweeps] * len(jobs))
    e1.record(stream)
    e1.synchronize()
    t_batched = reduce_max(dist, e0.elapsed_time(e1) / 1e3, device)
    hb = [lt.hash() for lt in lats]
    for lt in lats:
        lt.close()
    runner.close()

    lats = mk()
    torch.cuda.synchronize(device)
    barrier(dist, device)
    e0.record(stream)
    for lt in lats:
        lt.sweep(sweeps)
    e1.record(stream)
    e1.synchronize()
    t_plain = reduce_max(dist, e0.elapsed_time(e1) / 1e3, device)
    hp = [lt.hash() for lt in lats]
    for lt in lats:
        lt.close()
    assert hb == hp, "batched run differs from the plain path"
    return {"value": whole_job(updates, world, t_batched), "plain": whole_job(updates, world, t_plain),
            "unit": UNIT, "speedup": t_plain / t_batched, "replicas": len(jobs), "sweeps": sweeps,
            "spins": int(sum(j.L * j.L for j in jobs)), "bit_exact": True,
            "tiles": {"%s L=%d" % ("ising" if m == 0 else "bc", L): t for (m, L), t in sorted(sched.items())},
            "workload": "512 replicas, L in {64..4096} with weights 1/L, 384 Ising T~U[0.8,1.2]Tc, "
                        "128 Blume-Capel Delta=1 T~U[1.2,1.6], seeds 2025+id, 500 sweeps, E/M every sweep"}


def end_to_end(b, mk, stream, device, dist, wl, K, world, final_hash):
    import torch
    lat = mk()
    nbytes = b.lat_state_bytes(lat.params)
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    host_np = host.numpy()
    b.lat_get_state(lat.handle, nbytes, host_np)
    lat.sweep_index = 0
    torch.cuda.synchronize(device)
    barrier(dist, device)
    t0 = time.perf_counter()
    b.lat_set_state(lat.handle, host_np)
    t1 = time.perf_counter()
    sweep_ms, _, _, _, nobs, corr_rows, corr_s, _ = run_job(lat, K, wl, stream)
    t2 = time.perf_counter()
    b.lat_get_state(lat.handle, nbytes, host_np)
    torch.cuda.synchronize(device)
    t3 = time.perf_counter()
    e2e_secs = reduce_max(dist, t3 - t0, device)
    assert lat.hash() == final_hash, "end-to-end run diverged from the device-resident run"
    lat.close()
    d2h = nbytes + nobs * 40 + corr_rows * (2 * 8 + (4 + 8 if wl.get("protocol") else 0))
    L2 = float(wl["L"]) ** 2
    return {"value": whole_job(L2 * K, world, e2e_secs), "unit": UNIT,
            "h2d_bytes_per_step": nbytes / K, "d2h_bytes_per_step": d2h / K,
            "seconds": {"upload": t1 - t0, "job": t2 - t1, "download": t3 - t2,
                        "job_kernels_by_events": sweep_ms / 1e3 + corr_s}}


def finish(args, wl, rank, world, K, W, value, max_secs, ncorr, nlaunch, roofline, e2e, clocks, dist, batched=None):
    L2 = float(wl["L"]) ** 2
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": max_secs * 1e3 / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wl["name"].replace("K sweeps", "%d sweeps" % K), "L": wl["L"], "T": wl["T"],
                       "Delta": wl["Delta"], "seed": wl["seed"], "rmax": wl["rmax"], "sweeps": K,
                       "correlation_points": ncorr, "correlation_share_of_time": wl.get("corr_share"),
                       "thresholds": wl.get("thresholds"),
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (packed lattice %d MiB vs 126 MiB L2), no flush" %
                             (L2 / 8 / (1 << 20) * (1 if wl["model"] == 0 else 2))},
            "roofline": roofline, "e2e": e2e, "gpu_launches": nlaunch + wl.get("corr_launches", 2 * ncorr),
            "clocks": clocks}
    if batched is not None:
        line["batched"] = batched
    if rank == 0:
        if args.cpu_seconds > 0:
            line["cpu_baseline"] = cpu_baseline(wl, budget_s=args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def measured_hbm_gbs() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


def kernel_rev() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in ("k_sweep.cu", "sweep_item.cuh", "philox.cuh", "sweep_args.cuh"):
        with open(os.path.join(ROOT, "paper_2502_18624_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------ oracle (CPU)
def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _timed_sweeps(fn, budget_s: float, max_calls: int):
    """Call fn(i) for i = 0, 1, ... until budget_s has passed (at least once,
    at most max_calls times); returns (calls, seconds)."""
    n, t0 = 0, time.perf_counter()
    while True:
        fn(n)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= max_calls:
            return n, el


def cpu_baseline(wl, budget_s: float = 12.0):
    """The unmodified oracle timed on the host, on one thread and on every
    core (its row-parallel sweep, which equals the sequential one exactly),
    over three workloads: the parity configuration whole (Ising L = 256,
    T = Tc, seed 1234, 100 sweeps), Ising L = 4096 for up to 20 sweeps, and
    the transition-check sweep of this workload (a strip of rows of the full
    lattice, with its halo).  The line's value is the all-core rate on the
    strip, the sample closest to the GPU job."""
    import oracle
    oracle.build()
    nth = host_threads()
    legs = {}

    def leg(name, model, L, T, Delta, seed, sweeps, frac, strip_rows=None):
        thr = oracle.thresholds(model, 1.0, T, Delta)
        out = {}
        for label, threads in (("one_thread", 1), ("all_cores", nth)):
            if strip_rows:
                H = strip_rows
                base = oracle.init_rows(model, L, seed, L - 2, H + 4)
                strip = base.copy()
                fn = lambda i: oracle.sweep_strip_par(model, L, seed, thr, i, 0, strip, threads)
                per_call = (H + 1) * L  # colour 0 on H+2 rows, colour 1 on H rows
            else:
                s = oracle.init(model, L, seed)
                fn = lambda i: oracle.sweep_par(model, s, seed, thr, i, threads)
                per_call = L * L
            b = budget_s * frac * (0.75 if threads == 1 else 0.25)
            n, el = _timed_sweeps(fn, b, sweeps)
            out[label] = {"flips_per_ns": per_call * n / (el * 1e9), "sweeps": n, "seconds": round(el, 3)}
        legs[name] = out

    leg("ising L=256 T=Tc seed=1234, 100 sweeps", 0, 256, TC, 0.0, 1234, 100, 0.1)
    leg("ising L=4096 T=Tc seed=7, 20 sweeps", 0, 4096, TC, 0.0, 7, 20, 0.45)
    H = 64
    strip_name = "%s L=%d: one sweep of a %d-row strip (+2 halo rows each side)" % (
        "ising" if wl["model"] == 0 else "blume-capel", wl["L"], H)
    leg(strip_name, wl["model"], wl["L"], wl["T"], wl["Delta"], wl["seed"], 1 << 30, 0.45, strip_rows=H)
    main = legs[strip_name]
    return {"value": main["all_cores"]["flips_per_ns"], "unit": UNIT, "cores": nth, "kind": "oracle",
            "single_thread": main["one_thread"]["flips_per_ns"], "nproc": os.cpu_count(),
            "sample": "%d sweeps of a %d-row strip (+halo) of the L=%d lattice on %d threads (%.1f s); "
                      "one thread: %d sweeps" % (main["all_cores"]["sweeps"], H, wl["L"], nth,
                                                 main["all_cores"]["seconds"], main["one_thread"]["sweeps"]),
            "legs": legs}


def served_bench(args):
    """Continuous batching on a bounded prefix of the served job stream,
    against the same jobs run one after another on the plain path."""
    import torch

    from paper_2502_18624_gb300 import autotune, serve, workloads
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = dist_init(world, "nccl")
    jobs = workloads.served_jobs(rate=args.rate)[: args.jobs]
    if world > 1:
        jobs = [workloads.Job(j.id, j.model, j.L, j.T, j.Delta, j.seed + 1000003 * rank, j.sweeps, j.arrival)
                for j in jobs]
    sample = workloads.served_jobs(n=64, rate=args.rate, seed=777)
    tiles = autotune.tune(sample, use_cache=False)
    # warm-up: a few tiny jobs through both paths
    warm = workloads.served_jobs(n=6, rate=1e6, seed=5, kmin=8, kmax=8, smin=4, smax=8)
    for _ in range(max(1, args.warmup // 3)):
        e = serve.GpuEngine(8, 8)
        serve.Server(e, 1 << 30, 8).run(warm)
        e.close()
    config = {"workload": "served: first %d jobs of the Poisson stream (%.0f jobs/s, Ising p=0.7 / "
                          "Blume-Capel Delta in {0.5,1,1.5}, L=2^8..2^14, T=[0.7,1.3] Tc_ref, "
                          "sweeps log-uniform 10..10000, C(r<=min(L/2,1024)) at sweeps 2^k), "
                          "seed 20250" % (len(jobs), args.rate),
              "mem_budget_gib": args.mem_gib, "max_batch": args.max_batch, "policy": args.policy,
              "step_updates": args.step_updates, "parallelism": "replicas" if world > 1 else "single"}
    if args.served_part in ("both", "served"):
        eng = serve.GpuEngine(args.max_batch, args.step_sweeps, tiles=tiles)
        srv = serve.Server(eng, mem_budget=int(args.mem_gib * (1 << 30)), max_batch=args.max_batch,
                           step_updates=args.step_updates, max_step_sweeps=args.step_sweeps, policy=args.policy)
        sampler = ClockSampler(gpu_id_for(local)).start()
        barrier(dist, device)
        res = srv.run(jobs)
        clocks = sampler.stop()
        srv_launches = eng.launches
        eng.close()
        served = dict(serve.summarize(res, srv.wall), steps=srv.steps, peak_batch=srv.peak_batch,
                      peak_mem=srv.peak_mem)
        wall = reduce_max(dist, srv.wall, device)
        srv_digests = [serve.digest(r) for r in res]
        if args.served_part == "served":
            # the sequential run follows in another process (it compares these digests)
            if rank == 0 and args.digests:
                with open(args.digests, "w") as f:
                    json.dump({"config": config, "served": served, "wall": wall, "clocks": clocks,
                               "gpu_launches": srv_launches, "ids": [r.job.id for r in res],
                               "digests": srv_digests}, f)
            if rank == 0:
                print(json.dumps({"served_part": "served", "config": config, "served": served, "clocks": clocks,
                                  "gpu_launches": srv_launches, "digests_file": args.digests}), flush=True)
            if dist is not None:
                dist.destroy_process_group()
            return
    else:
        with open(args.digests) as f:
            rec = json.load(f)
        assert rec["config"] == config, "the digests were written for another served workload"
        served, wall, clocks, srv_launches = rec["served"], rec["wall"], rec["clocks"], rec["gpu_launches"]
        srv_digests = rec["digests"]
    seq_eng = serve.GpuEngine(1, 1)
    seq_sampler = ClockSampler(gpu_id_for(local)).start()
    barrier(dist, device)
    t0 = time.perf_counter()
    seq = serve.run_sequential(seq_eng, jobs)
    seq_wall = time.perf_counter() - t0
    seq_clocks = seq_sampler.stop()
    seq_launches = seq_eng.launches
    seq_eng.close()
    s_seq = serve.summarize(seq, seq_wall)
    exact = len(seq) == len(srv_digests) and all(serve.digest(r) == d for r, d in zip(seq, srv_digests))
    value = whole_job(served["updates"], world, wall)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": len(jobs),
                "warmup": args.warmup, "ms_per_step": wall * 1e3 / max(1, len(jobs)), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": config,
                "served": served, "sequential_plain": dict(s_seq, gpu_launches=seq_launches, clocks=seq_clocks),
                "bit_exact": exact, "bit_exact_by": "SHA-256 of every job's records, C(r) and final hash",
                "clocks": clocks, "gpu_launches": srv_launches,
                "served_part": args.served_part}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def reference(args, wl):
    """The oracle as the reference arm: every step is one sweep of a strip of
    rows of the workload's lattice (with its halo), on every host core, the
    strip sized so that warm-up and timed steps end within about a minute."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    nth = host_threads()
    L = wl["L"]
    thr = oracle.thresholds(wl["model"], 1.0, wl["T"], wl["Delta"])
    probe = oracle.init_rows(wl["model"], L, wl["seed"], L - 2, 64 + 4)
    t0 = time.perf_counter()
    oracle.sweep_strip_par(wl["model"], L, wl["seed"], thr, 0, 0, probe, nth)
    per_row = (time.perf_counter() - t0) / 65
    steps_total = max(1, args.steps + args.warmup)
    H = int(max(1, min(1024, 60.0 / steps_total / per_row - 1)))
    strip = oracle.init_rows(wl["model"], L, wl["seed"], L - 2, H + 4)
    for t in range(args.warmup):
        oracle.sweep_strip_par(wl["model"], L, wl["seed"], thr, t, 0, strip, nth)
    t0 = time.perf_counter()
    for t in range(args.steps):
        oracle.sweep_strip_par(wl["model"], L, wl["seed"], thr, args.warmup + t, 0, strip, nth)
    el = time.perf_counter() - t0
    value = (H + 1) * L * args.steps / (el * 1e9)
    sample = ("each step: one sweep of a %d-row strip (+2 halo rows each side) of the L=%d lattice, "
              "on %d host threads" % (H, L, nth))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i8",
            "data": "synthetic",
            "config": {"workload": wl["name"].replace("K sweeps", "%d sweeps" % args.steps), "L": L, "T": wl["T"],
                       "Delta": wl["Delta"], "seed": wl["seed"], "sample_rows": H},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nth, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["served"], default="ising-tc")
    ap.add_argument("--jobs", type=int, default=200, help="served: jobs taken from the start of the stream")
    ap.add_argument("--rate", type=float, default=200.0, help="served: mean arrival rate, jobs/s")
    ap.add_argument("--mem-gib", type=float, default=48.0, help="served: device memory budget")
    ap.add_argument("--max-batch", type=int, default=256, help="served: most jobs resident at once")
    ap.add_argument("--step-updates", type=float, default=1e10, help="served: work per step (spin updates)")
    ap.add_argument("--step-sweeps", type=int, default=16, help="served: most sweeps per job per step")
    ap.add_argument("--policy", choices=["fair", "srpt"], default="srpt",
                    help="served: per-step sweep plan (equal quotas, or shortest remaining work first)")
    ap.add_argument("--served-part", choices=["both", "served", "sequential"], default="both",
                    help="served: run both paths, or one of them (the sequential part compares the digests the "
                         "served part wrote, for streams too long for one process)")
    ap.add_argument("--digests", default=None, help="served: file of per-job result digests (written / read)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="oracle CPU-baseline budget; 0 skips it (profiling runs)")
    ap.add_argument("--L", type=int, default=None, help="override the linear size (small profiling cases)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain leg (profiling runs)")
    args = ap.parse_args(argv)
    if args.workload == "served":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the served workload has no CPU reference arm"}))
            return
        return served_bench(args)
    wl = dict(WORKLOADS[args.workload])
    if args.L:
        wl["L"] = args.L
        wl["rmax"] = min(wl["rmax"], args.L // 2)
        wl["name"] = wl["name"].replace("L=%d" % WORKLOADS[args.workload]["L"], "L=%d" % args.L)
    if args.impl == "reference":
        reference(args, wl)
    else:
        native(args, wl)


if __name__ == "__main__":
    main()
