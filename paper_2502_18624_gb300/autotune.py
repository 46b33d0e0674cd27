"""Autotuner for the runner's tile schedule.

The runner splits every colour phase of a lattice into tiles of
`tile_items` work items; the best size depends on the lattice size (small
lattices want one tile, large ones enough tiles to spread over the SMs and
to start the next phase before the slowest tile of this one ends) and on
what else is in the batch.  tune() times the real mixed batch for a few
sweeps and does one round of coordinate descent over the (model, L) size
classes, trying each candidate tile size for one class while the others
keep their current choice.  Results do not depend on the schedule, only the
time does.  A cache keyed by GPU name and size class avoids re-tuning.
"""
from __future__ import annotations

import json
import os

CANDIDATES = (256, 1024, 4096, 16384, 65536)


def _items(model: int, L: int) -> int:
    W = L // 64
    return L * (W // 2 if (model == 0 and W % 2 == 0) else W)


def _cache_path(gpu_name: str) -> str:
    root = os.environ.get("LAT_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "gb300_lattice"))
    return os.path.join(root, "tiles-%s.json" % gpu_name.replace(" ", "_"))


def load_cache(gpu_name: str) -> dict:
    try:
        with open(_cache_path(gpu_name)) as f:
            return {tuple(map(int, k.split(":"))): int(v) for k, v in json.load(f).items()}
    except (OSError, ValueError):
        return {}


def save_cache(gpu_name: str, sched: dict) -> None:
    path = _cache_path(gpu_name)
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump({"%d:%d" % k: v for k, v in sched.items()}, f, indent=1)
    except OSError:
        pass


def apply(runner, sched: dict) -> None:
    for (model, L), tile in sched.items():
        runner.set_tile(model, L, tile)


def tune(jobs, sweeps: int = 6, repeats: int = 2, use_cache: bool = True, verbose: bool = False) -> dict:
    """Pick a tile size per (model, L) class present in `jobs` (workloads.Job list)."""
    import torch

    from . import binding as b

    gpu = torch.cuda.get_device_name()
    classes = sorted({(j.model, j.L) for j in jobs})
    if use_cache:
        cached = load_cache(gpu)
        if all(c in cached for c in classes):
            return {c: cached[c] for c in classes}
    lats = [b.Lattice(j.model, j.L, j.T, j.seed, Delta=j.Delta) for j in jobs]
    runner = b.Runner(len(jobs), sweeps)
    stream = runner.stream
    sched = {c: min(4096, max(256, (_items(*c) + 255) // 256 * 256)) for c in classes}

    def timed() -> float:
        apply(runner, sched)
        best = float("inf")
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            runner.run(lats, [sweeps] * len(lats), record=False)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    base = timed()
    for c in sorted(classes, key=lambda c: -c[1]):  # largest lattices first: they carry most of the work
        items = _items(*c)
        best_tile, best_t = sched[c], base
        for tile in CANDIDATES:
            if tile > max(256, items) * 2 or tile == sched[c]:
                continue
            old = sched[c]
            sched[c] = tile
            t = timed()
            if verbose:
                print("tile", c, tile, "%.3f ms" % t)
            if t < best_t:
                best_tile, best_t = tile, t
            sched[c] = old
        sched[c] = best_tile
        base = best_t
    runner.close()
    for lt in lats:
        lt.close()
    if use_cache:
        merged = load_cache(gpu)
        merged.update(sched)
        save_cache(gpu, merged)
    return sched
