"""ctypes binding of include/lat.h: the same entry-point names, argument
marshalling only.  Every step of the simulation runs in liblat.so's CUDA
kernels; if the library is missing or cannot be built this module raises, it
never falls back to anything else.

PyTorch is used only for device memory (a uint8 tensor handed to lat_create
as the caller-owned buffer) and for streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

LAT_OK, LAT_EINVAL, LAT_ENOMEM, LAT_ECUDA, LAT_ETIMEDOUT, LAT_ESTATE = 0, -1, -2, -3, -4, -5
LAT_ISING, LAT_BLUME_CAPEL = 0, 1
LAT_RNG_SITE, LAT_RNG_TABLE = 0, 1
LAT_MAX_L = 1 << 20
TC_ISING = 2.0 / np.log(1.0 + np.sqrt(2.0))


class LatError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s failed: %s (%d)" % (what, strerror(code), code))
        self.code = code


class lat_params(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("L", ctypes.c_uint32), ("J", ctypes.c_double),
                ("Delta", ctypes.c_double), ("T", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("rng", ctypes.c_int32)]


class lat_obs(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("B", ctypes.c_int64), ("Q", ctypes.c_int64),
                ("sweep", ctypes.c_uint64), ("draws", ctypes.c_uint64)]


OBS_DTYPE = np.dtype([("M", np.int64), ("B", np.int64), ("Q", np.int64), ("sweep", np.uint64),
                      ("draws", np.uint64)])

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblat.so (building it first if needed); raise if that fails."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("liblat.so is missing (%s); run build()" % _build.LIB)
    lib = ctypes.CDLL(_build.LIB)
    P, sz, u32, u64, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    PP = ctypes.POINTER(lat_params)
    sigs = {
        "lat_footprint": (sz, [PP]),
        "lat_state_bytes": (sz, [PP]),
        "lat_thresholds": (i32, [PP, P, sz]),
        "lat_lut_table": (i32, [PP, P]),
        "lat_create": (i32, [PP, P, sz, P, ctypes.POINTER(P)]),
        "lat_sweep": (i32, [P, u32, P]),
        "lat_sweep_sd": (i32, [P, u32, P, P]),
        "lat_measure": (i32, [P, P]),
        "lat_correlation": (i32, [P, u32, P, P]),
        "lat_protocol_rc": (u64, [u32, u64]),
        "lat_protocol_distances": (u32, [u32, u64, u32, P, u32]),
        "lat_protocol_times": (u32, [u64, P, u32]),
        "lat_correlation_sampled": (i32, [P, u32, P, u32, P, P]),
        "lat_correlation_protocol": (i32, [P, u64, u32, u32, P, P, P, P, P]),
        "lat_sd_hist": (i32, [P, P]),
        "lat_spin_counts": (i32, [P, P]),
        "lat_hash": (i32, [P, P]),
        "lat_get_spins": (i32, [P, P]),
        "lat_get_rows": (i32, [P, u32, u32, P]),
        "lat_set_spins": (i32, [P, P]),
        "lat_get_state": (i32, [P, P, sz]),
        "lat_set_state": (i32, [P, P, sz]),
        "lat_get_sweep_index": (i32, [P, P]),
        "lat_set_sweep_index": (i32, [P, u64]),
        "lat_get_thresholds": (i32, [P, P, sz]),
        "lat_destroy": (i32, [P]),
        "lat_strerror": (ctypes.c_char_p, [i32]),
        "lat_runner_footprint": (sz, [u32, u32]),
        "lat_runner_create": (i32, [u32, u32, P, sz, P, ctypes.POINTER(P)]),
        "lat_runner_set_tile": (i32, [P, ctypes.c_int32, u32, u32]),
        "lat_runner_set_timeout": (i32, [P, u64]),
        "lat_runner_run": (i32, [P, P, u32, P, P]),
        "lat_runner_destroy": (i32, [P]),
        "lat_runner_inject_stall": (i32, [P, u32]),
        "lat_runner_set_counter_base": (i32, [P, u64]),
        "lat_runner_submit": (i32, [P, P, u32, P]),
        "lat_runner_collect": (i32, [P, P]),
        "lat_correlation_async": (i32, [P, u32, P, P]),
        "lat_hash_async": (i32, [P, P]),
        "lat_probe_rates": (i32, [P, P]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(code: int, what: str) -> None:
    if code != LAT_OK:
        raise LatError(code, what)


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def make_params(model: int, L: int, T: float, seed: int, J: float = 1.0, Delta: float = 0.0,
                rng: int = LAT_RNG_SITE) -> lat_params:
    return lat_params(int(model), int(L), float(J), float(Delta), float(T), int(seed) & (2**64 - 1), int(rng))


def strerror(code: int) -> str:
    return load().lat_strerror(code).decode()


# ---- entry points with the C names -----------------------------------------

def lat_footprint(p: lat_params) -> int:
    return int(load().lat_footprint(ctypes.byref(p)))


def lat_state_bytes(p: lat_params) -> int:
    return int(load().lat_state_bytes(ctypes.byref(p)))


def lat_thresholds(p: lat_params) -> np.ndarray:
    out = np.zeros(54, dtype=np.uint64)
    _check(load().lat_thresholds(ctypes.byref(p), _ptr(out), out.size), "lat_thresholds")
    return out[: (5 if p.model == LAT_ISING else 54)].copy()


def lat_lut_table(p: lat_params) -> np.ndarray:
    out = np.zeros(16, dtype=np.uint32)
    _check(load().lat_lut_table(ctypes.byref(p), _ptr(out)), "lat_lut_table")
    return out


def lat_create(p: lat_params, dev_buf: int | None, nbytes: int, stream: int | None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().lat_create(ctypes.byref(p), dev_buf, nbytes, stream, ctypes.byref(h)), "lat_create")
    return h


def lat_sweep(h, nsweeps: int, record: bool = True):
    obs = np.zeros(nsweeps, dtype=OBS_DTYPE) if record else None
    _check(load().lat_sweep(h, nsweeps, _ptr(obs) if record and nsweeps else None), "lat_sweep")
    return obs


def lat_sweep_sd(h, nsweeps: int, record: bool = True):
    """nsweeps sweeps with the fused Schwinger-Dyson histogram after each:
    returns (records or None, int64 array (nsweeps, 9))."""
    obs = np.zeros(nsweeps, dtype=OBS_DTYPE) if record else None
    sd = np.zeros((max(nsweeps, 1), 9), dtype=np.int64)
    _check(load().lat_sweep_sd(h, nsweeps, _ptr(obs) if record and nsweeps else None, _ptr(sd)), "lat_sweep_sd")
    return obs, sd[:nsweeps]


def lat_measure(h) -> tuple[int, int, int, int]:
    o = lat_obs()
    _check(load().lat_measure(h, ctypes.byref(o)), "lat_measure")
    return o.M, o.B, o.Q, o.sweep


def lat_correlation(h, rmax: int) -> tuple[np.ndarray, np.ndarray]:
    cx = np.zeros(rmax + 1, dtype=np.int64)
    cy = np.zeros(rmax + 1, dtype=np.int64)
    _check(load().lat_correlation(h, rmax, _ptr(cx), _ptr(cy)), "lat_correlation")
    return cx, cy


def lat_protocol_rc(L: int, t: int) -> int:
    return int(load().lat_protocol_rc(L, t))


def lat_protocol_distances(L: int, t: int, R: int = 16) -> np.ndarray:
    n = int(load().lat_protocol_distances(L, t, R, None, 0))
    out = np.zeros(max(n, 1), dtype=np.uint32)
    load().lat_protocol_distances(L, t, R, _ptr(out), n)
    return out[:n]


def lat_protocol_times(tmax: int) -> np.ndarray:
    n = int(load().lat_protocol_times(tmax, None, 0))
    out = np.zeros(max(n, 1), dtype=np.uint64)
    load().lat_protocol_times(tmax, _ptr(out), n)
    return out[:n]


def lat_correlation_sampled(h, R: int, r) -> tuple[np.ndarray, np.ndarray]:
    rr = np.ascontiguousarray(np.asarray(r, dtype=np.uint32).reshape(-1))
    cx = np.zeros(max(rr.size, 1), dtype=np.int64)
    cy = np.zeros(max(rr.size, 1), dtype=np.int64)
    _check(load().lat_correlation_sampled(h, R, _ptr(rr) if rr.size else None, rr.size, _ptr(cx), _ptr(cy)),
           "lat_correlation_sampled")
    return cx[:rr.size], cy[:rr.size]


def lat_correlation_protocol(h, t: int, R: int = 16) -> dict:
    """One section 3.3 measurement: {"r", "cx", "cy", "nsrc"} rows in ascending r."""
    n = ctypes.c_uint32(0)
    _check(load().lat_correlation_protocol(h, t, R, 0, ctypes.byref(n), None, None, None, None),
           "lat_correlation_protocol")
    k = n.value
    r = np.zeros(k, dtype=np.uint32)
    cx = np.zeros(k, dtype=np.int64)
    cy = np.zeros(k, dtype=np.int64)
    ns = np.zeros(k, dtype=np.uint64)
    _check(load().lat_correlation_protocol(h, t, R, k, ctypes.byref(n), _ptr(r), _ptr(cx), _ptr(cy), _ptr(ns)),
           "lat_correlation_protocol")
    return {"r": r, "cx": cx, "cy": cy, "nsrc": ns}


def lat_spin_counts(h) -> np.ndarray:
    """Sites holding -1, 0, +1, and invalid Blume-Capel codes (int64[4])."""
    out = np.zeros(4, dtype=np.int64)
    _check(load().lat_spin_counts(h, _ptr(out)), "lat_spin_counts")
    return out


def lat_sd_hist(h) -> np.ndarray:
    out = np.zeros(9, dtype=np.int64)
    _check(load().lat_sd_hist(h, _ptr(out)), "lat_sd_hist")
    return out


def lat_hash(h) -> int:
    out = np.zeros(1, dtype=np.uint64)
    _check(load().lat_hash(h, _ptr(out)), "lat_hash")
    return int(out[0])


def lat_get_spins(h, L: int) -> np.ndarray:
    out = np.empty((L, L), dtype=np.int8)
    _check(load().lat_get_spins(h, _ptr(out)), "lat_get_spins")
    return out


def lat_get_rows(h, L: int, y0: int, nrows: int) -> np.ndarray:
    out = np.empty((nrows, L), dtype=np.int8)
    _check(load().lat_get_rows(h, y0, nrows, _ptr(out)), "lat_get_rows")
    return out


def lat_set_spins(h, s: np.ndarray) -> None:
    s = np.ascontiguousarray(s, dtype=np.int8)
    _check(load().lat_set_spins(h, _ptr(s)), "lat_set_spins")


def lat_get_state(h, nbytes: int, out: np.ndarray | None = None) -> np.ndarray:
    out = np.empty(nbytes, dtype=np.uint8) if out is None else out
    _check(load().lat_get_state(h, _ptr(out), nbytes), "lat_get_state")
    return out


def lat_set_state(h, state: np.ndarray) -> None:
    state = np.ascontiguousarray(state).view(np.uint8)
    _check(load().lat_set_state(h, _ptr(state), state.nbytes), "lat_set_state")


def lat_get_sweep_index(h) -> int:
    v = ctypes.c_uint64()
    _check(load().lat_get_sweep_index(h, ctypes.byref(v)), "lat_get_sweep_index")
    return v.value


def lat_set_sweep_index(h, t: int) -> None:
    _check(load().lat_set_sweep_index(h, t), "lat_set_sweep_index")


def lat_get_thresholds(h, model: int) -> np.ndarray:
    out = np.zeros(54, dtype=np.uint64)
    _check(load().lat_get_thresholds(h, _ptr(out), out.size), "lat_get_thresholds")
    return out[: (5 if model == LAT_ISING else 54)].copy()


def lat_destroy(h) -> None:
    _check(load().lat_destroy(h), "lat_destroy")


def lat_probe_rates() -> dict:
    """Measured integer-pipe rates of the current device (lane-operations per second;
    Philox in full blocks per second)."""
    r = np.zeros(5, dtype=np.float64)
    t = np.zeros(5, dtype=np.float64)
    _check(load().lat_probe_rates(_ptr(r), _ptr(t)), "lat_probe_rates")
    return {"imad_ops_per_s": float(r[0]), "lop3_per_s": float(r[1]), "popc_per_s": float(r[2]),
            "philox_blocks_per_s": float(r[3]), "imad32_per_s": float(r[4]), "seconds": [float(x) for x in t]}


# ---- convenience wrapper over torch device memory ---------------------------

class Lattice:
    """One lattice on the current CUDA device, in a torch-owned buffer."""

    def __init__(self, model: int, L: int, T: float, seed: int, J: float = 1.0, Delta: float = 0.0,
                 stream=None, device=None, rng: int = LAT_RNG_SITE):
        import torch

        self.params = make_params(model, L, T, seed, J, Delta, rng)
        self.model, self.L = int(model), int(L)
        nbytes = lat_footprint(self.params)
        if nbytes == 0:
            raise LatError(LAT_EINVAL, "lat_footprint")
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.handle = lat_create(self.params, self.buffer.data_ptr(), nbytes, self.stream.cuda_stream)

    def sweep(self, n: int, record: bool = True):
        return lat_sweep(self.handle, n, record)

    def sweep_sd(self, n: int, record: bool = True):
        return lat_sweep_sd(self.handle, n, record)

    def measure(self):
        return lat_measure(self.handle)

    def correlation(self, rmax: int):
        return lat_correlation(self.handle, rmax)

    def correlation_sampled(self, R: int, r):
        return lat_correlation_sampled(self.handle, R, r)

    def correlation_protocol(self, t: int, R: int = 16) -> dict:
        return lat_correlation_protocol(self.handle, t, R)

    def sd_hist(self):
        return lat_sd_hist(self.handle)

    def spin_counts(self) -> np.ndarray:
        return lat_spin_counts(self.handle)

    def hash(self) -> int:
        return lat_hash(self.handle)

    def spins(self) -> np.ndarray:
        return lat_get_spins(self.handle, self.L)

    def rows(self, y0: int, nrows: int) -> np.ndarray:
        return lat_get_rows(self.handle, self.L, y0, nrows)

    def set_spins(self, s: np.ndarray) -> None:
        lat_set_spins(self.handle, s)

    def state(self) -> np.ndarray:
        return lat_get_state(self.handle, lat_state_bytes(self.params))

    def set_state(self, st: np.ndarray) -> None:
        lat_set_state(self.handle, st)

    @property
    def sweep_index(self) -> int:
        return lat_get_sweep_index(self.handle)

    @sweep_index.setter
    def sweep_index(self, t: int) -> None:
        lat_set_sweep_index(self.handle, t)

    def thresholds(self) -> np.ndarray:
        return lat_get_thresholds(self.handle, self.model)

    def close(self) -> None:
        if getattr(self, "handle", None):
            lat_destroy(self.handle)
            self.handle = None
        self.buffer = None  # the device buffer goes back to torch's allocator

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- runner: many lattices in one persistent launch -------------------------

def lat_runner_footprint(max_lattices: int, max_sweeps: int) -> int:
    return int(load().lat_runner_footprint(max_lattices, max_sweeps))


def lat_runner_create(max_lattices: int, max_sweeps: int, dev_buf: int | None, nbytes: int,
                      stream: int | None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().lat_runner_create(max_lattices, max_sweeps, dev_buf, nbytes, stream, ctypes.byref(h)),
           "lat_runner_create")
    return h


def lat_runner_set_tile(r, model: int, L: int, tile_items: int) -> None:
    _check(load().lat_runner_set_tile(r, model, L, tile_items), "lat_runner_set_tile")


def lat_runner_set_timeout(r, ns: int) -> None:
    _check(load().lat_runner_set_timeout(r, ns), "lat_runner_set_timeout")


def lat_runner_run(r, handles, nsweeps, record: bool = True):
    """Advance handles[i] by nsweeps[i]; returns a list of per-sweep record arrays (or None)."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value for h in handles])
    ns = np.ascontiguousarray(nsweeps, dtype=np.uint32)
    outs = [np.zeros(int(k), dtype=OBS_DTYPE) for k in ns] if record else None
    ptrs = (ctypes.c_void_p * n)(*[o.ctypes.data if (o is not None and o.size) else None for o in outs]) \
        if record else None
    code = load().lat_runner_run(r, hs, n, _ptr(ns), ptrs)
    _check(code, "lat_runner_run")
    return outs


def lat_runner_submit(r, handles, nsweeps) -> None:
    """Enqueue a run (advance handles[i] by nsweeps[i]) without waiting."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value for h in handles])
    ns = np.ascontiguousarray(nsweeps, dtype=np.uint32)
    _check(load().lat_runner_submit(r, hs, n, _ptr(ns)), "lat_runner_submit")


def lat_runner_collect(r, nsweeps, record: bool = True):
    """Wait for the submitted run; per-sweep record arrays (or None)."""
    n = len(nsweeps)
    outs = [np.zeros(int(k), dtype=OBS_DTYPE) for k in nsweeps] if record else None
    ptrs = (ctypes.c_void_p * n)(*[o.ctypes.data if (o is not None and o.size) else None for o in outs]) \
        if record else None
    _check(load().lat_runner_collect(r, ptrs), "lat_runner_collect")
    return outs


def lat_correlation_async(h, rmax: int, cx: np.ndarray, cy: np.ndarray) -> None:
    """Enqueue C(r <= rmax) into cx, cy (int64, rmax+1 each; page-locked memory for no wait)."""
    assert cx.dtype == np.int64 and cy.dtype == np.int64 and cx.size > rmax and cy.size > rmax
    _check(load().lat_correlation_async(h, rmax, _ptr(cx), _ptr(cy)), "lat_correlation_async")


def lat_hash_async(h, out: np.ndarray) -> None:
    """Enqueue the lattice hash into out[0] (uint64, page-locked memory for no wait)."""
    assert out.dtype == np.uint64 and out.size >= 1
    _check(load().lat_hash_async(h, _ptr(out)), "lat_hash_async")


def lat_runner_inject_stall(r, index: int) -> None:
    _check(load().lat_runner_inject_stall(r, index), "lat_runner_inject_stall")


def lat_runner_set_counter_base(r, base: int) -> None:
    _check(load().lat_runner_set_counter_base(r, base), "lat_runner_set_counter_base")


def lat_runner_destroy(r) -> None:
    _check(load().lat_runner_destroy(r), "lat_runner_destroy")


class Runner:
    """A runner in a torch-owned device buffer, on the current stream."""

    def __init__(self, max_lattices: int, max_sweeps: int, stream=None, device=None):
        import torch

        nbytes = lat_runner_footprint(max_lattices, max_sweeps)
        if nbytes == 0:
            raise LatError(LAT_EINVAL, "lat_runner_footprint")
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.handle = lat_runner_create(max_lattices, max_sweeps, self.buffer.data_ptr(), nbytes,
                                        self.stream.cuda_stream)
        self.max_lattices, self.max_sweeps = max_lattices, max_sweeps

    def set_tile(self, model: int, L: int, tile_items: int) -> None:
        lat_runner_set_tile(self.handle, model, L, tile_items)

    def set_timeout(self, ns: int) -> None:
        lat_runner_set_timeout(self.handle, ns)

    def inject_stall(self, index: int) -> None:
        lat_runner_inject_stall(self.handle, index)

    def set_counter_base(self, base: int) -> None:
        lat_runner_set_counter_base(self.handle, base)

    def run(self, lattices, nsweeps, record: bool = True):
        return lat_runner_run(self.handle, [lt.handle for lt in lattices], nsweeps, record)

    def submit(self, lattices, nsweeps) -> None:
        lat_runner_submit(self.handle, [lt.handle for lt in lattices], nsweeps)

    def collect(self, nsweeps, record: bool = True):
        return lat_runner_collect(self.handle, nsweeps, record)

    def close(self) -> None:
        if getattr(self, "handle", None):
            lat_runner_destroy(self.handle)
            self.handle = None
        self.buffer = None  # the device buffer goes back to torch's allocator

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
