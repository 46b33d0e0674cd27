"""CPU oracle for the checkerboard Metropolis method (arXiv 2502.18624).

TEST INFRASTRUCTURE ONLY: tests/, the smoke check in __graft_entry__.py and
the CPU-baseline leg of bench.py may import this package; the CUDA library
and its Python binding never do.  The arithmetic lives in oracle.c (plain C,
int8 spins, exact int64 sums); this module compiles it with gcc and wraps
each function with numpy arrays.  See oracle.c for the passage each
function restates and for what pins it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")

ALWAYS = 1 << 32
INIT_SWEEP = 0xFFFFFFFF
TC_ISING = 2.0 / np.log(1.0 + np.sqrt(2.0))  # Onsager's critical temperature, J = 1

_lib = None


_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile oracle.c into lib/liboracle.so with the host gcc (with OpenMP
    for the multi-threaded timing functions when gcc has it)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        try:
            subprocess.check_call(["gcc"] + _CFLAGS + ["-fopenmp", _SRC, "-o", tmp, "-lm"],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(["gcc"] + _CFLAGS + [_SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    """Declare the C signatures on a loaded oracle library and return it."""
    P = ctypes.c_void_p
    u32, u64, i32, f64, sz = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                              ctypes.c_double, ctypes.c_size_t)
    sig = {
        "or_philox4x32_10": (None, [P, P, P]),
        "or_philox_many": (None, [P, sz, P, P]),
        "or_thresholds_ising": (None, [f64, f64, P]),
        "or_thresholds_bc": (None, [f64, f64, f64, P]),
        "or_init": (None, [i32, u32, u64, P]),
        "or_init_rows": (None, [i32, u32, u64, u64, u32, P]),
        "or_sweep": (None, [i32, u32, u64, P, u32, P]),
        "or_run": (None, [i32, u32, u64, P, u32, u32, P, P]),
        "or_sweep_strip": (None, [i32, u32, u64, P, u32, u64, u32, P]),
        "or_measure": (None, [i32, u32, P, P]),
        "or_correlation": (None, [u32, P, u32, P, P]),
        "or_protocol_rc": (u64, [u32, u64]),
        "or_protocol_distances": (u32, [u32, u64, u32, P, u32]),
        "or_protocol_times": (u32, [u64, P, u32]),
        "or_correlation_sampled": (None, [u32, P, u32, P, u32, P, P]),
        "or_sd_hist": (None, [u32, P, P]),
        "or_pack": (None, [i32, u32, P, P]),
        "or_hash_words": (u64, [P, u64]),
        "or_hash": (u64, [i32, u32, P]),
        "or_lut_table": (None, [f64, f64, P]),
        "or_sweep_lut": (None, [u32, u64, P, u32, P]),
        "or_run_lut": (None, [u32, u64, P, u32, u32, P, P]),
        "or_lut_word": (u32, [u64, P, u64, u32, u32, i32]),
        "or_sweep_strip_lut": (None, [u32, u64, P, u32, u64, u32, P]),
        "or_threads_available": (i32, []),
        "or_sweep_par": (None, [i32, u32, u64, P, u32, P, i32]),
        "or_sweep_strip_par": (None, [i32, u32, u64, P, u32, u64, u32, P, i32]),
        "or_init_window": (None, [i32, u32, u64, u64, u64, u32, u32, P]),
        "or_sweep_window": (None, [i32, u32, u64, P, u32, u64, u64, u32, u32, P]),
        "or_sweep_window_lut": (None, [u32, u64, P, u32, u64, u64, u32, u32, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def compile_variant(source_text: str, out_dir: str) -> str:
    """Compile a modified copy of oracle.c (used by tests that plant mistakes)."""
    src = os.path.join(out_dir, "oracle_variant.c")
    lib = os.path.join(out_dir, "liboracle_variant.so")
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", src, "-o", lib, "-lm"])
    return lib


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _key(seed: int) -> np.ndarray:
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one or many counters: ctr (...,4) uint32, key (2,)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(c)
    _load().or_philox_many(_p(c), c.shape[0], _p(k), _p(out))
    return out.reshape(np.shape(ctr))


def thresholds(model: int, J: float, T: float, Delta: float = 0.0) -> np.ndarray:
    """Integer acceptance table: 5 entries (Ising) or 54 (Blume-Capel)."""
    if model == 0:
        t = np.zeros(5, dtype=np.uint64)
        _load().or_thresholds_ising(J, T, _p(t))
    else:
        t = np.zeros(54, dtype=np.uint64)
        _load().or_thresholds_bc(J, Delta, T, _p(t))
    return t


def init(model: int, L: int, seed: int) -> np.ndarray:
    s = np.zeros((L, L), dtype=np.int8)
    _load().or_init(model, L, seed, _p(s))
    return s


def init_rows(model: int, L: int, seed: int, y0: int, nrows: int) -> np.ndarray:
    """Rows y0..y0+nrows-1 (mod L) of the quench, shape (nrows, L)."""
    s = np.zeros((nrows, L), dtype=np.int8)
    _load().or_init_rows(model, L, seed, y0, nrows, _p(s))
    return s


def sweep(model: int, s: np.ndarray, seed: int, thr: np.ndarray, t: int) -> np.ndarray:
    """One sweep (index t) in place; returns s."""
    thr = np.ascontiguousarray(thr, dtype=np.uint64)
    _load().or_sweep(model, s.shape[0], seed, _p(thr), t, _p(s))
    return s


def run(model: int, s: np.ndarray, seed: int, thr: np.ndarray, first: int, n: int,
        record: bool = True):
    """n sweeps from index `first` in place; returns (n,3) int64 (M, B, Q) per sweep."""
    thr = np.ascontiguousarray(thr, dtype=np.uint64)
    obs = np.zeros((n, 3), dtype=np.int64) if record else None
    _load().or_run(model, s.shape[0], seed, _p(thr), first, n, _p(s),
                   _p(obs) if record else None)
    return obs


def sweep_strip(model: int, L: int, seed: int, thr: np.ndarray, t: int, y0: int,
                strip: np.ndarray) -> np.ndarray:
    """Strip form of one sweep: strip holds rows y0-2..y0+H+1; rows 2..H+1 become exact."""
    H = strip.shape[0] - 4
    assert strip.shape == (H + 4, L) and strip.dtype == np.int8
    thr = np.ascontiguousarray(thr, dtype=np.uint64)
    _load().or_sweep_strip(model, L, seed, _p(thr), t, y0, H, _p(strip))
    return strip


def threads_available() -> int:
    """Threads the multi-threaded forms use by default (1 without OpenMP)."""
    return int(_load().or_threads_available())


def sweep_par(model: int, s: np.ndarray, seed: int, thr: np.ndarray, t: int, nthreads: int) -> np.ndarray:
    """One sweep in place on nthreads threads (same result as sweep)."""
    thr = np.ascontiguousarray(thr, dtype=np.uint64)
    _load().or_sweep_par(model, s.shape[0], seed, _p(thr), t, _p(s), nthreads)
    return s


def sweep_strip_par(model: int, L: int, seed: int, thr: np.ndarray, t: int, y0: int, strip: np.ndarray,
                    nthreads: int) -> np.ndarray:
    """Strip sweep on nthreads threads (same result as sweep_strip)."""
    H = strip.shape[0] - 4
    assert strip.shape == (H + 4, L) and strip.dtype == np.int8
    thr = np.ascontiguousarray(thr, dtype=np.uint64)
    _load().or_sweep_strip_par(model, L, seed, _p(thr), t, y0, H, _p(strip), nthreads)
    return strip


def measure(model: int, s: np.ndarray) -> tuple[int, int, int]:
    out = np.zeros(3, dtype=np.int64)
    _load().or_measure(model, s.shape[0], _p(np.ascontiguousarray(s)), _p(out))
    return int(out[0]), int(out[1]), int(out[2])


def correlation(s: np.ndarray, rmax: int) -> tuple[np.ndarray, np.ndarray]:
    cx = np.zeros(rmax + 1, dtype=np.int64)
    cy = np.zeros(rmax + 1, dtype=np.int64)
    _load().or_correlation(s.shape[0], _p(np.ascontiguousarray(s)), rmax, _p(cx), _p(cy))
    return cx, cy


def protocol_rc(L: int, t: int) -> int:
    """r_c(t) of the section 3.3 protocol."""
    return int(_load().or_protocol_rc(L, t))


def protocol_distances(L: int, t: int, R: int = 16) -> np.ndarray:
    """Distances measured from the downsampled sources at time t (uint32, ascending)."""
    n = int(_load().or_protocol_distances(L, t, R, None, 0))
    out = np.zeros(max(n, 1), dtype=np.uint32)
    _load().or_protocol_distances(L, t, R, _p(out), n)
    return out[:n]


def protocol_times(tmax: int) -> np.ndarray:
    """Measurement times floor(2^(x/8) + 0.5) <= tmax (uint64, ascending, distinct)."""
    n = int(_load().or_protocol_times(tmax, None, 0))
    out = np.zeros(max(n, 1), dtype=np.uint64)
    _load().or_protocol_times(tmax, _p(out), n)
    return out[:n]


def correlation_sampled(s: np.ndarray, R: int, r) -> tuple[np.ndarray, np.ndarray]:
    """Sums over one source per R x R square (top-left corner) for each r in the list."""
    rr = np.ascontiguousarray(np.asarray(r, dtype=np.uint32).reshape(-1))
    cx = np.zeros(rr.size, dtype=np.int64)
    cy = np.zeros(rr.size, dtype=np.int64)
    _load().or_correlation_sampled(s.shape[0], _p(np.ascontiguousarray(s)), R, _p(rr), rr.size, _p(cx), _p(cy))
    return cx, cy


def sd_hist(s: np.ndarray) -> np.ndarray:
    h = np.zeros(9, dtype=np.int64)
    _load().or_sd_hist(s.shape[0], _p(np.ascontiguousarray(s)), _p(h))
    return h


def sd_value(hist: np.ndarray, J: float, T: float) -> float:
    """Right-hand side of Eq. (3) from a sigma*h histogram."""
    v = np.arange(-4, 5, dtype=np.float64)
    n = float(hist.sum())
    return float(np.sum(hist.astype(np.float64) * np.exp(-2.0 * J * v / T)) / n)


def pack(model: int, s: np.ndarray) -> np.ndarray:
    L = s.shape[0]
    n = L * (L // 64) * (1 if model == 0 else 2)
    w = np.zeros(n, dtype=np.uint64)
    _load().or_pack(model, L, _p(np.ascontiguousarray(s)), _p(w))
    return w


def lattice_hash(model: int, s: np.ndarray) -> int:
    return int(_load().or_hash(model, s.shape[0], _p(np.ascontiguousarray(s))))


def hash_words(words: np.ndarray) -> int:
    w = np.ascontiguousarray(words, dtype=np.uint64)
    return int(_load().or_hash_words(_p(w), w.size))


def energy(model: int, obs, J: float = 1.0, Delta: float = 0.0) -> float:
    """E = -J B + Delta Q from exact (M, B, Q) integers (Eqs. (1)-(2))."""
    _, B, Q = obs
    return -J * float(B) + (Delta * float(Q) if model == 1 else 0.0)


# ---- the paper's lookup-table random bits (Ising, section 3.2) ----------------

def lut_table(J: float, T: float) -> np.ndarray:
    t = np.zeros(16, dtype=np.uint32)
    _load().or_lut_table(J, T, _p(t))
    return t


def sweep_lut(s: np.ndarray, seed: int, tbl: np.ndarray, t: int) -> np.ndarray:
    tbl = np.ascontiguousarray(tbl, dtype=np.uint32)
    _load().or_sweep_lut(s.shape[0], seed, _p(tbl), t, _p(s))
    return s


def run_lut(s: np.ndarray, seed: int, tbl: np.ndarray, first: int, n: int, record: bool = True):
    tbl = np.ascontiguousarray(tbl, dtype=np.uint32)
    obs = np.zeros((n, 3), dtype=np.int64) if record else None
    _load().or_run_lut(s.shape[0], seed, _p(tbl), first, n, _p(s), _p(obs) if record else None)
    return obs


def lut_word(seed: int, tbl: np.ndarray, w: int, t: int, colour: int, which: int) -> int:
    tbl = np.ascontiguousarray(tbl, dtype=np.uint32)
    return int(_load().or_lut_word(seed, _p(tbl), w, t, colour, which))


def sweep_strip_lut(L: int, seed: int, tbl: np.ndarray, t: int, y0: int, strip: np.ndarray) -> np.ndarray:
    H = strip.shape[0] - 4
    assert strip.shape == (H + 4, L) and strip.dtype == np.int8
    tbl = np.ascontiguousarray(tbl, dtype=np.uint32)
    _load().or_sweep_strip_lut(L, seed, _p(tbl), t, y0, H, _p(strip))
    return strip


# ---- light-cone windows (lattices too large to hold as int8) ------------------

def init_window(model: int, L: int, seed: int, y0: int, x0: int, H: int, Wd: int) -> np.ndarray:
    """Quench of the H x Wd window at (y0, x0), wrapping modulo L."""
    w = np.zeros((H, Wd), dtype=np.int8)
    _load().or_init_window(model, L, seed, y0, x0, H, Wd, _p(w))
    return w


def sweep_window(model: int, L: int, seed: int, thr: np.ndarray, t: int, y0: int, x0: int,
                 win: np.ndarray) -> np.ndarray:
    """One non-periodic window sweep in place; the exact block shrinks by 2 per side."""
    thr = np.ascontiguousarray(thr, dtype=np.uint64)
    H, Wd = win.shape
    assert win.dtype == np.int8 and win.flags["C_CONTIGUOUS"] and H <= L and Wd <= L
    _load().or_sweep_window(model, L, seed, _p(thr), t, y0, x0, H, Wd, _p(win))
    return win


def sweep_window_lut(L: int, seed: int, tbl: np.ndarray, t: int, y0: int, x0: int, win: np.ndarray) -> np.ndarray:
    tbl = np.ascontiguousarray(tbl, dtype=np.uint32)
    H, Wd = win.shape
    assert win.dtype == np.int8 and win.flags["C_CONTIGUOUS"] and H <= L and Wd <= L
    _load().or_sweep_window_lut(L, seed, _p(tbl), t, y0, x0, H, Wd, _p(win))
    return win


def light_cone(model: int, L: int, seed: int, T: float, t: int, y0: int, x0: int, W: int,
               Delta: float = 0.0, lut: bool = False) -> np.ndarray:
    """The W x W block at (y0, x0) after t sweeps from the quench, computed on
    the (W + 4t)^2 window around it (its light cone)."""
    m = 2 * t
    win = init_window(model, L, seed, (y0 - m) % L, (x0 - m) % L, W + 2 * m, W + 2 * m)
    if lut:
        tbl = lut_table(1.0, T)
        for k in range(t):
            sweep_window_lut(L, seed, tbl, k, (y0 - m) % L, (x0 - m) % L, win)
    else:
        thr = thresholds(model, 1.0, T, Delta)
        for k in range(t):
            sweep_window(model, L, seed, thr, k, (y0 - m) % L, (x0 - m) % L, win)
    return win[m:m + W, m:m + W].copy()
