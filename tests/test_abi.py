"""The C-ABI library on a machine without a GPU: it loads, exports every
symbol include/*.h declares, its host-only calls work, and the calls that
need a device fail with LAT_ECUDA instead of computing anything on the CPU.
The acceptance table it builds (its own FP64 code) equals the oracle's bit
for bit over the workload parameter ranges.
"""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2502_18624_gb300 import binding as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b([a-z_][a-z0-9_]*)\s*\(", text):
            name = m.group(1)
            if name.startswith("lat_") and not name.endswith("_t"):
                names.add(name)
    return sorted(names)


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(b.load().__dict__["_name"])
    names = _declared_functions()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm103a():
    # The build passes exactly one -gencode for sm_103a.
    from paper_2502_18624_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(_build.LIB)


@pytest.mark.parametrize("model,L,J,T,Delta", [
    (0, 64, 1.0, 1.0, 0.0), (1, 64, 1.0, 1.0, 0.0),
    (0, 100, 1.0, 1.0, 0.0), (0, 32, 1.0, 1.0, 0.0), (0, 0, 1.0, 1.0, 0.0),
    (0, (1 << 20) + 64, 1.0, 1.0, 0.0), (1, 1 << 20, 1.0, 1.0, 0.0),
    (0, 64, 0.0, 1.0, 0.0), (0, 64, -1.0, 1.0, 0.0), (0, 64, 1.0, 0.0, 0.0), (0, 64, 1.0, -2.0, 0.0),
    (2, 64, 1.0, 1.0, 0.0), (0, 64, float("nan"), 1.0, 0.0), (1, 64, 1.0, 1.0, float("inf")),
])
def test_parameter_validation(model, L, J, T, Delta):
    p = b.make_params(model, L, T, 1, J, Delta)
    valid = model in (0, 1) and L >= 64 and L % 64 == 0 and J > 0 and T > 0 and np.isfinite(J) \
        and np.isfinite(Delta) and L <= (1 << 20) and not (model == 1 and L > (1 << 19))
    assert (b.lat_footprint(p) > 0) == valid
    if not valid:
        with pytest.raises(b.LatError) as e:
            b.lat_thresholds(p)
        assert e.value.code == b.LAT_EINVAL


def test_footprint_covers_the_packed_lattice():
    for model, L in [(0, 64), (0, 1 << 17), (0, 1 << 19), (1, 1 << 16), (1, 192)]:
        p = b.make_params(model, L, 1.0, 1)
        state = b.lat_state_bytes(p)
        assert state == L * L // (8 if model == 0 else 4)
        # + a 1/16 copy of the source columns (downsampled correlation) and small buffers
        assert state <= b.lat_footprint(p) <= state + state // 16 + (6 << 20) + 40 * L


def test_protocol_host_functions_equal_the_oracle(orc):
    """r_c(t), the downsampled distances and the measurement times: library
    (host C++) and oracle (C) compute them separately, in FP64, and must give
    the same integers."""
    for L in (64, 256, 1024, 3 << 10, 1 << 16, 1 << 17, 1 << 19, 1 << 20):
        for t in list(range(1, 400)) + [1000, 1850, 10**5, 524288, 10**7, 10**9]:
            assert b.lat_protocol_rc(L, t) == orc.protocol_rc(L, t)
        for t in (1, 1000, 10**5, 10**7):
            for R in (1, 16, 64):
                assert np.array_equal(b.lat_protocol_distances(L, t, R), orc.protocol_distances(L, t, R)), (L, t, R)
    for tmax in (1, 13, 1000, 1 << 20, 1 << 40):
        assert np.array_equal(b.lat_protocol_times(tmax), orc.protocol_times(tmax))


def test_device_calls_fail_loudly_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = b.make_params(0, 256, b.TC_ISING, 1234)
    with pytest.raises(b.LatError) as e:
        b.lat_create(p, None, 0, None)
    assert e.value.code == b.LAT_ECUDA


def _cases():
    rng = np.random.default_rng(2025)
    cases = [(0, 1.0, b.TC_ISING, 0.0), (0, 1.0, 0.9 * b.TC_ISING, 0.0), (0, 1.0, 2.269185, 0.0),
             (1, 1.0, 1.398, 1.0), (1, 1.0, 1.69, 0.5), (1, 1.0, 1.69, 1.5), (1, 1.0, 0.608, 1.966),
             (0, 1.0, 1e-3, 0.0), (0, 1.0, 1e15, 0.0), (1, 1.0, 1e-3, 1.0), (1, 0.7, 2.5, -0.3)]
    for _ in range(40):
        cases.append((0, 1.0, float(rng.uniform(0.8, 1.2) * 2.269185), 0.0))
        cases.append((1, 1.0, float(rng.uniform(1.2, 1.6)), 1.0))
        cases.append((1, 1.0, float(rng.uniform(0.7, 1.3) * 1.69), float(rng.choice([0.5, 1.5]))))
    return cases


def test_thresholds_equal_the_oracle_bit_for_bit(orc):
    for model, J, T, Delta in _cases():
        p = b.make_params(model, 64, T, 1, J, Delta)
        lib = b.lat_thresholds(p)
        ref = orc.thresholds(model, J, T, Delta)
        assert np.array_equal(lib, ref), (model, J, T, Delta)


def test_lut_tables_equal_the_oracle_bit_for_bit(orc):
    rng = np.random.default_rng(9)
    temps = [b.TC_ISING, 0.9 * b.TC_ISING, 0.05, 0.3, 50.0, 1e12] + list(rng.uniform(0.5, 5.0, 40))
    for T in temps:
        for J in (1.0, 0.5):
            p = b.make_params(0, 128, float(T), 1, J=J, rng=b.LAT_RNG_TABLE)
            assert np.array_equal(b.lat_lut_table(p), orc.lut_table(J, float(T))), (J, T)


def test_lut_mode_is_ising_only():
    assert b.lat_footprint(b.make_params(1, 128, 1.0, 1, rng=b.LAT_RNG_TABLE)) == 0
    assert b.lat_footprint(b.make_params(0, 128, 1.0, 1, rng=2)) == 0
    assert b.lat_footprint(b.make_params(0, 128, 1.0, 1, rng=b.LAT_RNG_TABLE)) > 0


def test_static_correlation_checks_arguments_before_any_device_call():
    """lat_correlation_static (the entry point that allocates nothing)
    rejects a lattice pointer the correlation kernels could not load from
    (not 16-byte aligned), an rmax beyond its fixed scratch, and bad sizes,
    with LAT_EINVAL before it touches the device; its limit in lat.h is
    4096 distances."""
    text = open(os.path.join(ROOT, "include", "lat.h")).read()
    m = re.search(r"#define\s+LAT_STATIC_RMAX\s+(\d+)u?", text)
    assert m and int(m.group(1)) == 4096
    f = b.load().lat_correlation_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    cx = np.zeros(4098, dtype=np.int64)
    cy = np.zeros(4098, dtype=np.int64)
    px, py = cx.ctypes.data_as(ctypes.c_void_p), cy.ctypes.data_as(ctypes.c_void_p)
    fake = 1 << 40   # never dereferenced: every case below must fail its argument checks first
    for model, L, ptr, rmax in [(0, 256, fake + 8, 4), (1, 256, fake + 4, 4), (0, 256, fake + 1, 0),
                                (0, 16384, fake, 4097), (0, 256, fake, 129), (0, 100, fake, 4), (2, 256, fake, 4),
                                (0, 256, None, 4)]:
        assert f(model, L, ptr, rmax, px, py, None) == b.LAT_EINVAL, (model, L, ptr, rmax)
    assert f(0, 256, fake, 4, None, py, None) == b.LAT_EINVAL


def test_entry_points_check_null_arguments_without_a_device():
    """Calls that take a handle refuse a NULL one (and the runner's halves a
    NULL runner) with LAT_EINVAL, before any device work."""
    lib = b.load()
    P = ctypes.c_void_p
    buf = np.zeros(16, dtype=np.int64)
    ptr = buf.ctypes.data_as(P)
    for name, args in [("lat_sweep_sd", [None, 1, None, ptr]), ("lat_correlation_async", [None, 4, ptr, ptr]),
                       ("lat_hash_async", [None, ptr]), ("lat_runner_submit", [None, None, 1, ptr]),
                       ("lat_runner_collect", [None, None]), ("lat_runner_set_counter_base", [None, 0]),
                       ("lat_probe_rates", [None, None])]:
        assert getattr(lib, name)(*args) == b.LAT_EINVAL, name
