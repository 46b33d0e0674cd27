"""lat_correlation_static, the correlation entry point that allocates nothing.

It is for callers that cannot allocate device memory when they measure (a
library inside another framework whose caching allocator owns the GPU, or a
serving loop where cudaMalloc would synchronise the device); its scratch is a
fixed device array inside the library.  These tests call it through the C
ABI and check that it returns exactly what lat_correlation returns for the
same lattice, on consecutive calls that reuse the shared scratch (with
distances that take both of its kernel paths, the near-distance kernel for
rmax <= 32 and the window kernels beyond, and rmax = 0), and exactly what
the CPU oracle computes from the lattice's spins.  The file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2502_18624_gb300 import binding as b

pytestmark = pytest.mark.gpu

STATIC_RMAX = 4096


def _static_fn():
    f = b.load().lat_correlation_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    return f


def _static_corr(lat, rmax):
    cx = np.full(rmax + 1, -7, dtype=np.int64)
    cy = np.full(rmax + 1, -7, dtype=np.int64)
    rc = _static_fn()(lat.model, lat.L, lat.buffer.data_ptr(), rmax, cx.ctypes.data_as(ctypes.c_void_p),
                      cy.ctypes.data_as(ctypes.c_void_p), lat.stream.cuda_stream)
    return rc, cx, cy


@pytest.mark.parametrize("model,L,T,Delta", [(0, 1024, b.TC_ISING, 0.0), (1, 512, 1.398, 1.0)])
def test_static_correlation_matches_handle_path_on_consecutive_calls(gpu, model, L, T, Delta):
    lat = b.Lattice(model, L, T, 2024 + model, Delta=Delta)
    # each call reuses scratch that held a longer result before it
    for nsweeps, rmax in [(3, L // 2), (5, 37), (1, 32), (2, 1), (1, 0), (2, 33)]:
        lat.sweep(nsweeps, record=False)
        ref_x, ref_y = lat.correlation(rmax)
        rc, cx, cy = _static_corr(lat, rmax)
        assert rc == b.LAT_OK
        assert np.array_equal(cx, ref_x) and np.array_equal(cy, ref_y)
    lat.close()


def test_static_correlation_two_lattices_in_a_row(gpu):
    a = b.Lattice(0, 256, b.TC_ISING, 1)
    c = b.Lattice(0, 256, 1.0, 2)
    a.sweep(4, record=False)
    c.sweep(4, record=False)
    for lat in (a, c):
        rc, cx, cy = _static_corr(lat, 128)
        rx, ry = lat.correlation(128)
        assert rc == b.LAT_OK and np.array_equal(cx, rx) and np.array_equal(cy, ry)
    a.close(); c.close()


def test_static_correlation_rejects_sizes_beyond_its_scratch(gpu):
    lat = b.Lattice(0, 16384, b.TC_ISING, 3)
    rc, _, _ = _static_corr(lat, STATIC_RMAX + 1)
    assert rc == b.LAT_EINVAL
    rc, cx, cy = _static_corr(lat, STATIC_RMAX)
    rx, ry = lat.correlation(STATIC_RMAX)
    assert rc == b.LAT_OK and np.array_equal(cx, rx) and np.array_equal(cy, ry)
    small = b.Lattice(0, 128, b.TC_ISING, 3)
    assert _static_corr(small, 65)[0] == b.LAT_EINVAL   # beyond L/2
    lat.close(); small.close()


@pytest.mark.parametrize("model,L,T,Delta", [(0, 256, b.TC_ISING, 0.0), (1, 192, 1.398, 1.0)])
def test_static_correlation_equals_the_oracle(gpu, orc, model, L, T, Delta):
    lat = b.Lattice(model, L, T, 4040 + model, Delta=Delta)
    for nsweeps, rmax in [(6, L // 2), (3, 32), (2, 0), (4, 77)]:
        lat.sweep(nsweeps, record=False)
        s = lat.spins()
        ox, oy = orc.correlation(s, rmax)
        for _ in range(2):                      # two calls in a row on the same lattice
            rc, cx, cy = _static_corr(lat, rmax)
            assert rc == b.LAT_OK
            assert np.array_equal(cx, ox) and np.array_equal(cy, oy)
    lat.close()
