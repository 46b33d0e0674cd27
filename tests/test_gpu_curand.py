"""Pin the oracle's Philox on every counter word against cuRAND's device API
(the generator the paper uses, section 3.2), including counter word 3 and
the sweep index 0xFFFFFFFF that the host-side generator cannot reach."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _ref_lib():
    from paper_2502_18624_gb300 import _build
    src = os.path.join(HERE, "cuda", "curand_ref.cu")
    out_dir = os.path.join(HERE, "lib")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libcurand_ref.so")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        subprocess.check_call([_build.nvcc(), "-shared", "-Xcompiler", "-fPIC", "-O2", *_build.ARCH,
                               src, "-o", so])
    lib = ctypes.CDLL(so)
    lib.curand_philox_ref.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_ulonglong, ctypes.c_void_p]
    lib.curand_philox_ref.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("seed", [1234, 7, 99, 0xFEDCBA9876543210, 2**64 - 1])
def test_oracle_philox_matches_curand_device_api(gpu, orc, seed):
    lib = _ref_lib()
    rng = np.random.default_rng(seed & 0xFFFF)
    n = 50000
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[: n // 4, 2] = 0xFFFFFFFF            # the quench's sweep index
    ctr[: n // 4, 3] = 0
    ctr[n // 4: n // 2, 3] = rng.integers(0, 2, size=n // 4)   # colours
    ctr[n // 2: 3 * n // 4, 1] = 0
    ctr = np.ascontiguousarray(ctr)
    out = np.zeros_like(ctr)
    assert lib.curand_philox_ref(ctr.ctypes.data_as(ctypes.c_void_p), n, seed,
                                 out.ctypes.data_as(ctypes.c_void_p)) == 0
    got = orc.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])
    assert np.array_equal(got, out)
