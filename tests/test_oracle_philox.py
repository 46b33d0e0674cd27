"""Pin the oracle's Philox4x32-10 to an implementation it shares nothing with.

cuRAND's host-side PHILOX4_32_10 generator runs on the CPU.  With the default
ordering, element 4*b + i of its output stream (after setting the element
offset) is word i of Philox(key = (seed lo, seed hi), counter = (q lo, q hi,
p, 0)) with q = b // 65536 and p = b % 65536; that layout was established by
probing the library and is itself checked here for every block compared.
This reaches arbitrary key words and counter words 0, 1 and 2; counter word 3
is covered by the GPU test against cuRAND's device API.
"""
import ctypes
import ctypes.util
import glob
import os

import numpy as np
import pytest

SUBSEQ = 65536


def _curand():
    cands = []
    for root in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if root:
            cands += sorted(glob.glob(os.path.join(root, "lib64", "libcurand.so*")))
            cands += sorted(glob.glob(os.path.join(root, "targets", "*", "lib", "libcurand.so*")))
    found = ctypes.util.find_library("curand")
    if found:
        cands.append(found)
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    pytest.skip("libcurand not found")


def _host_stream(lib, seed, offset, n):
    gen = ctypes.c_void_p()
    PHILOX = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
        return out
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed,block0,nblocks", [
    (1234, 0, 4 * SUBSEQ + 17),                   # crosses counter-word-0 steps
    (7, 0, 1000),
    (0xDEADBEEFCAFEF00D, 12345 * SUBSEQ - 300, 2000),
    (2025, (0xFFFFFFFF - 3) * SUBSEQ + 60000, 9000),  # counter word 0 wraps into word 1
    ((1 << 63) | 99, ((1 << 44) + 77) * SUBSEQ + 3, 600),  # large counter word 1
    (0xFFFFFFFFFFFFFFFF, ((1 << 45) - 1) * SUBSEQ + SUBSEQ - 5, 50),
])
def test_oracle_philox_matches_curand_host(orc, seed, block0, nblocks):
    lib = _curand()
    ref = _host_stream(lib, seed, 4 * block0, 4 * nblocks).reshape(nblocks, 4)
    b = np.arange(block0, block0 + nblocks, dtype=np.uint64)
    q, p = b // SUBSEQ, b % SUBSEQ
    ctr = np.stack([q & 0xFFFFFFFF, q >> np.uint64(32), p, np.zeros_like(p)], axis=1).astype(np.uint32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    got = orc.philox(ctr, key)
    mism = np.nonzero(np.any(got != ref, axis=1))[0]
    assert mism.size == 0, f"first mismatch at block {block0 + int(mism[0])}"


def test_oracle_philox_is_a_bijection_on_a_sample(orc):
    # Distinct counters under one key give distinct outputs (Philox is a permutation).
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2**32, size=(200000, 4), dtype=np.uint64).astype(np.uint32)
    ctr = np.unique(ctr, axis=0)
    out = orc.philox(ctr, [3, 4])
    assert np.unique(out, axis=0).shape[0] == ctr.shape[0]
