"""Parity of the section 3.3 correlation protocol on the GPU (through the C ABI).

The downsampled sums are integer work: bit-exact against the oracle.  Small
lattices cover every R in 1..64 (both y paths: the compact source-column copy
for R >= 16 and direct lattice reads below), ragged source rows (L/R not a
multiple of 64), repeats and arbitrary order in the distance list, and both
models.  At full size (L = 2^17 Ising, 2^16 Blume-Capel) the lattice is a
periodic tiling of a random tile, so every sum is (L/P)^2 times the oracle's
sum on the tile; the same tiling checks the bench's all-sites C(r <= 1024)
element by element at full size, and a swept full-size lattice checks R = 1
against the all-sites kernel.
"""
import numpy as np
import pytest

from paper_2502_18624_gb300 import binding as b

pytestmark = pytest.mark.gpu

TC = b.TC_ISING


def _lattice(model, L, seed=11, sweeps=3):
    T, Delta = (TC, 0.0) if model == 0 else (1.398, 1.0)
    lat = b.Lattice(model, L, T, seed, Delta=Delta)
    lat.sweep(sweeps, record=False)
    return lat


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("L,R", [(64, 1), (64, 16), (64, 64), (128, 2), (128, 16), (192, 4), (192, 16), (256, 8),
                                 (256, 32), (320, 64), (512, 16), (1088, 16), (1024, 1), (2048, 16)])
def test_sampled_parity(gpu, orc, model, L, R):
    lat = _lattice(model, L)
    s = lat.spins()
    rng = np.random.default_rng(L + R)
    rl = np.concatenate([np.arange(0, L // 2 + 1) if L <= 512 else np.arange(0, 70),
                         rng.integers(0, L // 2 + 1, 40), [L // 2, 0, 1, 1]]).astype(np.uint32)
    rng.shuffle(rl)
    cx, cy = lat.correlation_sampled(R, rl)
    ox, oy = orc.correlation_sampled(s, R, rl)
    assert np.array_equal(cx, ox) and np.array_equal(cy, oy)
    lat.close()


@pytest.mark.parametrize("model", [0, 1])
def test_sampled_R1_equals_all_sites(gpu, model):
    lat = _lattice(model, 4096, sweeps=5)
    fx, fy = lat.correlation(300)
    cx, cy = lat.correlation_sampled(1, np.arange(301))
    assert np.array_equal(cx, fx) and np.array_equal(cy, fy)
    lat.close()


@pytest.mark.parametrize("model,L", [(0, 256), (0, 1024), (1, 1024), (0, 2048), (1, 576)])
@pytest.mark.parametrize("t", [1, 1000, 10**6])
def test_protocol_parity(gpu, orc, model, L, t):
    R = 16
    lat = _lattice(model, L)
    s = lat.spins()
    out = lat.correlation_protocol(t, R)
    rfull = min(2 * R, L // 2)
    d = orc.protocol_distances(L, t, R)
    assert out["r"].tolist() == list(range(rfull + 1)) + d.tolist()
    fx, fy = orc.correlation(s, rfull)
    sx, sy = orc.correlation_sampled(s, R, d)
    assert np.array_equal(out["cx"], np.concatenate([fx, sx]))
    assert np.array_equal(out["cy"], np.concatenate([fy, sy]))
    assert out["nsrc"].tolist() == [L * L] * (rfull + 1) + [(L // R) ** 2] * d.size
    lat.close()


def test_sampled_rejects_bad_arguments(gpu):
    lat = _lattice(0, 128, sweeps=0)
    for R in (0, 3, 128):
        with pytest.raises(b.LatError) as e:
            lat.correlation_sampled(R, [1])
        assert e.value.code == b.LAT_EINVAL
    with pytest.raises(b.LatError):
        lat.correlation_sampled(16, [65])  # > L/2
    assert lat.correlation_sampled(16, [])[0].size == 0
    lat.close()


def _tiled_state(model, L, tile):
    """Packed device state of the lattice that repeats `tile` (P x P) in both axes."""
    P = tile.shape[0]
    big_row = np.tile(tile, (1, L // P))              # P x L int8
    bits = lambda m: np.packbits(m.astype(np.uint8), axis=1, bitorder="little").view(np.uint64)
    if model == 0:
        rows = bits(big_row == 1)                     # P x W
    else:
        n, g = bits(big_row != 0), bits(big_row == -1)
        rows = np.empty((P, 2 * n.shape[1]), dtype=np.uint64)
        rows[:, 0::2], rows[:, 1::2] = n, g
    return np.ascontiguousarray(np.tile(rows, (L // P, 1)).reshape(-1))


@pytest.mark.parametrize("model,L", [(0, 1 << 17), (1, 1 << 16)])
def test_full_size_tiled_lattice(gpu, orc, model, L):
    """Every sum on a periodic tiling of a P x P tile is (L/P)^2 times the tile's sum."""
    P, R, t = 256, 16, 1000
    rng = np.random.default_rng(5)
    vals = np.array([-1, 1] if model == 0 else [-1, 0, 1], dtype=np.int8)
    tile = vals[rng.integers(0, vals.size, size=(P, P))]
    T, Delta = (TC, 0.0) if model == 0 else (1.398, 1.0)
    lat = b.Lattice(model, L, T, 3, Delta=Delta)
    lat.set_state(_tiled_state(model, L, tile))
    k = (L // P) ** 2
    out = lat.correlation_protocol(t, R)
    d = orc.protocol_distances(L, t, R)
    assert out["r"].tolist() == list(range(2 * R + 1)) + d.tolist()
    fx, fy = orc.correlation(tile, 2 * R)
    sx, sy = orc.correlation_sampled(tile, R, d % P)
    assert np.array_equal(out["cx"], k * np.concatenate([fx, sx]))
    assert np.array_equal(out["cy"], k * np.concatenate([fy, sy]))
    # direct y path (R < 16) at full size
    rl = np.array([0, 1, 5, 33, 255, 256, 4097, L // 2], dtype=np.uint32)
    cx, cy = lat.correlation_sampled(8, rl)
    ox, oy = orc.correlation_sampled(tile, 8, rl % P)
    assert np.array_equal(cx, k * ox) and np.array_equal(cy, k * oy)
    lat.close()


def test_full_size_swept_R1_equals_all_sites(gpu):
    L = 1 << 17
    lat = b.Lattice(0, L, TC, 7)
    lat.sweep(2, record=False)
    fx, fy = lat.correlation(40)
    cx, cy = lat.correlation_sampled(1, np.arange(41))
    assert np.array_equal(cx, fx) and np.array_equal(cy, fy)
    M, B, Q, _ = lat.measure()
    assert cx[1] + cy[1] == B
    lat.close()


@pytest.mark.parametrize("model,L,rmax", [(0, 1 << 17, 1024), (1, 1 << 16, 512)])
def test_full_size_all_sites_correlation_tiled(gpu, orc, model, L, rmax):
    """The bench's C(r) from every site, at its full size and rmax, element by
    element: on a periodic tiling of a P x P tile every sum is (L/P)^2 times
    the oracle's sum on the tile (distances taken on the tile's torus)."""
    P = 256
    rng = np.random.default_rng(9 + model)
    vals = np.array([-1, 1] if model == 0 else [-1, 0, 1], dtype=np.int8)
    tile = vals[rng.integers(0, vals.size, size=(P, P))]
    T, Delta = (TC, 0.0) if model == 0 else (1.398, 1.0)
    lat = b.Lattice(model, L, T, 3, Delta=Delta)
    lat.set_state(_tiled_state(model, L, tile))
    cx, cy = lat.correlation(rmax)
    ox, oy = orc.correlation(tile, rmax)
    k = (L // P) ** 2
    assert np.array_equal(cx, k * ox) and np.array_equal(cy, k * oy)
    # the separate (M, B, Q) reduction and the spin counts scale the same way
    M, B, Q = orc.measure(model, tile)
    assert lat.measure()[:3] == (k * M, k * B, k * Q)
    assert lat.spin_counts().tolist() == [k * int((tile == v).sum()) for v in (-1, 0, 1)] + [0]
    assert np.array_equal(lat.sd_hist(), k * orc.sd_hist(tile))
    lat.close()
