"""Pin the oracle's canonical lattice hash (or_hash, or_hash_words).

The hash compares two lattices without moving them: H = sum over canonical
words i of mix(i XOR word_i) mod 2^64, mix the SplitMix64 finaliser
(Steele, Lea and Flood, OOPSLA 2014).  What makes such a comparison
meaningful, and what each test below fixes:

* every change of one bit of one canonical word changes H (mix is a
  bijection, so one changed term always changes the sum) -- exhaustively on
  a 64 x 64 Ising lattice and on both planes of a 64 x 64 Blume-Capel one;
* H depends on where each word sits: exchanging two unequal words changes
  it (the i XOR word_i term), for every pair of words of a small lattice;
* the two Blume-Capel planes are not interchangeable;
* mix avalanches: flipping any one input bit flips each output bit with
  probability close to 1/2 (the property a finaliser exists for; a mixer
  with a step missing has input bits that never reach some output bits);
* or_hash is or_hash_words of or_pack, whose layout numpy.packbits pins
  (tests/test_oracle_measure.py).
"""
import numpy as np
import pytest


def _random_state(model, L, seed):
    rng = np.random.default_rng(seed)
    vals = np.array([-1, 1] if model == 0 else [-1, 0, 1], dtype=np.int8)
    return vals[rng.integers(0, vals.size, size=(L, L))]


@pytest.mark.parametrize("model", [0, 1])
def test_every_single_bit_change_changes_the_hash(orc, model):
    s = _random_state(model, 64, 40 + model)
    w = orc.pack(model, s)
    h0 = orc.hash_words(w)
    assert h0 == orc.lattice_hash(model, s)
    for i in range(w.size):               # Ising: 64 words; Blume-Capel: 128 (both planes)
        for b in range(64):
            t = w.copy()
            t[i] ^= np.uint64(1) << np.uint64(b)
            assert orc.hash_words(t) != h0, (i, b)


@pytest.mark.parametrize("model", [0, 1])
def test_every_single_site_change_changes_the_lattice_hash(orc, model):
    L = 64
    s = _random_state(model, L, 50 + model)
    h0 = orc.lattice_hash(model, s)
    vals = (-1, 1) if model == 0 else (-1, 0, 1)
    for y in range(0, L, 7):
        for x in range(L):
            for v in vals:
                if v == s[y, x]:
                    continue
                t = s.copy()
                t[y, x] = v
                assert orc.lattice_hash(model, t) != h0, (y, x, v)


@pytest.mark.parametrize("model", [0, 1])
def test_exchanging_two_unequal_words_changes_the_hash(orc, model):
    s = _random_state(model, 64, 60 + model)
    w = orc.pack(model, s)
    h0 = orc.hash_words(w)
    n = w.size
    for i in range(n):
        for j in range(i + 1, n):
            if w[i] == w[j]:
                continue
            t = w.copy()
            t[i], t[j] = w[j], w[i]
            assert orc.hash_words(t) != h0, (i, j)


def test_blume_capel_planes_are_not_interchangeable(orc):
    L = 64
    n = L * L // 64
    for seed in range(5):
        s = _random_state(1, L, 70 + seed)
        w = orc.pack(1, s)
        swapped = np.concatenate([w[n:], w[:n]])
        assert orc.hash_words(swapped) != orc.hash_words(w)
        # the same lattice read as the other plane order is a different lattice
        neg = (-s).astype(np.int8)
        assert orc.lattice_hash(1, neg) != orc.lattice_hash(1, s)


def test_equal_lattices_hash_equal_and_order_of_words_is_fixed(orc):
    s = _random_state(0, 128, 80)
    assert orc.lattice_hash(0, s) == orc.lattice_hash(0, s.copy())
    w = orc.pack(0, s)
    # word i enters as mix(i ^ w_i): hashing the words one at a time at their
    # positions and adding the single-word hashes of (i ^ w_i) gives H
    total = 0
    for i in range(w.size):
        total = (total + orc.hash_words(np.array([np.uint64(i) ^ w[i]], dtype=np.uint64))) % (1 << 64)
    assert total == orc.hash_words(w)


def test_mixer_avalanche(orc):
    """Flip each of the 64 input bits of 2048 random words: every output bit
    must flip with frequency in [0.40, 0.60] (expected 0.5, sd 0.011), and
    the mean number of flipped output bits must be within 32 +- 0.5."""
    rng = np.random.default_rng(2024)
    xs = rng.integers(0, 2**63, size=2048, dtype=np.int64).astype(np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=2048).astype(np.uint64)
    mix = lambda z: orc.hash_words(np.array([z], dtype=np.uint64))   # word 0: mix(0 ^ z)
    base = np.array([mix(z) for z in xs], dtype=np.uint64)
    bits = np.arange(64, dtype=np.uint64)
    for j in range(64):
        flipped = np.array([mix(z ^ (np.uint64(1) << np.uint64(j))) for z in xs], dtype=np.uint64)
        diff = base ^ flipped
        per_bit = ((diff[:, None] >> bits[None, :]) & np.uint64(1)).astype(np.float64).mean(axis=0)
        assert per_bit.min() >= 0.40 and per_bit.max() <= 0.60, (j, per_bit.min(), per_bit.max())
        assert abs(per_bit.sum() - 32.0) < 0.5, (j, per_bit.sum())
