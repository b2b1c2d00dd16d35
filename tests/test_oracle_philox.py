"""Pins of the oracle's counter-based uniforms (Philox4x32-10).

The oracle's Philox is pinned against (1) cuRAND's host-side Philox4_32_10
generator, an independent implementation called as a library on the CPU,
whose k-th block of four outputs for seed s equals Philox(counter = (0, 0, k,
0), key = (s_lo, s_hi)); (2) a numpy implementation written separately from
the SC'11 description; and (3) statistical properties that a mistake in the
round function or the word mapping would break (uniformity, independence
across counter words, avalanche).
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

from tests import philox_ref


def _curand():
    cands = ["/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")]
    for c in cands:
        if c and os.path.exists(c):
            try:
                return ctypes.CDLL(c)
            except OSError:
                pass
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(oracle_mod, seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        blocks = 512
        out = np.zeros(4 * blocks, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    mine = np.concatenate([oracle_mod.philox4x32_10([0, 0, k, 0], key) for k in range(blocks)])
    np.testing.assert_array_equal(mine, out)


def test_philox_matches_independent_numpy_implementation(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(200):
        ctr = rng.integers(0, 2**32, size=4, dtype=np.uint64)
        key = rng.integers(0, 2**32, size=2, dtype=np.uint64)
        ref = philox_ref.philox(*ctr, *key)
        got = oracle_mod.philox4x32_10(ctr.astype(np.uint32), key.astype(np.uint32))
        np.testing.assert_array_equal(got, np.array([r.item() for r in ref], dtype=np.uint32))


def test_uniform_word_and_counter_mapping(oracle_mod):
    """u = top 24 bits of word (rep mod 4) of Philox((node, step, rep//4, 0), seed)."""
    seed = 0xDEADBEEFCAFEF00D
    for rep in (0, 1, 2, 3, 4, 7, 13):
        for step in (0, 1, 999):
            for node in (0, 5, 123456):
                w = oracle_mod.philox4x32_10([node, step, rep // 4, 0], [seed & 0xFFFFFFFF, seed >> 32])
                expect = float(w[rep % 4] >> 8) / 2**24
                assert oracle_mod.uniform(seed, rep, step, node) == expect
    # exactly representable in float32 and inside [0, 1)
    u = philox_ref.uniforms(1, 0, 3, np.arange(100000))
    assert (u >= 0).all() and (u < 1).all()
    assert (u.astype(np.float32).astype(np.float64) == u).all()


def test_uniforms_are_uniform_and_independent():
    """Chi-square over 64 bins, lag correlation across nodes and steps."""
    n = 1_000_000
    u = philox_ref.uniforms(1, 0, 0, np.arange(n))
    hist = np.bincount((u * 64).astype(np.int64), minlength=64)
    chi2 = (((hist - n / 64) ** 2) / (n / 64)).sum()
    assert chi2 < 120.0          # 63 dof: p ~ 1e-5 threshold
    v = philox_ref.uniforms(1, 0, 1, np.arange(n))       # next step, same nodes
    w = philox_ref.uniforms(1, 1, 0, np.arange(n))       # next replicate
    for other in (v, w, np.roll(u, 1)):
        r = np.corrcoef(u, other)[0, 1]
        assert abs(r) < 5.0 / np.sqrt(n)
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)


def test_avalanche_on_counter_words(oracle_mod):
    rng = np.random.default_rng(3)
    flips = []
    for _ in range(300):
        ctr = rng.integers(0, 2**32, size=4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, size=2, dtype=np.uint64).astype(np.uint32)
        word = rng.integers(0, 4)
        bit = rng.integers(0, 32)
        c2 = ctr.copy()
        c2[word] ^= np.uint32(1 << int(bit))
        a = oracle_mod.philox4x32_10(ctr, key)
        b = oracle_mod.philox4x32_10(c2, key)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert 60 < np.mean(flips) < 68      # half of 128 bits
