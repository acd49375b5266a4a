"""Pins for the oracle's uniforms: Philox4x32-10 and the word -> U(0,1) map.

The oracle's generator is checked against cuRAND's host-side Philox4x32-10 generator, a library
that is run here (never copied). Its stream places output block g at counter
(low 64 bits = g div 65536, subsequence = g mod 65536) under key = seed, which lets the test reach
counters with every 64-bit low half and 16-bit subsequences.
"""

import ctypes as C
import os

import numpy as np
import pytest

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return C.CDLL(path)
        except OSError:
            continue
    pytest.skip("libcurand not found")


def _curand_host_stream(cr, seed: int, block0: int, n_blocks: int) -> np.ndarray:
    g = C.c_void_p()
    assert cr.curandCreateGeneratorHost(C.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(g, C.c_ulonglong(seed)) == 0
        assert cr.curandSetGeneratorOffset(g, C.c_ulonglong(4 * block0)) == 0
        out = np.zeros(4 * n_blocks, dtype=np.uint32)
        assert cr.curandGenerate(g, out.ctypes.data_as(C.c_void_p), C.c_size_t(out.size)) == 0
    finally:
        cr.curandDestroyGenerator(g)
    return out.reshape(n_blocks, 4)


@pytest.mark.parametrize("seed", [42, 0, 7, 0xFEDCBA9876543210, 0x00000001FFFFFFFF])
@pytest.mark.parametrize("block0", [0, 65536 * 5 + 7, 65536 * (1 << 32) + 3,
                                    65536 * ((3 << 32) + 11) + 60000, 123456789012345])
def test_philox_matches_curand_host_generator(oracle, seed, block0):
    cr = _curand()
    n = 96
    ref = _curand_host_stream(cr, seed, block0, n)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in range(n):
        g = block0 + b
        hi, sub = g // 65536, g % 65536
        ctr = [hi & 0xFFFFFFFF, (hi >> 32) & 0xFFFFFFFF, sub, 0]
        got = oracle.philox4x32_10(ctr, key)
        assert (got == ref[b]).all(), (seed, g, got, ref[b])


def test_philox_is_a_bijection_on_a_sample(oracle):
    # Distinct counters under one key give distinct outputs (a permutation of 2^128).
    seen = set()
    for c in range(4096):
        out = tuple(oracle.philox4x32_10([c, 0, c * 7 % 13, 0], [42, 0]))
        seen.add(out)
    assert len(seen) == 4096


def test_uniform_map_exhaustive(oracle):
    j = np.arange(1 << 23, dtype=np.uint64)
    low = (np.arange(1 << 23, dtype=np.uint64) * 2654435761) & 0x1FF  # arbitrary low 9 bits
    words = ((j << 9) | low).astype(np.uint32)
    u = oracle.uniform_n(words)
    # every value is exactly representable in binary32 and lies strictly inside (0, 1)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert u.min() > 0.0 and u.max() < 1.0
    assert u.min() == 2.0 ** -24 and u.max() == 1.0 - 2.0 ** -24
    # strictly increasing in the upper 23 bits, independent of the low 9
    assert np.all(np.diff(u) > 0)
    # symmetric grid: u(j) + u(2^23 - 1 - j) == 1 exactly, so 1 - u is exact too
    assert np.array_equal(u + u[::-1], np.ones_like(u))
    # equal spacing 2^-23, mean 1/2
    assert np.all(np.diff(u) == 2.0 ** -23)


def test_su_uniform_keying(oracle):
    # (trial, event position, ELT handle) each change the draw; the same key repeats it.
    base = oracle.su_uniform(42, 5, 3, 2)
    assert oracle.su_uniform(42, 5, 3, 2) == base
    others = {oracle.su_uniform(42, 6, 3, 2), oracle.su_uniform(42, 5, 4, 2),
              oracle.su_uniform(42, 5, 3, 1), oracle.su_uniform(42, 5, 3, 6),
              oracle.su_uniform(43, 5, 3, 2), oracle.su_uniform(42, 5 + (1 << 32), 3, 2)}
    assert base not in others and len(others) == 6
    # ELT handles 4q..4q+3 share one Philox block: word elt mod 4 of counter (k, i, q, 0)
    words = oracle.philox4x32_10([3, 5, 1, 0], [42, 0])
    for e in range(4, 8):
        assert oracle.su_uniform(42, 5, 3, e) == oracle.uniform(int(words[e & 3]))


def test_su_uniform_is_uniform(oracle):
    # 40,000 draws: Kolmogorov-Smirnov distance well inside the 0.1% critical value.
    u = np.array([oracle.su_uniform(42, i, k, 0) for i in range(200) for k in range(200)])
    u.sort()
    n = u.size
    ecdf_hi = np.arange(1, n + 1) / n
    ecdf_lo = np.arange(0, n) / n
    d = max(np.max(ecdf_hi - u), np.max(u - ecdf_lo))
    assert d < 1.95 / np.sqrt(n)
