"""Pins of the oracle's random-number generation (CPU only).

Philox4x32-10 (Salmon et al., SC'11) is checked against an independent implementation run as a
library: cuRAND's host-side PHILOX4_32_10 generator, whose output block B (seed s) is
Philox(counter = (B / 65536 as a 64-bit value in words 0-1, B mod 65536 in word 2, 0), key = s).
The Box-Muller mapping is checked on its exact edge cases and statistically.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from tests import literal_bssmppi as lit


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if path and os.path.exists(path) or (path and not path.startswith("/")):
            try:
                return ctypes.CDLL(path)
            except OSError:
                pass
    return None


def _curand_words(lib, seed, offset, n):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
        return out
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    key = (seed & 0xFFFFFFFF, seed >> 32)
    words = _curand_words(lib, seed, 0, 4 * 300).reshape(-1, 4)
    for b in list(range(40)) + [123, 299]:
        assert (words[b] == oracle.philox([0, 0, b, 0], key)).all(), b
    # counter words 0 and 1 through the generator offset (in 32-bit outputs)
    for c0, c1 in ((1, 0), (9, 0), (0, 1), (7, 3), (0xFFFFFFFF, 0x1234)):
        off = 4 * 65536 * ((c1 << 32) | c0)
        w = _curand_words(lib, seed, off, 8).reshape(-1, 4)
        assert (w[0] == oracle.philox([c0, c1, 0, 0], key)).all()
        assert (w[1] == oracle.philox([c0, c1, 1, 0], key)).all()


def test_philox_literal_python_agrees_on_all_words():
    rng = np.random.default_rng(5)
    for _ in range(200):
        ctr = [int(x) for x in rng.integers(0, 2**32, size=4, dtype=np.uint64)]
        key = [int(x) for x in rng.integers(0, 2**32, size=2, dtype=np.uint64)]
        assert list(oracle.philox(ctr, key)) == lit.philox4x32_10(ctr, key)


def test_philox_word3_is_live():
    key = (17, 99)
    base = oracle.philox([1, 2, 3, 0], key)
    assert not (oracle.philox([1, 2, 3, 1], key) == base).all()
    assert not (oracle.philox([1, 2, 3, 1 << 31], key) == base).all()


def test_box_muller_edges():
    # a = 0xffffffff -> u1 = 1 exactly -> radius 0
    z = oracle.gaussian_pair(0xFFFFFFFF, 12345)
    assert z[0] == 0.0 and abs(z[1]) == 0.0
    # a = 0 -> u1 = 2^-24: radius sqrt(48 ln 2); b = 0 -> angle 0
    z = oracle.gaussian_pair(0, 0)
    assert z[0] == pytest.approx(math.sqrt(48.0 * math.log(2.0)), rel=1e-15)
    assert z[1] == 0.0
    # b = 2^30 -> u2 = 1/4 -> angle pi/2
    z = oracle.gaussian_pair(0, 1 << 30)
    assert abs(z[0]) < 1e-15 and z[1] == pytest.approx(math.sqrt(48.0 * math.log(2.0)), rel=1e-15)
    # low 8 bits are discarded
    assert (oracle.gaussian_pair(0x12345600, 0x9ABCDE00) == oracle.gaussian_pair(0x123456FF, 0x9ABCDEFF)).all()


def test_box_muller_distribution():
    key = (3, 4)
    z = []
    for i in range(20000):
        w = oracle.philox([i, 0, 7, 1 << 28], key)
        z.extend(oracle.gaussian_pair(w[0], w[1]))
        z.extend(oracle.gaussian_pair(w[2], w[3]))
    z = np.asarray(z)
    n = z.size
    assert abs(z.mean()) < 5.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # cos and sin outputs of one pair are uncorrelated
    zz = z.reshape(-1, 2)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 5.0 / math.sqrt(zz.shape[0])
