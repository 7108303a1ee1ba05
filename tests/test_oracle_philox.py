"""Pins of the oracle's Philox4x32-10 and uniform mapping against something
other than the oracle: NVIDIA's cuRAND host-side Philox4_32_10 generator
(an independent implementation of the same published generator, run as a
library on the CPU) and exact properties of the (0,1) mapping."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    cands = ['/usr/local/cuda/lib64/libcurand.so', ctypes.util.find_library('curand')]
    for c in cands:
        if c and (os.path.exists(c) or not c.startswith('/')):
            try:
                return ctypes.CDLL(c)
            except OSError:
                pass
    pytest.skip('libcurand not available')


def _curand_blocks(seed, n_blocks, offset_blocks=0):
    cr = _curand()
    g = ctypes.c_void_p()
    if cr.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip('cuRAND host generator unavailable')
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        if offset_blocks:
            assert cr.curandSetGeneratorOffset(g, ctypes.c_ulonglong(4 * offset_blocks)) == 0
        out = np.zeros(4 * n_blocks, np.uint32)
        assert cr.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.c_size_t(out.size)) == 0
    finally:
        cr.curandDestroyGenerator(g)
    return out.reshape(-1, 4)


# cuRAND's default host ordering emits block i of seed s as
# Philox4x32-10(counter = (i // 65536 as 64 bits in words 0-1, i % 65536, 0),
#               key = (s low word, s high word)).
def _ctr(i):
    q, r = divmod(i, 65536)
    return [q & 0xFFFFFFFF, q >> 32, r, 0]


@pytest.mark.parametrize('seed', [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_word2_and_key(orc, seed):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    blocks = _curand_blocks(seed, 300)
    for i in range(300):
        assert orc.philox(_ctr(i), key).tolist() == blocks[i].tolist(), i


@pytest.mark.parametrize('off', [65536 * 3 + 11, 65536 * (1 << 32) + 7, 65536 * 0x12345678ABC + 65535])
def test_philox_matches_curand_words0_1(orc, off):
    seed = 0xDEADBEEF12345
    key = [seed & 0xFFFFFFFF, seed >> 32]
    blocks = _curand_blocks(seed, 8, offset_blocks=off)
    for i in range(8):
        assert orc.philox(_ctr(off + i), key).tolist() == blocks[i].tolist()


def test_u01_is_exact_and_open(orc):
    assert orc.u01(0, 0) == 2.0 ** -53
    assert orc.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert orc.u01(0x80000000, 0) == 0.5 + 2.0 ** -53
    # the low 12 bits are dropped, the next bit counts
    assert orc.u01(0, 0xFFF) == orc.u01(0, 0)
    assert orc.u01(0, 0x1000) == 3 * 2.0 ** -53


def test_u01_uniformity(orc):
    # 40k uniforms from consecutive Philox blocks: a 20-bin chi-square and
    # the Kolmogorov-Smirnov statistic stay far inside their 99.9% bounds.
    from scipy import stats
    u = []
    for e in range(20000):
        w = orc.philox([e, 5, 0, 0], [123, 456])
        u.append(orc.u01(int(w[0]), int(w[1])))
        u.append(orc.u01(int(w[2]), int(w[3])))
    u = np.asarray(u)
    assert u.min() > 0 and u.max() < 1
    counts = np.histogram(u, bins=20, range=(0, 1))[0]
    chi2 = ((counts - u.size / 20) ** 2 / (u.size / 20)).sum()
    assert chi2 < stats.chi2.ppf(0.999, 19)
    assert stats.kstest(u, 'uniform').pvalue > 1e-3
