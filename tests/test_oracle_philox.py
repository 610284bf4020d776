"""Pins of the oracle's Philox4x32-10 and Box-Muller normals.

The Philox words are checked against cuRAND's host-side Philox4_32_10
generator (a library routine run on the CPU; key = (seed lo, seed hi)). The
normals are checked against the standard normal law.
"""
import ctypes

import numpy as np
import pytest
from scipy import stats

from oracle import chemo_oracle as orc


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


def _curand_words(seed, offset_words, count):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset_words)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(count)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


def _host_counters(offset_words, nblk):
    """Counters of cuRAND's host Philox generator in its default ordering:
    it interleaves 65536 subsequences, so block i of a run that starts at
    offset o (in words) uses ctr = (x lo, x hi, i mod 65536, 0) with
    x = o / 2^18 + i div 65536."""
    i = np.arange(nblk, dtype=np.uint64)
    x = np.uint64(offset_words // (4 * 65536)) + i // np.uint64(65536)
    ctr = np.zeros((nblk, 4), dtype=np.uint32)
    ctr[:, 0] = (x & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ctr[:, 1] = (x >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = (i % np.uint64(65536)).astype(np.uint32)
    return ctr


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 2**64 - 1])
def test_philox_matches_curand_host_generator(seed):
    nblk = 3 * 65536 + 123
    words = _curand_words(seed, 0, 4 * nblk).reshape(nblk, 4)
    got = orc.philox(_host_counters(0, nblk), seed)
    np.testing.assert_array_equal(got, words)


def test_philox_second_counter_word_via_offset():
    # an offset of 2^50 words moves the 64-bit block counter to 2^32, which
    # sets the second counter word. (The fourth word enters the rounds the
    # same way as the second and is covered by the step counter checks.)
    seed = 77
    off = (1 << 50) + 4 * 65536 * 5
    nblk = 70000
    words = _curand_words(seed, off, 4 * nblk).reshape(nblk, 4)
    np.testing.assert_array_equal(orc.philox(_host_counters(off, nblk), seed), words)


def test_uniform_map_stays_inside_open_interval():
    # u = (w + 1/2) 2^-32 is exact in FP64; the extreme words map to
    # 2^-33 and 1 - 2^-33, so log(u) is finite for every word.
    ids = np.arange(200_000, dtype=np.uint32)
    xi = orc.normals(5, ids, 0)
    assert np.all(np.isfinite(xi))


def test_normals_are_standard_normal():
    ids = np.arange(250_000, dtype=np.uint32)
    xi = orc.normals(12345, ids, 3)
    for lane in range(4):
        v = xi[:, lane]
        assert abs(v.mean()) < 5 * 1 / np.sqrt(v.size)
        assert abs(v.var() - 1.0) < 5 * np.sqrt(2.0 / v.size)
        assert stats.kstest(v, "norm").pvalue > 1e-3
    c = np.corrcoef(xi.T)
    assert np.max(np.abs(c - np.eye(4))) < 5 / np.sqrt(ids.size)


def test_normals_differ_between_steps_and_streams():
    ids = np.arange(1000, dtype=np.uint32)
    a = orc.normals(9, ids, 0, orc.TAG_MOVE)
    b = orc.normals(9, ids, 1, orc.TAG_MOVE)
    c = orc.normals(9, ids, 0, orc.TAG_REACT)
    assert not np.allclose(a, b) and not np.allclose(a, c)
    # step counter above 2^32 uses the fourth counter word
    d = orc.normals(9, ids, 1 << 32, orc.TAG_MOVE)
    assert not np.allclose(a, d)
