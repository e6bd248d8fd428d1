"""The oracle's Philox4x32-10 against an independent implementation: cuRAND's
host generator (CURAND_RNG_PSEUDO_PHILOX4_32_10, CPU code of NVIDIA's
library; no GPU involved). Salmon et al.'s known-answer vectors pin the
oracle on a few counters (tests/golden/philox4x32_10_kat.txt); this compares
whole streams.

Mapping (probed, then fixed here): with seed s, block i of the generator's
output (words 4i..4i+3) is Philox4x32-10 under key (lo32(s), hi32(s)) of
counter (i >> 16, 0, i & 0xffff, 0) -- 65 536 subsequences in the third
counter word, each advancing in the first; an offset of 4k words starts the
output at block k."""
import ctypes as C
import os

import numpy as np
import pytest

import oracle as O

PHILOX4_32_10 = 161   # curandRngType_t


def _curand():
    names = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcurand.so"),
             "libcurand.so", "libcurand.so.10"]
    for n in names:
        try:
            return C.CDLL(n)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def _stream(L, seed: int, n_words: int, offset: int = 0) -> np.ndarray:
    gen = C.c_void_p()
    assert L.curandCreateGeneratorHost(C.byref(gen), PHILOX4_32_10) == 0
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
        if offset:
            assert L.curandSetGeneratorOffset(gen, C.c_ulonglong(offset)) == 0
        out = np.zeros(n_words, np.uint32)
        assert L.curandGenerate(gen, out.ctypes.data_as(C.c_void_p), C.c_size_t(n_words)) == 0
    finally:
        L.curandDestroyGenerator(gen)
    return out


def _counter(i: int):
    return (i >> 16, 0, i & 0xFFFF, 0)


def _oracle_block(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    O.lib().or_philox4x32_10(c, k, o)
    return list(o)


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_oracle_philox_equals_curand_stream(seed):
    L = _curand()
    n_blocks = 70_000   # past the first 65 536-block round
    ref = _stream(L, seed, 4 * n_blocks).reshape(n_blocks, 4)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    got = np.array([_oracle_block(_counter(i), key) for i in range(n_blocks)], np.uint32)
    np.testing.assert_array_equal(got, ref)


def test_oracle_philox_equals_curand_with_offset():
    """The generator's offset (4k words) starts the stream at block k, whose
    counter the oracle must turn into the same words."""
    L = _curand()
    seed = 0x0BADC0DE12345678
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for k in (1, 4097, 65_535, 2**20 + 3, 2**31 + 5):
        ref = _stream(L, seed, 8, offset=4 * k).reshape(2, 4)
        got = np.array([_oracle_block(_counter(k + j), key) for j in range(2)], np.uint32)
        np.testing.assert_array_equal(got, ref)
