"""Pins of the oracle's Philox4x32-10 and inverse-CDF sampler.

Philox is pinned to an external implementation: cuRAND's host-side
PHILOX4_32_10 generator (run through its public C API, no GPU needed), whose
output block g is Philox4x32-10 of counter (g div 65536 split into words 0 and 1,
g mod 65536 in word 2, 0) under key = (seed lo, seed hi).  The sampler is pinned
by exact thresholds for dyadic pmfs, boundary uniforms, zero-probability states
and sample frequencies.
"""
import ctypes
import ctypes.util

import numpy as np
import pytest

from oracle import oracle as O


def _curand():
    for name in ("libcurand.so.10", "libcurand.so", ctypes.util.find_library("curand") or ""):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    for p in ("/usr/local/cuda/lib64/libcurand.so",):
        try:
            return ctypes.CDLL(p)
        except OSError:
            pass
    return None


def _curand_host_philox(lib, seed, offset, count):
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(count)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed,offset", [
    (0, 0),
    (0x0123456789ABCDEF, 0),
    (0xFEEDFACE12345, 4 * 7),
    (0xFFFFFFFFFFFFFFFF, 1 << 34),
    (42, (1 << 50) + 4 * 12345),   # counter word 1 non-zero
])
def test_philox_matches_curand_host_generator(seed, offset):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    count = 1 << 20
    out = _curand_host_philox(lib, seed, offset, count)
    rng = np.random.default_rng(seed & 0xFFFF)
    blocks = np.unique(np.concatenate([np.arange(8), np.arange(65530, 65542),
                                       rng.integers(0, count // 4, 300)]))
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in blocks:
        g = offset // 4 + int(b)
        hi = g // 65536
        ctr = [hi & 0xFFFFFFFF, hi >> 32, g % 65536, 0]
        assert np.array_equal(O.philox4x32_10(ctr, key), out[4 * b:4 * b + 4]), (seed, offset, b)


def test_thresholds_dyadic_exact():
    pmf = np.array([[0.25, 0.75],
                    [0.5, 0.5],
                    [0.0, 1.0],
                    [1.0, 0.0]])
    T = O.thresholds(pmf)
    assert T[:, 0].tolist() == [1 << 30, 1 << 31, 0, 1 << 32]


def test_thresholds_multistate_exact():
    pmf = np.array([[0.125, 0.375, 0.0, 0.5], [0.0, 0.0, 0.5, 0.5]])
    T = O.thresholds(pmf)
    assert T.tolist() == [[1 << 29, 1 << 31, 1 << 31], [0, 0, 1 << 31]]


def test_state_boundaries():
    pmf = np.array([[0.25, 0.25, 0.5]])
    T = O.thresholds(pmf)[0]
    assert T.tolist() == [1 << 30, 1 << 31]
    # u below the first threshold -> 0; u equal to a threshold -> the higher state
    assert O.state_from_uniform(0, T) == 0
    assert O.state_from_uniform((1 << 30) - 1, T) == 0
    assert O.state_from_uniform(1 << 30, T) == 1
    assert O.state_from_uniform((1 << 31) - 1, T) == 1
    assert O.state_from_uniform(1 << 31, T) == 2
    assert O.state_from_uniform(0xFFFFFFFF, T) == 2


def test_zero_probability_states_never_drawn():
    # q = 0 for state 0 of comp 0, state 1 of comp 1, state 2 of comp 2 (top)
    pmf = np.array([[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
    T = O.thresholds(pmf)
    for i in range(3):
        for u in (0, 1, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, 0xFFFFFFFE, 0xFFFFFFFF):
            assert O.state_from_uniform(u, T[i]) != [0, 1, 2][i]
    X = O.sample(pmf, seed=3, offset=0, N=20000)
    assert not np.any(X[:, 0] == 0)
    assert not np.any(X[:, 1] == 1)
    assert not np.any(X[:, 2] == 2)


def test_sample_frequencies_match_pmf():
    rng = np.random.default_rng(0)
    pmf = rng.dirichlet(np.ones(4), size=6)
    N = 200000
    X = O.sample(pmf, seed=11, offset=5, N=N)
    for i in range(6):
        freq = np.bincount(X[:, i], minlength=4) / N
        se = np.sqrt(pmf[i] * (1 - pmf[i]) / N)
        assert np.all(np.abs(freq - pmf[i]) <= 5 * se + 1e-12), (i, freq, pmf[i])


def test_sample_offset_is_a_window_of_the_stream():
    pmf = np.array([[0.3, 0.7]] * 9)
    full = O.sample(pmf, seed=99, offset=0, N=64)
    part = O.sample(pmf, seed=99, offset=17, N=20)
    assert np.array_equal(full[17:37], part)


def test_sample_uses_the_documented_counter_layout():
    # component i of sample h is word i%4 of Philox(ctr=(h lo, h hi, i//4, 0), key=(seed lo, seed hi))
    pmf = np.array([[0.5, 0.5]] * 7)
    seed, h = 0x1122334455667788, (1 << 33) + 5
    X = O.sample(pmf, seed=seed, offset=h, N=1)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(7):
        w = O.philox4x32_10([h & 0xFFFFFFFF, h >> 32, i // 4, 0], key)[i % 4]
        assert X[0, i] == (1 if w >= (1 << 31) else 0)
