"""Pins of the oracle's random-number layer against things other than itself.

* Philox4x32-10 (Salmon et al., SC'11) against cuRAND's host-side Philox generator,
  run (not read) through its public C API: that generator keys Philox with the 64-bit
  seed and spreads its counters over 65536 virtual threads (word 2 = thread, words 0-1
  = iteration), which pins counter words 0, 1, 2 and both key words.
* Box-Muller normals, Marsaglia-Tsang gammas and inversion Poisson draws against the
  exact distributions in scipy.stats (KS / chi-square at fixed seeds).
The samplers feed the MBS thermostat (Eqs. 5-7: E_k ~ Gamma(f/2, kT)), the AT+a random
velocities and the phantom particles (Sec. II, Boundary conditions).
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest
from scipy import stats

import oracle


def _curand():
    cands = ["/usr/local/cuda/lib64/libcurand.so", "/usr/local/cuda/lib64/libcurand.so.10",
             ctypes.util.find_library("curand")]
    for c in cands:
        if c and (os.path.exists(c) or not c.startswith("/")):
            try:
                return ctypes.CDLL(c)
            except OSError:
                continue
    return None


def _curand_stream(lib, seed, offset, n):
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


# cuRAND's host Philox emulates 65536 device threads: output block b (4 words) comes
# from counter (b // 65536 as a 64-bit value in words 0-1, b % 65536 in word 2, 0).
_THREADS = 65536


def _ctr_of_block(b):
    it, j = divmod(b, _THREADS)
    return [it & 0xFFFFFFFF, it >> 32, j, 0]


@pytest.mark.parametrize("seed", [0, 1, 3, 0x1234567890ABCDEF, 2**64 - 1])
def test_philox_matches_curand_host(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for first_block in (0, _THREADS - 3, 5 * _THREADS + 17):
        ref = _curand_stream(lib, seed, 4 * first_block, 32).reshape(-1, 4)
        for k in range(ref.shape[0]):
            c = _ctr_of_block(first_block + k)
            assert np.array_equal(oracle.philox(c, key), ref[k]), (seed, c)


def test_philox_counter_carry_matches_curand_host():
    """Word 1 (the step in our keying) is reached through the carry out of word 0."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    seed = 7
    key = [7, 0]
    for it in (2**32 - 1, 2**32, 2**32 + 1, 5 * 2**32 + 3):
        b = it * _THREADS + 11
        ref = _curand_stream(lib, seed, 4 * b, 4)
        c = _ctr_of_block(b)
        assert c[1] == it >> 32
        assert np.array_equal(oracle.philox(c, key), ref), c


def test_philox_high_words_change_output():
    # word 3 (the box index in our keying) stays zero in cuRAND's host stream; words
    # 0-2 are pinned above, so word 3 is the remaining input -- check that it mixes
    base = oracle.philox([1, 2, 3, 4], [5, 6])
    for w in (2, 3):
        for bit in (0, 13, 31):
            c = [1, 2, 3, 4]
            c[w] ^= 1 << bit
            o = oracle.philox(c, [5, 6])
            assert np.all(o != base)


def test_normal_sampler_ks():
    z = oracle.sample_normal(11, 200_000)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)


@pytest.mark.parametrize("shape", [1.0, 1.5, 4.5, 13.5, 73.5])
def test_gamma_sampler_ks(shape):
    x = oracle.sample_gamma(5, shape, 100_000)
    assert stats.kstest(x, stats.gamma(shape).cdf).pvalue > 1e-3
    assert abs(x.mean() - shape) < 5 * np.sqrt(shape / x.size)


@pytest.mark.parametrize("lam", [0.05, 0.7, 3.3, 10.0, 50.0])
def test_poisson_sampler_chi2(lam):
    k = oracle.sample_poisson(9, lam, 100_000)
    kmax = int(lam + 8 * np.sqrt(lam) + 5)
    obs = np.bincount(np.minimum(k, kmax), minlength=kmax + 1).astype(float)
    pmf = stats.poisson(lam).pmf(np.arange(kmax + 1))
    pmf[-1] += stats.poisson(lam).sf(kmax)
    exp = pmf * k.size
    keep = exp > 5
    o2 = np.append(obs[keep], obs[~keep].sum())
    e2 = np.append(exp[keep], exp[~keep].sum())
    if e2[-1] == 0:
        o2, e2 = o2[:-1], e2[:-1]
    assert stats.chisquare(o2, e2 * o2.sum() / e2.sum()).pvalue > 1e-4


def test_shift_is_uniform_and_below_one_cell():
    """Sec. II: the lattice is shifted by a random vector of up to one cell per axis."""
    p = oracle.params(L=16)
    F = oracle.fixed_bits(p)
    S = np.array([oracle.shift(p, s) for s in range(4000)], dtype=np.float64) / 2.0**F
    assert S.min() >= 0 and S.max() < 1
    for ax in range(3):
        assert stats.kstest(S[:, ax], "uniform").pvalue > 1e-3
