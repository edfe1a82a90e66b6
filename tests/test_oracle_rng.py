"""Pins for the oracle's random numbers (Philox4x32-10, Salmon et al. 2011).

The reference for the generator itself is an independent library run: cuRAND's
host-side PHILOX4_32_10 generator.  Seeded with s, it emits output block m from
counter (m >> 16, 0, m & 0xffff, 0) under key (s low 32 bits, s high 32 bits).
"""
import ctypes

import numpy as np
import pytest

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcurand is not available")


def _curand_blocks(seed, n_blocks):
    cr = _curand()
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(4 * n_blocks, dtype=np.uint32)
        assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        cr.curandDestroyGenerator(gen)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 1, 4357, 0x123456789ABCDEF0, 2**64 - 1])
def test_philox_matches_curand_host_generator(oracle, seed):
    n_blocks = (1 << 16) + 300
    ref = _curand_blocks(seed, n_blocks)
    rng = np.random.default_rng(seed % 1000)
    blocks = sorted(set([0, 1, 2, 3, 65535, 65536, 65537, n_blocks - 1]) |
                    set(rng.integers(0, n_blocks, 64).tolist()))
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for m in blocks:
        got = oracle.philox([m >> 16, 0, m & 0xFFFF, 0], key)
        assert got == [int(v) for v in ref[m]], f"block {m}"


def test_uniform_conversion_is_exact_and_open(oracle):
    # (r + 1/2) 2^-32: the smallest and largest values stay strictly inside (0, 1)
    lib = oracle.lib()
    seen = []
    for pid in range(2000):
        seen.append(oracle.draw4(pid, 0, 0, 0))
    u = np.concatenate(seen)
    assert u.min() > 0.0 and u.max() < 1.0
    # every uniform is an odd multiple of 2^-33
    scaled = u * 2.0**33
    assert np.all(scaled == np.round(scaled)) and np.all(np.mod(scaled, 2) == 1)
    del lib


def test_draw_counter_layout(oracle):
    """Counter = (pid low, pid high, event, (lambda << 8) | block), key = (seed, model)."""
    for pid, lam, ev, blk, seed, model in [(0, 0, 0, 0, 0, 0), (2**40 + 17, 3, 5, 1, 99, 7),
                                          (2**33 - 1, 255, 1000, 0, 2**32 - 1, 4095)]:
        r = oracle.philox([pid & 0xFFFFFFFF, pid >> 32, ev, (lam << 8) | blk], [seed, model])
        expect = (np.array(r, dtype=np.float64) + 0.5) * 2.0**-32
        np.testing.assert_array_equal(oracle.draw4(pid, lam, ev, blk, seed, model), expect)


def test_uniforms_are_uniform_and_independent(oracle):
    """Kolmogorov-Smirnov on 40k draws and a lag correlation check."""
    from scipy import stats
    u = np.concatenate([oracle.draw4(p, 1, 3, 0, seed=11) for p in range(10000)])
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    c = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(c) < 4.0 / np.sqrt(u.size)
