"""Pins of the oracle's counter-based generator (Philox4x32-10, Salmon et al. SC'11).

The draws are keyed by (particle id, step, tag, j) so that both the CPU oracle and
the CUDA path draw the same numbers for the same particle and step (the MCC draw
of Eq. 4, injection, scattering angles). The oracle's implementation is pinned to
an independent implementation -- cuRAND's host-side Philox4_32_10 generator,
a library routine -- and to uniformity/independence statistics.
"""
import ctypes as C
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def _curand():
    try:
        return C.CDLL("libcurand.so.10")
    except OSError:
        try:
            return C.CDLL("libcurand.so")
        except OSError:
            return None


@pytest.mark.parametrize("seed", [0, 42, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    gen = C.c_void_p()
    assert cr.curandCreateGeneratorHost(C.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
        n_threads = 65536  # the host generator's subsequence stride
        rounds = 3
        out = np.zeros(4 * n_threads * rounds, dtype=np.uint32)
        assert cr.curandGenerate(gen, out.ctypes.data_as(C.c_void_p), C.c_size_t(out.size)) == 0
    finally:
        cr.curandDestroyGenerator(gen)
    blocks = out.reshape(-1, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    rng = np.random.default_rng(seed & 0xFFFF)
    picks = np.concatenate([np.arange(8), rng.integers(0, blocks.shape[0], 300), [blocks.shape[0] - 1]])
    for g in picks:
        g = int(g)
        ctr = [g // n_threads, 0, g % n_threads, 0]
        assert (O.philox(ctr, key) == blocks[g]).all(), (g, ctr)


def test_u01_is_exact_midpoint_of_52_bit_grid():
    for a, b in [(0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0x12345678, 0x9ABCDEF0), (1, 0xFFF), (0, 0x1000)]:
        m = (a << 20) | (b >> 12)
        expect = (Fraction(m) + Fraction(1, 2)) / Fraction(2 ** 52)
        assert Fraction(O.u01(a, b)) == expect
    assert 0.0 < O.u01(0, 0) < 1e-15
    assert 1.0 - 1e-15 < O.u01(0xFFFFFFFF, 0xFFFFFFFF) < 1.0


def test_uniformity_ks_and_chi2():
    from scipy import stats
    u = O.uniforms(seed=42, n=200_000, step=7, tag=0).reshape(-1)
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    hist, _ = np.histogram(u, bins=200, range=(0, 1))
    assert stats.chisquare(hist).pvalue > 1e-3
    # moments of U(0,1)
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / u.size)
    assert abs((u ** 2).mean() - 1 / 3) < 4 * np.sqrt(4 / 45 / u.size)


def test_independence_across_pid_step_tag_and_block():
    from scipy import stats
    n = 100_000
    a = O.uniforms(42, n, step=10, tag=0)[:, 0]
    b = O.uniforms(42, n, step=11, tag=0)[:, 0]     # next step, same particles (counter word 1)
    c = O.uniforms(42, n, step=10, tag=1)[:, 0]     # other tag (word 2)
    d = O.uniforms(42, n, step=10, tag=0, j=1)[:, 0]  # other block (word 3)
    e = O.uniforms(42, n, step=10, tag=0, pid0=1)[:, 0]  # neighbouring particle ids (word 0)
    f = O.uniforms(43, n, step=10, tag=0)[:, 0]     # other seed (key)
    for other in (b, c, d, e, f):
        r = np.corrcoef(a, other)[0, 1]
        assert abs(r) < 5 / np.sqrt(n)
        assert not np.array_equal(a, other)
    # 2-D uniformity of consecutive-step pairs
    h2, _, _ = np.histogram2d(a, b, bins=20, range=[[0, 1], [0, 1]])
    assert stats.chisquare(h2.reshape(-1)).pvalue > 1e-3


def test_same_counter_same_draw():
    x = O.uniforms(7, 1000, step=3, tag=2)
    y = O.uniforms(7, 1000, step=3, tag=2)
    assert np.array_equal(x, y)
