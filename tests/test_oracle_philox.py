"""Pins for oracle.philox: statistical properties of the draws.

Philox4x32-10's published known-answer vectors are not available here, so the generator is pinned by what
any correct implementation must show (uniform words, balanced independent bits, full avalanche across the
ten rounds) and the derived draws by their target distributions (N(0,1), Rademacher, uniform buckets,
uniform samples without replacement).  A dropped round, a missing XOR or a swapped word shows up as
avalanche or bit-balance failures.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import philox


def test_unit_interval_endpoints():
    assert philox.unit_interval(0) == 2.0 ** -24
    assert philox.unit_interval(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    u = philox.unit_interval(np.arange(0, 1 << 32, 1 << 20, dtype=np.uint64))
    assert np.all((u > 0) & (u < 1))
    assert np.all(u.astype(np.float32).astype(np.float64) == u)      # exact in FP32


def test_words_uniform_chi2():
    w = philox.draw(np.arange(1 << 16), 8, seed=12345)
    for col in range(4):
        counts = np.bincount(w[:, col] >> np.uint32(24), minlength=256)
        p = stats.chisquare(counts).pvalue
        assert p > 1e-4, (col, p)


def test_bit_balance():
    w = philox.draw(np.arange(1 << 15), 9, seed=7)
    bits = np.unpackbits(w.view(np.uint8), axis=1)
    frac = bits.mean(axis=0)
    # 2^15 samples per bit: 6 sigma ~ 0.0166
    assert np.all(np.abs(frac - 0.5) < 0.0166)


def test_avalanche_counter_and_key():
    n = 2000
    base = philox.draw(np.arange(n), 8, seed=99)
    flipped = philox.draw(np.arange(n) ^ 1, 8, seed=99)          # neighbouring counters
    d = np.unpackbits((base ^ flipped).view(np.uint8), axis=1).mean()
    assert abs(d - 0.5) < 0.01
    other_key = philox.draw(np.arange(n), 8, seed=99 ^ (1 << 40))
    d2 = np.unpackbits((base ^ other_key).view(np.uint8), axis=1).mean()
    assert abs(d2 - 0.5) < 0.01
    other_stream = philox.draw(np.arange(n), 10, seed=99)
    d3 = np.unpackbits((base ^ other_stream).view(np.uint8), axis=1).mean()
    assert abs(d3 - 0.5) < 0.01


def test_round_count_matters():
    """Ten rounds mix fully; a one-round map visibly does not (sanity of the avalanche test itself)."""
    c = philox.counters(np.arange(4096), 8)
    one = c.copy()
    one[:, 0] += 1

    def one_round(x):
        x = x.astype(np.uint64)
        p0 = np.uint64(philox.PHILOX_M0) * x[:, 0]
        p1 = np.uint64(philox.PHILOX_M1) * x[:, 2]
        m = np.uint64(0xFFFFFFFF)
        return np.stack([(p1 >> np.uint64(32)) ^ x[:, 1], p1 & m, (p0 >> np.uint64(32)) ^ x[:, 3], p0 & m], 1)
    d = np.unpackbits((one_round(c) ^ one_round(one)).astype(np.uint32).view(np.uint8), axis=1).mean()
    assert d < 0.3
    full = philox.philox4x32_10(c, 5) ^ philox.philox4x32_10(one, 5)
    assert abs(np.unpackbits(full.view(np.uint8), axis=1).mean() - 0.5) < 0.01


def test_gaussian_moments_and_ks():
    G = philox.gaussian_matrix(2024, 512, 256)
    z = G.ravel()
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 0.01
    assert abs(stats.skew(z)) < 0.02
    assert abs(stats.kurtosis(z)) < 0.04
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # cosine and sine halves of one Box-Muller pair are uncorrelated
    assert abs(np.corrcoef(G[:, 0], G[:, 1])[0, 1]) < 0.2


def test_gaussian_layout_and_subset():
    G = philox.gaussian_matrix(3, 10, 7)
    sub = philox.gaussian_matrix(3, 10, 7, col_subset=[6, 1, 4])
    np.testing.assert_array_equal(sub, G[:, [6, 1, 4]])
    # entry (i, j) is drawn from block i * ceil(7/4) + j // 4
    w = philox.draw([2 * 2 + 1], philox.STREAM_GAUSSIAN, 3)[0]
    z0, z1 = philox.box_muller(w[0], w[1])
    assert G[2, 4] == z0 and G[2, 5] == z1


def test_rademacher_and_buckets():
    g = philox.rademacher_signs(11, 1 << 16, philox.STREAM_SRHT_SIGN)
    assert set(np.unique(g)) == {-1.0, 1.0}
    assert abs(g.mean()) < 5 / np.sqrt(g.size)
    s = 97
    h, sg = philox.countsketch_hash(11, 1 << 16, s)
    assert h.min() >= 0 and h.max() < s
    assert stats.chisquare(np.bincount(h, minlength=s)).pvalue > 1e-4
    assert abs(sg.mean()) < 5 / np.sqrt(sg.size)
    # sign independent of bucket: same balance inside one bucket class
    assert abs(sg[h < s // 2].mean()) < 6 / np.sqrt((h < s // 2).sum())


@pytest.mark.parametrize("N,s", [(16, 16), (64, 5), (1024, 100)])
def test_srht_sample_basic(N, s):
    idx = philox.srht_sample(5, N, s)
    assert len(idx) == s and len(np.unique(idx)) == s
    assert np.all(np.diff(idx) > 0) and idx[0] >= 0 and idx[-1] < N


def test_srht_sample_uniform_inclusion():
    N, s, trials = 32, 8, 4000
    counts = np.zeros(N)
    for seed in range(trials):
        counts[philox.srht_sample(seed, N, s)] += 1
    # each index is included with probability s/N
    assert stats.chisquare(counts).pvalue > 1e-4
    assert abs(counts.sum() - trials * s) == 0


def test_sketch_gaussian_moments_ks_and_tail():
    """The 16-bit sketch normals (stream 4): the same moment and Kolmogorov-Smirnov pins as the 32-bit ones, and
    the closed-form bound of the draw: |z| <= sqrt(-2 ln u_min) with u_min = 2^-17."""
    G = philox.sketch_gaussian_matrix(2025, 1024, 256)
    z = G.ravel()
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 0.01
    assert abs(stats.skew(z)) < 0.02
    assert abs(stats.kurtosis(z)) < 0.04
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert np.abs(z).max() <= np.sqrt(-2 * np.log(2.0 ** -17)) + 1e-12
    for j in range(0, 8, 2):        # the two halves of each Box-Muller pair are uncorrelated
        assert abs(np.corrcoef(G[:, j], G[:, j + 1])[0, 1]) < 0.2
    # columns from different pairs of one block, and blocks of neighbouring rows, are uncorrelated
    assert abs(np.corrcoef(G[:, 0], G[:, 2])[0, 1]) < 0.2
    assert abs(np.corrcoef(G[:-1, 0], G[1:, 0])[0, 1]) < 0.2


def test_sketch_gaussian_layout_and_subset():
    G = philox.sketch_gaussian_matrix(3, 10, 19)
    np.testing.assert_array_equal(philox.sketch_gaussian_matrix(3, 10, 19, col_subset=[18, 1, 9]), G[:, [18, 1, 9]])
    # entry (i, j) comes from block i * ceil(19/8) + j // 8; columns 8b+2t, 8b+2t+1 from the halves 2t, 2t+1
    i, j = 4, 13                       # block 4 * 3 + 1, pair t = 2 (columns 12, 13): halves 4, 5 = word 2
    w = int(philox.draw([4 * 3 + 1], philox.STREAM_GAUSS_SKETCH, 3)[0][2])
    u1 = ((w & 0xFFFF) + 0.5) / 65536.0
    u2 = ((w >> 16) + 0.5) / 65536.0
    r = np.sqrt(-2 * np.log(u1))
    assert G[i, 12] == r * np.cos(2 * np.pi * u2) and G[i, j] == r * np.sin(2 * np.pi * u2)
    # the sketch matrix differs from the range finder's stream
    assert not np.allclose(G[:, :7], philox.gaussian_matrix(3, 10, 7))
