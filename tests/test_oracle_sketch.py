"""Pins for oracle.sketch against what Sec. 3 fixes and what mathematics fixes.

  * the paper's printed H_2 and count-sketch S^T (tests/golden/), and SciPy's independent Sylvester Hadamard;
  * H_N H_N^T = N I; the FWHT is its own inverse up to N;
  * exactly one +-1 per column of the count-sketch S^T (Sec. 3.2.3);
  * dense brute force C = S^T A with S built by a different route;
  * norm preservation of the SRHT at s = N (orthogonality), E||S^T x||^2 = ||x||^2 for all kinds;
  * the subspace-embedding property of Sec. 3.1 at a generous sketch size.
"""
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import philox, sketch
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def test_hadamard_matches_paper_H2_and_scipy():
    H2 = load_golden("hadamard_H2.txt")
    np.testing.assert_array_equal(sketch.fwht(np.eye(2)), H2)
    for N in [1, 2, 4, 8, 64, 1024]:
        H = sketch.fwht(np.eye(N))
        np.testing.assert_array_equal(H, scipy.linalg.hadamard(N))
        np.testing.assert_array_equal(H, sketch.hadamard(N))
        np.testing.assert_array_equal(H @ H.T, N * np.eye(N))


def test_fwht_involution_and_linearity():
    X = workloads.gaussian(256, 3, 1).astype(np.float64)
    np.testing.assert_allclose(sketch.fwht(sketch.fwht(X)), 256 * X, rtol=0, atol=1e-11)
    np.testing.assert_allclose(sketch.fwht(X), scipy.linalg.hadamard(256) @ X, rtol=0, atol=1e-11)


def test_countsketch_matches_printed_example():
    St = load_golden("countsketch_St_example.txt")
    s, n = St.shape
    assert (s, n) == (3, 15)
    # the printed matrix has exactly one +-1 per column (the defining structure)
    assert np.all((St != 0).sum(axis=0) == 1)
    assert set(np.unique(St[St != 0])) == {-1.0, 1.0}
    bucket = np.argmax(St != 0, axis=0)
    sign = St[bucket, np.arange(n)]
    np.testing.assert_array_equal(sketch.countsketch_St(bucket, sign, s), St)
    # the streaming algorithm (Algorithm 3.1) on a data matrix reproduces the product with the printed S^T
    A = workloads.gaussian(n, 4, 3).astype(np.float64)
    np.testing.assert_allclose(sketch.countsketch_from_hashes(A, bucket, sign, s), St @ A, atol=1e-14)


@pytest.mark.parametrize("m,s", [(50, 7), (1000, 64), (3, 1)])
def test_countsketch_structure(m, s):
    St = sketch.countsketch_S(m, s, seed=4).T
    assert np.all((St != 0).sum(axis=0) == 1)
    assert set(np.unique(St[St != 0])) <= {-1.0, 1.0}
    A = workloads.gaussian(m, 5, 9).astype(np.float64)
    C = sketch.countsketch(A, s, 4)
    np.testing.assert_allclose(C, St @ A, atol=1e-12)
    # row-sum identity: sum over buckets of C equals sum_i g_i A_i
    _, g = philox.countsketch_hash(4, m, s)
    np.testing.assert_allclose(C.sum(axis=0), g @ A, atol=1e-11)


def test_srht_dense_bruteforce_and_padding():
    for m, s in [(64, 16), (50, 20), (33, 64)]:
        A = workloads.gaussian(m, 6, m).astype(np.float64)
        C = sketch.srht_sketch(A, s, seed=21)
        N = sketch.next_pow2(m)
        g = philox.rademacher_signs(21, m, philox.STREAM_SRHT_SIGN)
        idx = philox.srht_sample(21, N, s)
        H = scipy.linalg.hadamard(N)                     # independent construction
        Cref = (H[idx][:, :m] * g) @ A / np.sqrt(s)
        np.testing.assert_allclose(C, Cref, atol=1e-12)
        np.testing.assert_allclose(sketch.srht_S(m, s, 21).T @ A, Cref, atol=1e-12)


def test_srht_rows_definition_matches_transform():
    A = workloads.gaussian(100, 7, 2).astype(np.float64)
    C = sketch.srht_sketch(A, 40, seed=8)
    rows = sketch.srht_sketch_rows(A, 40, 8, [0, 17, 39])
    np.testing.assert_allclose(rows, C[[0, 17, 39]], atol=1e-12)


def test_srht_full_sample_is_orthogonal():
    """At s = N the SRHT is (1/sqrt(N)) H_N D, an orthogonal map: norms are preserved exactly."""
    A = workloads.gaussian(128, 9, 5).astype(np.float64)
    C = sketch.srht_sketch(A, 128, seed=3)
    np.testing.assert_allclose(np.linalg.norm(C, axis=0), np.linalg.norm(A, axis=0), rtol=1e-13)
    np.testing.assert_allclose(C.T @ C, A.T @ A, atol=1e-11)


def test_gaussian_rows_match_full():
    A = workloads.gaussian(40, 5, 1).astype(np.float64)
    C = sketch.gaussian_sketch(A, 13, seed=6)
    np.testing.assert_allclose(sketch.gaussian_sketch_rows(A, 13, 6, [12, 0, 5]), C[[12, 0, 5]], atol=1e-13)
    np.testing.assert_allclose(sketch.gaussian_S(40, 13, 6).T @ A, C, atol=1e-12)


@pytest.mark.parametrize("kind", ["gaussian", "srht", "countsketch"])
def test_norm_preserved_in_expectation(kind):
    """E ||S^T x||^2 = ||x||^2 for all three operators (their scalings, Sec. 3.2)."""
    m, s, trials = 64, 16, 400
    x = workloads.gaussian(m, 1, 0).astype(np.float64)
    vals = [np.sum(sketch.sketch(x, s, kind, seed) ** 2) for seed in range(trials)]
    ratio = np.mean(vals) / np.sum(x ** 2)
    assert abs(ratio - 1) < 0.08, ratio


@pytest.mark.parametrize("kind", ["gaussian", "srht", "countsketch"])
def test_subspace_embedding(kind):
    """Property 3.1: for a generous s, ||y^T S^T A||^2 / ||y^T A||^2 ... i.e. the singular values of S^T U
    (U an orthonormal basis of range(A)) lie near 1."""
    m, d = 4096, 8
    s = {"gaussian": 512, "srht": 512, "countsketch": 2048}[kind]
    U = workloads.haar(m, d, workloads.rng(1))
    sv = np.linalg.svd(sketch.sketch(U, s, kind, seed=17), compute_uv=False)
    assert sv.max() < 1.35 and sv.min() > 0.65, sv


def test_sketch_of_augmented_matrix_splits():
    """Sketching [A, b] with one S equals sketching A and b separately with the same seed."""
    A = workloads.gaussian(70, 4, 1).astype(np.float64)
    b = workloads.gaussian(70, 1, 2).astype(np.float64)
    for kind in ["gaussian", "srht", "countsketch"]:
        C = sketch.sketch(np.hstack([A, b]), 12, kind, 5)
        np.testing.assert_allclose(C[:, :4], sketch.sketch(A, 12, kind, 5), atol=1e-12)
        np.testing.assert_allclose(C[:, 4:], sketch.sketch(b, 12, kind, 5), atol=1e-12)
