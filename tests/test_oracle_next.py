"""Pins of the oracle's machine-precision least squares (Algorithm 4.1), block Lanczos k-SVD (Algorithm 5.1),
faster k-SVD with its composite sketch (Sec. 3.2.4, Algorithm 5.3) and the Nystrom method (Sec. 6.4).

Each pin rests on something other than the oracle itself: LAPACK (numpy.linalg), a closed form of the
iteration, exact recovery of a low-rank matrix, an explicit sketching matrix built another way, or brute force.
"""
import math

import numpy as np
import pytest

from oracle import kernel, linalg, lsr, philox, rsvd, sketch
import workloads


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


# ------------------------------------------------------------------------------- Algorithm 4.1

@pytest.mark.parametrize("kind", ["gaussian", "srht", "countsketch"])
def test_lsr_precise_converges_to_lapack_solution(kind):
    """The iteration reaches the exact least-squares solution x* = A^+ b (LAPACK lstsq), not just the
    sketch-and-solve one."""
    A, b, _ = workloads.tall_lsr_numpy(3000, 12, seed=4)
    xs = np.linalg.lstsq(A.astype(np.float64), b.astype(np.float64), rcond=None)[0]
    x = lsr.lsr_precise(A, b, 300, kind, 9, iters=40)
    assert relerr(x, xs) < 1e-12
    x0 = lsr.lsr_sketch(A, b, 300, kind, 9)
    assert relerr(x0, xs) > 1e-6            # the sketched solution alone is not exact


def test_lsr_precise_matches_the_closed_form_of_gradient_descent():
    """In z = T^-1 x the iteration is z_{t+1} = z_t + theta T^T A^T (b - A T z_t), so
    x_t - x* = T (I - theta T^T A^T A T)^t T^-1 (x_0 - x*).  T is rebuilt here from an explicit sketching
    matrix and LAPACK's QR (column signs do not matter: T -> T D leaves x_t unchanged)."""
    A, b, _ = workloads.tall_lsr_numpy(600, 6, seed=2)
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    s, seed, theta, t = 120, 3, 0.7, 5
    S = sketch.sketch_matrix(600, s, "gaussian", seed)
    Y = S.T @ A64
    Qy, Ry = np.linalg.qr(Y)
    T = np.linalg.inv(Ry)
    x0 = T @ (Qy.T @ (S.T @ b64))
    xs = np.linalg.lstsq(A64, b64, rcond=None)[0]
    G = np.eye(6) - theta * (T.T @ A64.T @ A64 @ T)
    pred = xs + T @ np.linalg.matrix_power(G, t) @ np.linalg.solve(T, x0 - xs)
    _, hist = lsr.lsr_precise(A, b, s, "gaussian", seed, theta=theta, iters=t, history=True)
    assert relerr(hist[0], x0) < 1e-12
    assert relerr(hist[t], pred) < 1e-10


def test_default_step_is_the_optimal_step_of_the_marchenko_pastur_edges():
    for n, s in [(256, 4096), (20, 400), (256, 1024)]:
        e = math.sqrt(n / s)
        smax2, smin2 = (1 - e) ** -2, (1 + e) ** -2
        th = lsr.default_step(n, s)
        # optimal fixed step for singular values in [smin, smax]: both ends contract equally
        assert abs(abs(1 - th * smax2) - abs(1 - th * smin2)) < 1e-12


def test_upper_inverse_against_lapack():
    R = np.triu(workloads.gaussian(9, 9, 3).astype(np.float64)) + 4 * np.eye(9)
    np.testing.assert_allclose(linalg.upper_inverse(R) @ R, np.eye(9), atol=1e-12)


# ------------------------------------------------------------------------------- Algorithm 5.1

def test_block_lanczos_recovers_an_exact_rank_matrix():
    sig = np.linspace(5, 1, 8)
    A = workloads.exact_rank(2000, 300, 8, seed=2, sigma=sig, dtype=np.float64)
    U, s, V, _ = rsvd.block_lanczos(A, 8, 8, 2, 4)
    np.testing.assert_allclose(s, sig, rtol=1e-10)
    np.testing.assert_allclose((U * s) @ V.T, A, atol=1e-10)


def test_block_lanczos_converges_to_lapack_singular_values_as_q_grows():
    A = workloads.factor_rank_numpy(1500, 500, 200, seed=3)
    sv = np.linalg.svd(A.astype(np.float64), compute_uv=False)[:10]
    errs = [np.max(np.abs(rsvd.block_lanczos(A, 10, 20, q, 4)[1] - sv) / sv) for q in (1, 2, 4, 6)]
    assert errs[-1] < 1e-10
    assert all(a > b for a, b in zip(errs, errs[1:]))


def test_block_lanczos_with_one_block_is_the_prototype():
    """q = 1 keeps only C = A Omega: the basis, and so the result, of Algorithm 5.2 with l = s."""
    A = workloads.lowrank(800, 200)
    _, s1, _, _ = rsvd.block_lanczos(A, 6, 12, 1, 5)
    _, s2, _, _ = rsvd.rsvd(A, 6, 6, 0, 5)
    np.testing.assert_allclose(s1, s2, rtol=1e-12)


def test_block_lanczos_respects_eckart_young():
    A = workloads.factor_rank_numpy(600, 300, 100, seed=5).astype(np.float64)
    k = 8
    U, s, V, _ = rsvd.block_lanczos(A, k, 16, 3, 1)
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.linalg.norm(A - (U * s) @ V.T) >= np.sqrt(np.sum(sv[k:] ** 2)) * (1 - 1e-12)


# ------------------------------------------------------------------ Sec. 3.2.4 and Algorithm 5.3

def test_column_countsketch_is_a_times_an_explicit_s():
    A = workloads.gaussian(30, 50, 2).astype(np.float64)
    S = sketch.countsketch_S(50, 7, 11, instance=1)           # n x s, one +-1 per row
    assert np.all(np.count_nonzero(S, axis=1) == 1)
    np.testing.assert_allclose(sketch.countsketch_columns(A, 7, 11, instance=1), A @ S, atol=1e-12)


def test_gaussian_countsketch_is_the_product_of_the_two_explicit_operators():
    A = workloads.gaussian(200, 5, 4).astype(np.float64)
    Scs = sketch.countsketch_S(200, 40, 8, instance=2)        # m x s_cs
    Sgp = sketch.gaussian_S(40, 12, 8, instance=3)            # s_cs x s
    np.testing.assert_allclose(sketch.gaussian_countsketch(A, 40, 12, 8), (Scs @ Sgp).T @ A, atol=1e-12)


def test_faster_rsvd_recovers_an_exact_rank_matrix():
    """If rank(A) = k <= s and the sketches keep the rank, C spans range(A) and the rank-k least-squares
    problem of Algorithm 5.3 is solved exactly (derivation in Sec. 5.3)."""
    sig = np.linspace(5, 1, 8)
    A = workloads.exact_rank(3000, 400, 8, seed=2, sigma=sig, dtype=np.float64)
    U, s, V = rsvd.faster_rsvd(A, 8, 16, 256, 64, 4)
    np.testing.assert_allclose(s, sig, rtol=1e-10)
    np.testing.assert_allclose((U * s) @ V.T, A, atol=1e-10)
    np.testing.assert_allclose(U.T @ U, np.eye(8), atol=1e-10)
    np.testing.assert_allclose(V.T @ V, np.eye(8), atol=1e-10)


def test_faster_rsvd_respects_eckart_young():
    A = workloads.factor_rank_numpy(1500, 400, 200, seed=6).astype(np.float64)
    k = 10
    U, s, V = rsvd.faster_rsvd(A, k, 40, 400, 120, 2)
    sv = np.linalg.svd(A, compute_uv=False)
    err = np.linalg.norm(A - (U * s) @ V.T)
    assert err >= np.sqrt(np.sum(sv[k:] ** 2)) * (1 - 1e-12)
    assert err <= 1.5 * np.sqrt(np.sum(sv[k:] ** 2))         # a useful approximation, not an arbitrary one


# ------------------------------------------------------------------------------------- Sec. 6.4

def test_rbf_against_brute_force():
    g = np.random.default_rng(1)
    X1, X2 = g.standard_normal((7, 3)), g.standard_normal((5, 3))
    K = kernel.rbf(X1, X2, 1.3)
    for i in range(7):
        for j in range(5):
            d2 = sum((X1[i, c] - X2[j, c]) ** 2 for c in range(3))
            assert abs(K[i, j] - math.exp(-d2 / (2 * 1.3 ** 2))) < 1e-15
    np.testing.assert_allclose(np.diag(kernel.rbf(X1, X1, 0.5)), 1.0)


def test_nystrom_reproduces_the_rank_k_landmark_block():
    """C[S] = W, so L[S] L[S]^T = W U_k lam_k^-1 U_k^T W = W_k, the best rank-k part of W (LAPACK eigh)."""
    X = np.random.default_rng(0).standard_normal((500, 8))
    L, S, lam, _ = kernel.nystrom(X, 2.0, 40, 5)
    W = kernel.rbf(X[S], X[S], 2.0)
    w, V = np.linalg.eigh(W)
    w, V = w[::-1], V[:, ::-1]
    k = kernel.nystrom_rank(40)
    assert L.shape == (500, k) and k == 32
    np.testing.assert_allclose(lam, w[:k], rtol=1e-12)
    np.testing.assert_allclose(L[S] @ L[S].T, (V[:, :k] * w[:k]) @ V[:, :k].T, atol=1e-12)


def test_nystrom_with_every_point_as_landmark_is_exact():
    """s = n and k = n: W = K, so C W^-1 C^T = K."""
    X = np.random.default_rng(2).standard_normal((30, 2)) * 2
    L, S, _, _ = kernel.nystrom(X, 1.0, 30, 1, k=30)
    np.testing.assert_array_equal(S, np.arange(30))
    K = kernel.rbf(X, X, 1.0)
    np.testing.assert_allclose(L @ L.T, K, atol=1e-8)


def test_nystrom_landmarks_are_a_sorted_uniform_sample():
    S = kernel.landmarks(1000, 100, 3)
    assert len(set(S.tolist())) == 100 and np.all(np.diff(S) > 0)
    np.testing.assert_array_equal(S, philox.srht_sample(3, 1000, 100))
