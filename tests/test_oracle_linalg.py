"""Pins for oracle.linalg, oracle.rsvd and oracle.lsr.

  * Householder QR and Jacobi SVD against LAPACK (numpy.linalg), closed forms (diagonal and 2x2 SVD) and
    their defining identities;
  * rsvd: exact recovery of a rank-k matrix at q = 0 (the derivation of Sec. 5.2), the Eckart-Young lower
    bound (Sec. 2.2), agreement with the same algorithm run on LAPACK QR/SVD, error non-increasing in q;
  * least squares: noise-free b gives x~ = x*, SRHT at s = N gives x~ = x* (orthogonal invariance),
    normal equations agree on tiny inputs, the residual guarantee of Sec. 4.2 at a generous s.
"""
import numpy as np
import pytest

from oracle import linalg, lsr, philox, rsvd, sketch
import workloads


# ---------------------------------------------------------------- QR

@pytest.mark.parametrize("m,n", [(10, 10), (50, 7), (300, 40)])
def test_householder_qr(m, n):
    A = workloads.gaussian(m, n, m + n).astype(np.float64)
    Q, R = linalg.householder_qr(A)
    np.testing.assert_allclose(Q @ R, A, atol=1e-13)
    np.testing.assert_allclose(Q.T @ Q, np.eye(n), atol=1e-14)
    assert np.all(np.tril(R, -1) == 0)
    Rl = np.linalg.qr(A, mode="r")
    np.testing.assert_allclose(np.abs(np.diag(R)), np.abs(np.diag(Rl)), rtol=1e-12)


def test_householder_qr_rank_deficient():
    A = workloads.exact_rank(60, 8, 3, seed=1).astype(np.float64)
    A[:, 5] = 0.0
    Q, R = linalg.householder_qr(A)
    np.testing.assert_allclose(Q @ R, A, atol=1e-14)


# ---------------------------------------------------------------- SVD

@pytest.mark.parametrize("m,n", [(20, 20), (80, 12), (12, 30), (200, 64)])
def test_jacobi_svd_vs_lapack(m, n):
    A = workloads.gaussian(m, n, 3 * m + n).astype(np.float64)
    U, s, V = linalg.jacobi_svd(A)
    np.testing.assert_allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-12)
    np.testing.assert_allclose((U * s) @ V.T, A, atol=1e-12)
    r = min(m, n)
    np.testing.assert_allclose(U.T @ U, np.eye(r), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(r), atol=1e-12)


def test_jacobi_svd_closed_forms():
    d = np.array([3.0, -7.0, 0.5, 2.0])
    U, s, V = linalg.jacobi_svd(np.diag(d))
    np.testing.assert_allclose(s, [7.0, 3.0, 2.0, 0.5], rtol=1e-15)
    M = np.array([[2.0, 1.0], [-1.0, 3.0]])
    # the squared singular values are the roots of x^2 - ||M||_F^2 x + det(M)^2
    fro2, det = np.sum(M ** 2), np.linalg.det(M)
    disc = np.sqrt(fro2 ** 2 - 4 * det ** 2)
    expect = np.sqrt([(fro2 + disc) / 2, (fro2 - disc) / 2])
    np.testing.assert_allclose(linalg.jacobi_svd(M)[1], expect, rtol=1e-14)


def test_lstsq_against_lapack():
    A = workloads.gaussian(90, 6, 4).astype(np.float64)
    b = workloads.gaussian(90, 1, 5).astype(np.float64).ravel()
    x = linalg.lstsq_qr(A, b)
    np.testing.assert_allclose(x, np.linalg.lstsq(A, b, rcond=None)[0], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(linalg.lstsq_normal(A, b), x, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- rsvd

def test_rsvd_exact_recovery_rank_k():
    """Sec. 5.2: if range(C) contains range(A) then Q Q^T A = A, so a rank-k A is recovered exactly at q = 0."""
    k = 6
    A = workloads.exact_rank(300, 120, k, seed=2, sigma=[5, 4, 3, 2, 1, 0.5], dtype=np.float64)
    U, s, V, Q = rsvd.rsvd(A, k, 4, 0, seed=3)
    np.testing.assert_allclose(s, np.linalg.svd(A, compute_uv=False)[:k], rtol=1e-10)
    np.testing.assert_allclose((U * s) @ V.T, A, atol=1e-12)
    np.testing.assert_allclose(Q @ (Q.T @ A), A, atol=1e-12)


def test_rsvd_eckart_young_and_orthonormality():
    A = workloads.lowrank(400, 150, decay=0.8, noise_std=1e-2, seed=4).astype(np.float64)
    k = 8
    s_true = np.linalg.svd(A, compute_uv=False)
    best = np.sqrt(np.sum(s_true[k:] ** 2))            # ||A - A_k||_F
    for q in [0, 1, 2]:
        U, s, V, _ = rsvd.rsvd(A, k, 5, q, seed=9)
        err = np.linalg.norm(A - (U * s) @ V.T)
        assert err >= best * (1 - 1e-12)
        assert err <= best * 1.5
        np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-12)
        np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-12)
        assert np.all(s <= s_true[:k] * (1 + 1e-12))      # Ritz values never exceed the true ones


def test_rsvd_matches_lapack_pipeline():
    """The same steps on LAPACK's QR and SVD with the same Omega give the same subspace and values."""
    A = workloads.lowrank(256, 96, decay=0.85, seed=5).astype(np.float64)
    k, p, q = 7, 5, 1
    U, s, V, Q = rsvd.rsvd(A, k, p, q, seed=13)
    Om = philox.gaussian_matrix(13, A.shape[1], k + p)
    Ql = np.linalg.qr(A @ Om)[0]
    for _ in range(q):
        Zl = np.linalg.qr(A.T @ Ql)[0]
        Ql = np.linalg.qr(A @ Zl)[0]
    Ub, sl, Vt = np.linalg.svd(Ql.T @ A, full_matrices=False)
    np.testing.assert_allclose(s, sl[:k], rtol=1e-11)
    np.testing.assert_allclose(Q @ Q.T, Ql @ Ql.T, atol=1e-11)
    np.testing.assert_allclose(np.abs(V.T @ Vt[:k].T), np.eye(k), atol=1e-8)


def test_rsvd_error_nonincreasing_in_q():
    A = workloads.lowrank(300, 200, decay=0.97, noise_std=3e-2, seed=6).astype(np.float64)
    k = 10
    errs = []
    for q in [0, 1, 2]:
        e = [np.linalg.norm(A - (lambda r: (r[0] * r[1]) @ r[2].T)(rsvd.rsvd(A, k, 4, q, seed))) for seed in range(4)]
        errs.append(np.mean(e))
    assert errs[0] >= errs[1] - 1e-12 and errs[1] >= errs[2] - 1e-12


# ---------------------------------------------------------------- least squares

@pytest.mark.parametrize("kind", ["gaussian", "srht", "countsketch"])
def test_lsr_noise_free_is_exact(kind):
    """b in range(A) and S^T A of full column rank => the sketched solution is x* exactly."""
    A, _, x = workloads.tall_lsr_numpy(500, 6, seed=1, noise_std=0.0)
    A = A.astype(np.float64)
    b = A @ x
    xs = lsr.lsr_sketch(A, b, 40, kind, seed=2)
    np.testing.assert_allclose(xs, x, rtol=1e-10, atol=1e-10)


def test_lsr_full_srht_is_exact():
    """SRHT at s = N is orthogonal, so min ||S^T (A x - b)|| = min ||A x - b|| even for noisy b."""
    A, b, _ = workloads.tall_lsr_numpy(256, 5, seed=2, noise_std=1.0)
    xs = lsr.lsr_sketch(A, b, 256, "srht", seed=5)
    np.testing.assert_allclose(xs, lsr.lsr_exact(A, b), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("kind", ["gaussian", "srht", "countsketch"])
def test_lsr_normal_equations_agree(kind):
    A, b, _ = workloads.tall_lsr_numpy(200, 4, seed=3, noise_std=0.5)
    np.testing.assert_allclose(lsr.lsr_sketch_normal(A, b, 30, kind, 7), lsr.lsr_sketch(A, b, 30, kind, 7),
                               rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("kind", ["gaussian", "srht", "countsketch"])
def test_lsr_residual_guarantee(kind):
    """Sec. 4.2: ||A x~ - b||^2 <= eta^2 ||A x* - b||^2 with eta near 1 for a generous s."""
    A, b, _ = workloads.tall_lsr_numpy(8192, 10, seed=4, noise_std=1.0)
    xstar = lsr.lsr_exact(A, b)
    s = {"gaussian": 400, "srht": 400, "countsketch": 1600}[kind]
    ratio = lsr.residual_ratio(A, b, lsr.lsr_sketch(A, b, s, kind, 11), xstar)
    assert 1.0 - 1e-12 <= ratio < 1.2, ratio


def test_lsr_exact_against_lapack():
    A, b, _ = workloads.tall_lsr_numpy(300, 9, seed=5)
    np.testing.assert_allclose(lsr.lsr_exact(A, b), np.linalg.lstsq(A.astype(np.float64), b.astype(np.float64),
                                                                    rcond=None)[0], rtol=1e-11, atol=1e-12)
