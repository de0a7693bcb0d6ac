"""Planted mistakes: each test plants one plausible error in the oracle (on the CPU, through monkeypatch) and
checks that a pin from the other oracle tests rejects it.  This shows the pins can fail."""
import numpy as np
import pytest
import scipy.linalg

from oracle import linalg, lsr, philox, rsvd, sketch
import workloads


def test_dropped_butterfly_sign_is_caught(monkeypatch):
    def bad_fwht(X):
        Y = np.array(X, dtype=np.float64, copy=True)
        N, h = Y.shape[0], 1
        while h < N:
            Z = Y.reshape(N // (2 * h), 2, h, -1)
            Y = np.stack([Z[:, 0] + Z[:, 1], Z[:, 1] - Z[:, 0]], axis=1).reshape(Y.shape)   # sign flipped
            h *= 2
        return Y
    monkeypatch.setattr(sketch, "fwht", bad_fwht)
    assert not np.array_equal(sketch.fwht(np.eye(8)), scipy.linalg.hadamard(8))


def test_paper_literal_srht_scale_is_caught(monkeypatch):
    """The definition's 1/sqrt(s n) scale (as printed in Sec. 3.2.2) breaks norm preservation at s = N."""
    A = workloads.gaussian(64, 3, 1).astype(np.float64)
    good = sketch.srht_sketch(A, 64, 2)
    bad = good / np.sqrt(64)
    assert not np.allclose(np.linalg.norm(bad, axis=0), np.linalg.norm(A, axis=0), rtol=1e-3)
    assert np.allclose(np.linalg.norm(good, axis=0), np.linalg.norm(A, axis=0), rtol=1e-12)


def test_dropped_countsketch_sign_is_caught(monkeypatch):
    real = sketch.countsketch_from_hashes
    monkeypatch.setattr(sketch, "countsketch_from_hashes", lambda A, b, g, s: real(A, b, np.abs(g), s))
    St = np.loadtxt("tests/golden/countsketch_St_example.txt", comments="#")
    bucket = np.argmax(St != 0, axis=0)
    sign = St[bucket, np.arange(15)]
    A = workloads.gaussian(15, 2, 3).astype(np.float64)
    assert not np.allclose(sketch.countsketch_from_hashes(A, bucket, sign, 3), St @ A)


def test_mispaired_singular_vectors_are_caught(monkeypatch):
    """Pairing sigma_i with the wrong right singular vector breaks the exact-recovery pin."""
    real = linalg.jacobi_svd
    monkeypatch.setattr(linalg, "jacobi_svd", lambda M: (lambda u, s, v: (u, s, v[:, ::-1]))(*real(M)))
    k = 4
    A = workloads.exact_rank(40, 40, k, seed=2, dtype=np.float64)
    U, s, V, _ = rsvd.rsvd(A, k, 3, 0, seed=3)
    assert not np.allclose((U * s) @ V.T, A, atol=1e-8)


def test_wrong_rotation_sign_is_caught():
    A = workloads.gaussian(30, 6, 5).astype(np.float64)
    W = A.copy()
    # one Jacobi step with the rotation applied the wrong way round does not orthogonalise the pair
    a, b, g = W[:, 0] @ W[:, 0], W[:, 1] @ W[:, 1], W[:, 0] @ W[:, 1]
    zeta = (b - a) / (2 * g)
    t = np.copysign(1.0, zeta) / (abs(zeta) + np.sqrt(1 + zeta ** 2))
    c = 1 / np.sqrt(1 + t * t)
    s = c * t
    good = (c * W[:, 0] - s * W[:, 1]) @ (s * W[:, 0] + c * W[:, 1])
    bad = (c * W[:, 0] + s * W[:, 1]) @ (-s * W[:, 0] + c * W[:, 1])
    assert abs(good) < 1e-12 and abs(bad) > 1e-3


def test_b_sketched_with_another_seed_is_caught(monkeypatch):
    """Sketching A and b with different operators breaks the noise-free exactness pin."""
    A, _, x = workloads.tall_lsr_numpy(300, 5, seed=1, noise_std=0.0)
    A = A.astype(np.float64)
    b = A @ x
    SA = sketch.sketch(A, 30, "countsketch", 1)
    Sb = sketch.sketch(b[:, None], 30, "countsketch", 2)[:, 0]
    assert not np.allclose(linalg.lstsq_qr(SA, Sb), x, atol=1e-6)


def test_transposed_gaussian_layout_is_caught():
    """Reading Omega with rows and columns swapped changes the draw (the layout is part of the spec)."""
    G = philox.gaussian_matrix(4, 8, 8)
    assert not np.allclose(G, philox.gaussian_matrix(4, 8, 8).T)


def test_dropped_preconditioner_transpose_is_caught(monkeypatch):
    """Algorithm 4.1 with the gradient step z += theta A^T r (T^T dropped) no longer reaches x*."""
    A, b, _ = workloads.tall_lsr_numpy(2000, 8, seed=5)
    A = A * np.linspace(1, 30, 8).astype(np.float32)         # columns of different scale: T matters
    xs = np.linalg.lstsq(A.astype(np.float64), b.astype(np.float64), rcond=None)[0]
    good = lsr.lsr_precise(A, b, 200, "gaussian", 1, iters=40)
    assert np.linalg.norm(good - xs) / np.linalg.norm(xs) < 1e-10

    def bad(A_, b_, s, kind, seed, theta=None, iters=20, instance=0, history=False):
        A64, b64 = np.asarray(A_, np.float64), np.asarray(b_, np.float64)
        Y, Sb = lsr.sketch_augmented(A64, b64, s, kind, seed, instance)
        QY, RY = linalg.householder_qr(Y)
        T = linalg.upper_inverse(RY)
        z = QY.T @ Sb
        th = lsr.default_step(A64.shape[1], s) if theta is None else theta
        for _ in range(iters):
            z = z + th * (A64.T @ (b64 - A64 @ (T @ z)))       # planted: T^T missing
        return T @ z
    monkeypatch.setattr(lsr, "lsr_precise", bad)
    with np.errstate(all="ignore"):
        x = lsr.lsr_precise(A, b, 200, "gaussian", 1, iters=40)
    assert not (np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-10)


def test_block_lanczos_without_the_power_step_is_caught(monkeypatch):
    """Dropping A A^T from the Krylov blocks (every block = A Omega re-orthonormalised) stalls the
    convergence pin against LAPACK."""
    A = workloads.factor_rank_numpy(1500, 500, 200, seed=3)
    sv = np.linalg.svd(A.astype(np.float64), compute_uv=False)[:10]
    A64 = A.astype(np.float64)
    Om = rsvd.omega(500, 20, 4)
    blocks = [A64 @ Om]
    for _ in range(5):
        blocks.append(linalg.householder_qr(A64 @ Om)[0])       # planted: no (A A^T) applied
    Q, _ = linalg.householder_qr(np.hstack(blocks))
    s = np.linalg.svd(Q.T @ A64, compute_uv=False)[:10]
    assert not np.max(np.abs(s - sv) / sv) < 1e-10
    assert np.max(np.abs(rsvd.block_lanczos(A, 10, 20, 6, 4)[1] - sv) / sv) < 1e-10


def test_faster_rsvd_with_a_shared_hash_is_caught(monkeypatch):
    """Drawing P_cs with the same instance as S (one hash for the columns and the rows) is a plausible slip;
    on a square matrix it correlates the two sketches.  The explicit-operator pin of the composite sketch
    catches a wrong instance for P_gp."""
    A = workloads.gaussian(200, 5, 4).astype(np.float64)
    Scs = sketch.countsketch_S(200, 40, 8, instance=2)
    Sgp = sketch.gaussian_S(40, 12, 8, instance=3)
    bad = sketch.gaussian_countsketch(A, 40, 12, 8, instance_gp=2)
    assert not np.allclose(bad, (Scs @ Sgp).T @ A, atol=1e-6)


def test_nystrom_with_the_footnote_scaling_is_caught():
    """L = C U_k lam_k^-1 (the footnote of Sec. 6.4) instead of lam_k^-1/2 (the listing) breaks
    L[S] L[S]^T = W_k."""
    from oracle import kernel
    X = np.random.default_rng(0).standard_normal((300, 5))
    L, S, lam, U = kernel.nystrom(X, 2.0, 30, 5)
    C = kernel.rbf(X, X[S], 2.0)
    Lbad = C @ (U / lam)
    W = kernel.rbf(X[S], X[S], 2.0)
    w, V = np.linalg.eigh(W)
    w, V = w[::-1], V[:, ::-1]
    k = len(lam)
    Wk = (V[:, :k] * w[:k]) @ V[:, :k].T
    assert np.allclose(L[S] @ L[S].T, Wk, atol=1e-10)
    assert not np.allclose(Lbad[S] @ Lbad[S].T, Wk, atol=1e-3)
