"""Randomized k-SVD with power iterations (Sec. 5.2, Algorithm 5.2; the power step of Sec. 5.1), FP64.

Test infrastructure only.

rsvd(A, k, p, q, seed), l = k + p:
  1. Omega: n x l, iid N(0, 1) (stream 0 of the Philox layout, unscaled as in the listing of Sec. 5.1);
     C = A Omega;  Q = qr(C).Q                                     (Algorithm 5.2, steps 2-4)
  2. q times (the optional power step of the Sec. 5.1 listing, kept as subspace iteration with a QR after
     every product, because Sec. 5.1 warns that the plain Krylov powers lose stability):
       Z = qr(A^T Q).Q;  Q = qr(A Z).Q
  3. B = Q^T A (l x n); B = U_B diag(sigma) V_B^T (full SVD, then keep the top k: the advice that follows the
     listing of Sec. 5.2 prefers svd + truncation over svds)       (Algorithm 5.2, step 5)
  4. U = Q U_B[:, :k], Sigma = sigma[:k], V = V_B[:, :k]            (Algorithm 5.2, step 6)
Signs are fixed for comparison: the entry of largest magnitude in each column of V is made positive.
"""
import numpy as np

from . import linalg, philox


def omega(n, l, seed, instance=0):
    """The n x l Gaussian test matrix of the range finder."""
    return philox.gaussian_matrix(seed, n, l, instance)


def fix_signs(U, V):
    """Flip (u_i, v_i) pairs so the largest-magnitude entry of each v_i is positive."""
    idx = np.argmax(np.abs(V), axis=0)
    sgn = np.sign(V[idx, np.arange(V.shape[1])])
    sgn[sgn == 0] = 1.0
    return U * sgn, V * sgn


def range_finder(A, l, q, seed, instance=0):
    """Q (m x l) with orthonormal columns spanning (A A^T)^q A Omega (steps 1-2 above)."""
    A = np.asarray(A, dtype=np.float64)
    Om = omega(A.shape[1], l, seed, instance)
    Q, _ = linalg.householder_qr(A @ Om)
    for _ in range(q):
        Z, _ = linalg.householder_qr(A.T @ Q)
        Q, _ = linalg.householder_qr(A @ Z)
    return Q


def rsvd(A, k, p, q, seed, instance=0):
    """Returns U (m x k), sigma (k,), V (n x k) and the orthonormal basis Q (m x l)."""
    A = np.asarray(A, dtype=np.float64)
    l = k + p
    Q = range_finder(A, l, q, seed, instance)
    B = Q.T @ A
    # SVD of B through its transpose (n x l, tall), so the one-sided Jacobi works on l columns.
    Ub_t, sigma, Vb_t = linalg.jacobi_svd(B.T)       # B^T = Ub_t diag(sigma) Vb_t^T
    U = Q @ Vb_t[:, :k]                               # left singular vectors of B are Vb_t
    V = Ub_t[:, :k]
    U, V = fix_signs(U, V)
    return U, sigma[:k], V, Q
