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

from . import linalg, philox, sketch


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


def block_lanczos(A, k, s, q, seed, instance=0):
    """k-SVD by the simplified block Lanczos method (Algorithm 5.1 and the listing of Sec. 5.1), FP64:

      C = A Omega (Omega n x s iid N(0, 1), stream 0);   K = [C, (A A^T) C, ..., (A A^T)^(q-1) C] (m x s q),
      each new block formed as C = A (A^T C) from the previous one and orthonormalised (the listing's
      "optional" qr, kept for stability as the footnote of Sec. 5.1 advises);
      Q = qr(K).Q;   B = Q^T A (s q x n);   B = U_B diag(sigma) V_B^T;   keep the top k:
      U = Q U_B[:, :k], sigma[:k], V = V_B[:, :k]   (signs fixed as in ``rsvd``).
    Returns U, sigma, V and Q.
    """
    A = np.asarray(A, dtype=np.float64)
    C = A @ omega(A.shape[1], s, seed, instance)
    blocks = [C]
    for _ in range(1, q):
        C = A @ (A.T @ C)
        C, _ = linalg.householder_qr(C)
        blocks.append(C)
    Q, _ = linalg.householder_qr(np.hstack(blocks))
    B = Q.T @ A
    Ub_t, sigma, Vb_t = linalg.jacobi_svd(B.T)
    U = Q @ Vb_t[:, :k]
    V = Ub_t[:, :k]
    U, V = fix_signs(U, V)
    return U, sigma[:k], V, Q


# instances of the three sketching operators of the faster k-SVD (one seed, distinct Philox instances)
FAST_INSTANCE_S, FAST_INSTANCE_PCS, FAST_INSTANCE_PGP = 1, 2, 3


def faster_rsvd(A, k, s, p_cs, p, seed):
    """Faster randomized k-SVD (Algorithm 5.3 and the listing of Sec. 5.3), FP64:

      C = A S with S an n x s count sketch (the column form of Algorithm 3.1, instance 1);
      P = P_cs P_gp, P_cs an m x p_cs count sketch (instance 2), P_gp a p_cs x p Gaussian projection
      (instance 3);  D = P^T C (p x s),  L = P^T A (p x n), both from one sketch of [A, C];
      D = Q_D R_D (Householder);  (Q_D^T L)_k = U_bar diag(sigma_bar) V_bar^T (top k of a full SVD);
      C R_D^+ U_bar diag(sigma_bar) = U_t diag(sigma_t) V_hat^T (m x k, full SVD);  V_t = V_bar V_hat.
    Returns U_t (m x k), sigma_t (k,), V_t (n x k), signs fixed as in ``rsvd``.
    """
    A = np.asarray(A, dtype=np.float64)
    C = sketch.countsketch_columns(A, s, seed, FAST_INSTANCE_S)
    AC = np.hstack([A, C])
    P1 = sketch.countsketch(AC, p_cs, seed, FAST_INSTANCE_PCS)            # P_cs^T [A, C]   (p_cs x (n + s))
    P2 = sketch.gaussian_sketch(P1, p, seed, FAST_INSTANCE_PGP)           # P_gp^T P_cs^T [A, C]   (p x (n + s))
    n = A.shape[1]
    L, D = P2[:, :n], P2[:, n:]
    QD, RD = linalg.householder_qr(D)
    Ub_t, sb, Vb_t = linalg.jacobi_svd((QD.T @ L).T)                     # (Q_D^T L)^T = Ub_t diag(sb) Vb_t^T
    Ubar, sbar, Vbar = Vb_t[:, :k], sb[:k], Ub_t[:, :k]
    M = C @ (np.linalg.pinv(RD) @ (Ubar * sbar))                          # m x k
    Ut, st, Vhat = linalg.jacobi_svd(M)
    Vt = Vbar @ Vhat
    Ut, Vt = fix_signs(Ut, Vt)
    return Ut, st, Vt
