"""Dense FP64 building blocks for the oracle: thin Householder QR and one-sided Jacobi SVD.

Test infrastructure only.  Both are textbook algorithms written out from their definitions (Golub and
Van Loan, "Matrix Computations", Sec. 5.2 and Sec. 8.6) rather than LAPACK calls, so the oracle can be
checked AGAINST LAPACK (numpy.linalg) in the tests.  The paper uses them as black boxes: qr(., 0) and
svd(., 'econ') in the listings of Sec. 4.3 and Sec. 5.2 (QR and SVD are defined in Sec. 2.2).
"""
import numpy as np


def householder_qr(A):
    """Thin QR, A = Q R with Q (m x n) orthonormal columns and R (n x n) upper triangular, m >= n.

    For each column j: v = x + sign(x_0) ||x|| e_0 on the trailing part, H_j = I - 2 v v^T / (v^T v),
    apply H_j to the trailing columns; Q = H_0 H_1 ... H_{n-1} applied to the first n columns of I.
    A zero trailing column is skipped (H_j = I), so rank-deficient inputs are handled.
    """
    R = np.array(A, dtype=np.float64, copy=True)
    m, n = R.shape
    assert m >= n
    vs = []
    for j in range(n):
        x = R[j:, j]
        normx = np.linalg.norm(x)
        if normx == 0.0:
            vs.append(None)
            continue
        v = x.copy()
        v[0] += normx if x[0] >= 0 else -normx
        v /= np.linalg.norm(v)
        R[j:, j:] -= 2.0 * np.outer(v, v @ R[j:, j:])
        R[j + 1:, j] = 0.0
        vs.append(v)
    Q = np.zeros((m, n))
    Q[:n, :n] = np.eye(n)
    for j in range(n - 1, -1, -1):
        v = vs[j]
        if v is None:
            continue
        Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    return Q, np.triu(R[:n, :])


def jacobi_svd(A, tol=1e-15, max_sweeps=60):
    """Thin SVD A = U diag(sigma) V^T by one-sided (Hestenes) Jacobi, m >= n, sigma descending.

    Orthogonalise the columns of W = A pairwise with plane rotations J accumulated into V (W <- W J,
    V <- V J) until every pair satisfies |w_p^T w_q| <= tol * ||w_p|| ||w_q||.  Then sigma_j = ||w_j||,
    u_j = w_j / sigma_j.  For a pair with alpha = ||w_p||^2, beta = ||w_q||^2, gamma = w_p^T w_q:
    zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2),
    s = c t, and (w_p, w_q) <- (c w_p - s w_q, s w_p + c w_q), which zeroes the new w_p^T w_q.
    """
    W = np.array(A, dtype=np.float64, copy=True)
    m, n = W.shape
    transposed = False
    if m < n:
        W = W.T.copy()
        m, n = n, m
        transposed = True
    V = np.eye(n)
    for _ in range(max_sweeps):
        rotated = False
        for p in range(n - 1):
            for q in range(p + 1, n):
                alpha = W[:, p] @ W[:, p]
                beta = W[:, q] @ W[:, q]
                gamma = W[:, p] @ W[:, q]
                if gamma == 0.0 or abs(gamma) <= tol * np.sqrt(alpha * beta):
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                t = np.copysign(1.0, zeta) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                wp, wq = W[:, p].copy(), W[:, q].copy()
                W[:, p] = c * wp - s * wq
                W[:, q] = s * wp + c * wq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
        if not rotated:
            break
    sigma = np.linalg.norm(W, axis=0)
    order = np.argsort(-sigma, kind="stable")
    sigma = sigma[order]
    W = W[:, order]
    V = V[:, order]
    U = np.zeros_like(W)
    nz = sigma > 0
    U[:, nz] = W[:, nz] / sigma[nz]
    if transposed:
        return V, sigma, U
    return U, sigma, V


def lstsq_qr(A, b):
    """x = argmin ||A x - b||_2 through the thin QR of A: R x = Q^T b, back substitution (Sec. 4.1)."""
    Q, R = householder_qr(A)
    y = Q.T @ np.asarray(b, dtype=np.float64)
    n = R.shape[0]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (y[i] - R[i, i + 1:] @ x[i + 1:]) / R[i, i]
    return x


def lstsq_normal(A, b):
    """x from the normal equations (A^T A) x = A^T b, solved by Gaussian elimination with partial pivoting
    written out (tiny inputs only; squares the condition number)."""
    A = np.asarray(A, dtype=np.float64)
    M = A.T @ A
    r = A.T @ np.asarray(b, dtype=np.float64)
    n = M.shape[0]
    Ab = np.hstack([M, r[:, None]])
    for k in range(n):
        piv = k + int(np.argmax(np.abs(Ab[k:, k])))
        Ab[[k, piv]] = Ab[[piv, k]]
        Ab[k + 1:] -= np.outer(Ab[k + 1:, k] / Ab[k, k], Ab[k])
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (Ab[i, n] - Ab[i, i + 1:n] @ x[i + 1:]) / Ab[i, i]
    return x


def upper_inverse(R):
    """R^-1 for an upper-triangular R with non-zero diagonal, by back substitution on each column of I
    (column j solves R x = e_j from the last row up)."""
    R = np.asarray(R, dtype=np.float64)
    n = R.shape[0]
    X = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        for i in range(n - 1, -1, -1):
            X[i, j] = (e[i] - R[i, i + 1:] @ X[i + 1:, j]) / R[i, i]
    return X
