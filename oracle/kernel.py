"""Kernel approximation (Ch. 6): the Gaussian RBF kernel matrix (Sec. 6.1) and the Nystrom method
(Sec. 6.4), in FP64.  Test infrastructure only.

rbf(X1, X2, sigma): K_ij = exp(-||x_i - y_j||^2 / (2 sigma^2)).  The printed formula of Sec. 6.1 writes the
denominator as 2 sigma^-2; the listing that follows it divides the half squared distances by sigma^2, which
settles the reading 1 / (2 sigma^2).  The distance is summed directly from its definition (no expansion into
inner products, so no cancellation).

nystrom(X, sigma, s, seed): the listing of Sec. 6.4 --
  S = sort(randsample(n, s))            (s landmark indices, uniform without replacement, ascending: the rule
                                         of the SRHT sample, stream 3, drawn over [0, n));
  C = rbf(X, X[S], sigma) (n x s);  W = C[S, :] (s x s);
  k = ceil(0.8 s);  W = U_W diag(lam) U_W^T (W is symmetric PSD, its SVD is its eigendecomposition);
  L = C U_W[:, :k] diag(lam[:k]^-1/2)   (n x k), so that K ~ L L^T = C (W_k)^+ C^T.
(The footnote of Sec. 6.4 writes Lambda^-1; the listing takes 1/sqrt, which is what makes L L^T = C W_k^+ C^T.)
The columns of U_W are signed so that the entry of largest magnitude is positive.
"""
import math

import numpy as np

from . import linalg, philox


def rbf(X1, X2, sigma):
    X1 = np.asarray(X1, dtype=np.float64)
    X2 = np.asarray(X2, dtype=np.float64)
    d2 = np.zeros((X1.shape[0], X2.shape[0]))
    for c in range(X1.shape[1]):
        diff = X1[:, c][:, None] - X2[:, c][None, :]
        d2 += diff * diff
    return np.exp(-d2 / (2.0 * sigma * sigma))


def landmarks(n, s, seed, instance=0):
    """sort(randsample(n, s)): s distinct indices of [0, n), ascending."""
    return philox.srht_sample(seed, n, s, instance)


def nystrom_rank(s):
    return int(math.ceil(0.8 * s))


def nystrom(X, sigma, s, seed, k=None, instance=0):
    """Returns L (n x k), the landmark indices S, the eigenvalues lam[:k] of W and U_W[:, :k]."""
    X = np.asarray(X, dtype=np.float64)
    S = landmarks(X.shape[0], s, seed, instance)
    C = rbf(X, X[S], sigma)
    W = C[S, :]
    k = nystrom_rank(s) if k is None else k
    # one-sided Jacobi SVD of the symmetric PSD W: W = U diag(lam) V^T with U = V
    U, lam, _ = linalg.jacobi_svd(W)
    U = U[:, :k]
    idx = np.argmax(np.abs(U), axis=0)
    sgn = np.sign(U[idx, np.arange(k)])
    sgn[sgn == 0] = 1.0
    U = U * sgn
    L = C @ (U / np.sqrt(lam[:k]))
    return L, S, lam[:k], U
