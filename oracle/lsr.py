"""Least squares regression: the exact solution (Sec. 4.1) and sketch-and-solve (Sec. 4.2), FP64.

Test infrastructure only.

exact:        x* = argmin ||A x - b||_2 = A^+ b, by Householder QR of A.
lsr_sketch:   sketch [A, b] jointly with ONE sketching matrix S (the listing of Sec. 4.2 sketches the
              augmented matrix), then x~ = argmin ||(S^T A) x - S^T b||_2 by Householder QR of S^T A
              (the listing's backslash is a QR solve).
Guarantee (Sec. 4.2, proved there from the subspace-embedding property):
              ||A x~ - b||^2 <= eta^2 ||A x* - b||^2.
"""
import numpy as np

from . import linalg, sketch


def lsr_exact(A, b):
    return linalg.lstsq_qr(A, b)


def sketch_augmented(A, b, s, kind, seed, instance=0):
    """(S^T A, S^T b) from one sketch of the augmented matrix [A, b]."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64).reshape(-1, 1)
    C = sketch.sketch(np.hstack([A, b]), s, kind, seed, instance)
    return C[:, :-1], C[:, -1]


def lsr_sketch(A, b, s, kind, seed, instance=0):
    SA, Sb = sketch_augmented(A, b, s, kind, seed, instance)
    return linalg.lstsq_qr(SA, Sb)


def lsr_sketch_normal(A, b, s, kind, seed, instance=0):
    """The same sketched problem solved through its normal equations (tiny inputs)."""
    SA, Sb = sketch_augmented(A, b, s, kind, seed, instance)
    return linalg.lstsq_normal(SA, Sb)


def residual_ratio(A, b, x, xstar):
    """||A x - b||^2 / ||A x* - b||^2, the quantity the guarantee of Sec. 4.2 bounds by eta^2."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    r = A @ x - b
    r0 = A @ xstar - b
    return float(r @ r) / float(r0 @ r0)


def default_step(n, s):
    """Step size theta of Algorithm 4.1 when the caller gives none (the paper leaves it as an input).

    With T = R_Y^-1, (S^T A) T = Q_Y is orthonormal, so the singular values of A T are the inverses of those of
    S^T U_A (U_A an orthonormal basis of range(A)).  For a Gaussian sketch of size s those lie near the
    Marchenko-Pastur edges 1 -+ sqrt(n/s); gradient descent on ||A T z - b||^2 converges fastest with
    theta = 2 / (sigma_max^2 + sigma_min^2) of A T, i.e. 2 / ((1 - e)^-2 + (1 + e)^-2) with e = sqrt(n/s)
    (e is capped at 0.9 so the formula stays finite when s is close to n)."""
    e = min(0.9, float(np.sqrt(n / s)))
    return 2.0 / ((1.0 - e) ** -2 + (1.0 + e) ** -2)


def lsr_precise(A, b, s, kind, seed, theta=None, iters=20, instance=0, history=False):
    """Machine-precision least squares by sketch preconditioning (Algorithm 4.1, Sec. 4.3), in FP64 and in
    the algorithm's own order:

      Y = S^T A (s x n) and S^T b from one sketch of [A, b];   Y = Q_Y R_Y (Householder);   T = R_Y^-1;
      z0 = Q_Y^T (S^T b);
      for t = 1..iters:  r = b - A (T z);   z = z + theta T^T (A^T r);
      return x = T z.

    A T is never formed (the remark closing Sec. 4.3): every step applies T, then A, then A^T, then T^T to
    vectors.  With history=True also returns the iterates x_t = T z_t for t = 0..iters.
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = A.shape[1]
    if theta is None:
        theta = default_step(n, s)
    Y, Sb = sketch_augmented(A, b, s, kind, seed, instance)
    QY, RY = linalg.householder_qr(Y)
    T = linalg.upper_inverse(RY)
    z = QY.T @ Sb
    xs = [T @ z]
    for _ in range(iters):
        r = b - A @ (T @ z)
        z = z + theta * (T.T @ (A.T @ r))
        if history:
            xs.append(T @ z)
    x = T @ z
    return (x, xs) if history else x
