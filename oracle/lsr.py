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
