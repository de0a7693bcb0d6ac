"""The three sketching operators of Sec. 3.2, written out plainly in FP64.  Test infrastructure only.

Orientation: the library sketches the ROW dimension, C = S^T A with A (m x n) and S (m x s), so C is s x n.
This is the orientation Sec. 4.3 uses for least squares (the sketch S^T A, S^T b); the column sketch
C = A S of Ch. 3 is the same operator applied to A^T.

Every function takes the FP32 input bits, widens them to FP64 and draws its randomness from
``oracle.philox``.
"""
import numpy as np

from . import philox


def next_pow2(m):
    """Smallest power of two >= m (the SRHT pads the transformed dimension to it, Sec. 3.2.2)."""
    n = 1
    while n < m:
        n *= 2
    return n


# ---------------------------------------------------------------- Gaussian projection (Sec. 3.2.1)

def gaussian_sketch(A, s, seed, instance=0):
    """C = S^T A with S = G / sqrt(s), G an m x s matrix of iid N(0, 1) entries (Sec. 3.2.1), drawn from the
    sketch stream (philox.sketch_gaussian_matrix)."""
    A = np.asarray(A, dtype=np.float64)
    G = philox.sketch_gaussian_matrix(seed, A.shape[0], s, instance)
    return (G.T @ A) / np.sqrt(s)


def gaussian_sketch_rows(A, s, seed, rows, instance=0):
    """Selected rows of the Gaussian sketch, for matrices too large to sketch whole on the CPU."""
    A = np.asarray(A, dtype=np.float64)
    G = philox.sketch_gaussian_matrix(seed, A.shape[0], s, instance, col_subset=np.asarray(rows))
    return (G.T @ A) / np.sqrt(s)


def gaussian_S(m, s, seed, instance=0):
    """The explicit m x s Gaussian sketching matrix S = G / sqrt(s)."""
    return philox.sketch_gaussian_matrix(seed, m, s, instance) / np.sqrt(s)


# ---------------------------------------------------------------- SRHT (Sec. 3.2.2)

def fwht(X):
    """Unnormalised fast Walsh-Hadamard transform along axis 0 (length a power of two), natural (Sylvester)
    order: H_1 = [1], H_2n = [[H_n, H_n], [H_n, -H_n]] as in Sec. 3.2.2.  Textbook radix-2 butterflies:
    for h = 1, 2, 4, ..., every pair (i, i + h) inside a block of 2h rows becomes (x_i + x_{i+h},
    x_i - x_{i+h})."""
    Y = np.array(X, dtype=np.float64, copy=True)
    N = Y.shape[0]
    assert N & (N - 1) == 0, "length must be a power of two"
    h = 1
    while h < N:
        Z = Y.reshape(N // (2 * h), 2, h, -1)
        top = Z[:, 0] + Z[:, 1]
        bot = Z[:, 0] - Z[:, 1]
        Y = np.stack([top, bot], axis=1).reshape(Y.shape)
        h *= 2
    return Y


def hadamard(N):
    """H_N as a dense matrix, built by the recursion of Sec. 3.2.2."""
    H = np.ones((1, 1))
    while H.shape[0] < N:
        H = np.block([[H, H], [H, -H]])
    return H


def srht_sketch(A, s, seed, instance=0):
    """C = (1/sqrt(s)) * P^T H_N D A_pad (Sec. 3.2.2, row orientation).

    D: iid +1/-1 row signs (stream 1); A_pad: A with zero rows appended up to N = next_pow2(m);
    H_N: the unnormalised Hadamard matrix; P: s rows sampled without replacement, ascending (stream 3).
    Scale 1/sqrt(s) with unnormalised H: the listing's fwht divides by N and the listing multiplies back by
    n/sqrt(s), so the net factor is 1/sqrt(s), which makes E[S S^T] = I.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    N = next_pow2(m)
    g = philox.rademacher_signs(seed, m, philox.STREAM_SRHT_SIGN, instance)
    Apad = np.zeros((N, n))
    Apad[:m] = g[:, None] * A
    idx = philox.srht_sample(seed, N, s, instance)
    return fwht(Apad)[idx] / np.sqrt(s)


def srht_sketch_rows(A, s, seed, which, instance=0):
    """Rows ``which`` (positions in the sample, 0..s-1) of the SRHT sketch, straight from the definition
    (H_N)[r, i] = (-1)^popcount(r & i): one O(mn) sum per requested row, for matrices too large to
    transform whole on the CPU."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    N = next_pow2(m)
    g = philox.rademacher_signs(seed, m, philox.STREAM_SRHT_SIGN, instance)
    idx = philox.srht_sample(seed, N, s, instance)
    i = np.arange(m, dtype=np.uint64)
    out = np.empty((len(which), n))
    for t, pos in enumerate(which):
        r = np.uint64(idx[pos])
        bits = np.bitwise_count(i & r)
        h = np.where(bits & 1, -1.0, 1.0)
        out[t] = (h * g) @ A / np.sqrt(s)
    return out


def srht_S(m, s, seed, instance=0):
    """The explicit m x s SRHT sketching matrix (for tiny m): S^T = (1/sqrt(s)) P^T H_N D restricted to the
    first m columns."""
    N = next_pow2(m)
    g = philox.rademacher_signs(seed, m, philox.STREAM_SRHT_SIGN, instance)
    idx = philox.srht_sample(seed, N, s, instance)
    H = hadamard(N)
    St = H[idx][:, :m] * g[None, :] / np.sqrt(s)
    return St.T


# ---------------------------------------------------------------- count sketch (Sec. 3.2.3)

def countsketch_from_hashes(A, bucket, sign, s):
    """Algorithm 3.1 in the row orientation: C starts at zero; for each row i in increasing order,
    C[h(i), :] += g(i) * A[i, :]."""
    A = np.asarray(A, dtype=np.float64)
    C = np.zeros((s, A.shape[1]))
    np.add.at(C, bucket, sign[:, None] * A)
    return C


def countsketch(A, s, seed, instance=0):
    """Count sketch C = S^T A with hashes and signs from stream 2."""
    A = np.asarray(A, dtype=np.float64)
    bucket, sign = philox.countsketch_hash(seed, A.shape[0], s, instance)
    return countsketch_from_hashes(A, bucket, sign, s)


def countsketch_St(bucket, sign, s):
    """The explicit s x m matrix S^T: column i holds g(i) in row h(i) and zeros elsewhere (the worked
    example of Sec. 3.2.3 prints one such matrix)."""
    m = len(bucket)
    St = np.zeros((s, m))
    St[np.asarray(bucket), np.arange(m)] = sign
    return St


def countsketch_S(m, s, seed, instance=0):
    bucket, sign = philox.countsketch_hash(seed, m, s, instance)
    return countsketch_St(bucket, sign, s).T


# ---------------------------------------------------------------- dispatch

KINDS = {0: "gaussian", 1: "srht", 2: "countsketch"}


def sketch(A, s, kind, seed, instance=0):
    """C = S^T A for kind 0 (Gaussian), 1 (SRHT) or 2 (count sketch)."""
    kind = KINDS.get(kind, kind)
    if kind == "gaussian":
        return gaussian_sketch(A, s, seed, instance)
    if kind == "srht":
        return srht_sketch(A, s, seed, instance)
    if kind == "countsketch":
        return countsketch(A, s, seed, instance)
    raise ValueError(kind)


def sketch_matrix(m, s, kind, seed, instance=0):
    """The explicit m x s sketching matrix S of any kind (tiny inputs only)."""
    kind = KINDS.get(kind, kind)
    return {"gaussian": gaussian_S, "srht": srht_S, "countsketch": countsketch_S}[kind](m, s, seed, instance)


# ---------------------------------------------------------------- column count sketch (Sec. 3.2.3, Ch. 3 form)

def countsketch_columns(A, s, seed, instance=0):
    """C = A S with S an n x s count sketch (the column orientation of Ch. 3, Algorithm 3.1 over the columns):
    C starts at zero; for each column j in increasing order, C[:, h(j)] += g(j) A[:, j], with the hashes of
    stream 2 drawn for the n column indices.  Equal to countsketch(A^T, s)^T."""
    A = np.asarray(A, dtype=np.float64)
    bucket, sign = philox.countsketch_hash(seed, A.shape[1], s, instance)
    C = np.zeros((A.shape[0], s))
    for j in range(A.shape[1]):
        C[:, bucket[j]] += sign[j] * A[:, j]
    return C


# ---------------------------------------------------------------- Gaussian projection + count sketch (Sec. 3.2.4)

def gaussian_countsketch(A, s_cs, s, seed, instance_cs=2, instance_gp=3):
    """S = S_cs S_gp (m x s): a count sketch to s_cs rows followed by a Gaussian projection to s rows, in the
    row orientation: C = S_gp^T (S_cs^T A)."""
    return gaussian_sketch(countsketch(A, s_cs, seed, instance_cs), s, seed, instance_gp)
