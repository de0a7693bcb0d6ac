"""Counter-based random draws for the oracle: Philox4x32-10 and everything derived from it.

Test infrastructure only (see ``oracle/__init__.py``).

The paper draws its sketching randomness with MATLAB's global generator (``randn`` for the Gaussian
projection, Sec. 3.2.1; ``randi``/``randsample`` for the SRHT signs and sample, Sec. 3.2.2; ``randi``/
``randsample`` for the count-sketch signs and hashes, Sec. 3.2.3 and Algorithm 3.1).  A GPU cannot replay
a sequential generator, so both sides draw from Philox4x32-10, the counter-based generator of
Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).  This module is an
independent NumPy restatement of that published definition; the CUDA side has its own.

Philox4x32-10, as published:
  * state: a 128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1), all 32-bit words;
  * one round: (hi0, lo0) = M0 * c0 and (hi1, lo1) = M1 * c2 as full 64-bit products, then
    (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);
  * between rounds the key is bumped by the Weyl constants (k0 += W0, k1 += W1) mod 2^32;
  * ten rounds; the output is the final counter block.

Stream layout (one definition shared with the CUDA side through the library's public header):
  counter = (index mod 2^32, index div 2^32, stream, instance), key = (seed mod 2^32, seed div 2^32).
  stream 0: Gaussian entries (test matrices of the range finder), stream 1: SRHT row signs, stream 2:
  count-sketch bucket and sign, stream 3: SRHT sample keys, stream 4: entries of the Gaussian sketching matrix
  (eight per block, from 16-bit uniforms).  Streams 8 and up are free for test data.
"""
import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

STREAM_GAUSSIAN = 0
STREAM_SRHT_SIGN = 1
STREAM_COUNTSKETCH = 2
STREAM_SRHT_KEY = 3
STREAM_GAUSS_SKETCH = 4


def philox4x32_10(counters, seed):
    """Apply Philox4x32-10 to an (N, 4) array of uint32 counters under a 64-bit seed; returns (N, 4) uint32."""
    c = np.asarray(counters, dtype=np.uint64).reshape(-1, 4).copy()
    k0 = np.uint64(int(seed) & MASK32)
    k1 = np.uint64((int(seed) >> 32) & MASK32)
    m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
    w0, w1 = np.uint64(PHILOX_W0), np.uint64(PHILOX_W1)
    mask = np.uint64(MASK32)
    shift = np.uint64(32)
    for _ in range(10):
        p0 = m0 * c[:, 0]          # exact: both factors < 2^32
        p1 = m1 * c[:, 2]
        hi0, lo0 = p0 >> shift, p0 & mask
        hi1, lo1 = p1 >> shift, p1 & mask
        c = np.stack([hi1 ^ c[:, 1] ^ k0, lo1, hi0 ^ c[:, 3] ^ k1, lo0], axis=1)
        k0 = (k0 + w0) & mask
        k1 = (k1 + w1) & mask
    return c.astype(np.uint32)


def counters(index, stream, instance=0):
    """Counter blocks (index lo, index hi, stream, instance) for an array of 64-bit indices."""
    idx = np.asarray(index, dtype=np.uint64).ravel()
    out = np.empty((idx.size, 4), dtype=np.uint64)
    out[:, 0] = idx & np.uint64(MASK32)
    out[:, 1] = idx >> np.uint64(32)
    out[:, 2] = stream
    out[:, 3] = instance
    return out


def draw(index, stream, seed, instance=0):
    """The four 32-bit words Philox4x32-10 gives for each index of one stream."""
    return philox4x32_10(counters(index, stream, instance), seed)


def unit_interval(word):
    """Map a 32-bit word to the open interval (0, 1): ((word >> 9) + 1/2) * 2^-23.  The value has at most 24
    significant bits, so it is exact in FP32 as well as FP64 and both sides start from the same number."""
    w = np.asarray(word, dtype=np.uint64) >> np.uint64(9)
    return (w.astype(np.float64) + 0.5) * 2.0 ** -23


def box_muller(w_a, w_b):
    """Two independent N(0,1) values from two 32-bit words (Box and Muller, 1958), in FP64.

    u1, u2 uniform on (0,1); r = sqrt(-2 ln u1); z_cos = r cos(2 pi u2), z_sin = r sin(2 pi u2).
    """
    u1 = unit_interval(w_a)
    u2 = unit_interval(w_b)
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


def gaussian_matrix(seed, rows, cols, instance=0, col_subset=None):
    """Standard normal matrix G (rows x cols) from stream 0, in FP64.

    Entry (i, j) comes from the Philox block at index i * ceil(cols / 4) + j // 4: words (0, 1) give
    columns 4t and 4t+1 (cosine, sine), words (2, 3) give 4t+2 and 4t+3.
    ``col_subset`` restricts the returned columns (every row is still drawn).
    """
    groups = (cols + 3) // 4
    if col_subset is None:
        col_subset = np.arange(cols)
    col_subset = np.asarray(col_subset, dtype=np.int64)
    need = np.unique(col_subset // 4)
    idx = (np.arange(rows, dtype=np.uint64)[:, None] * np.uint64(groups) + need.astype(np.uint64)[None, :]).ravel()
    w = draw(idx, STREAM_GAUSSIAN, seed, instance).reshape(rows, need.size, 4)
    z0, z1 = box_muller(w[..., 0], w[..., 1])
    z2, z3 = box_muller(w[..., 2], w[..., 3])
    block = np.stack([z0, z1, z2, z3], axis=2)            # rows x groups x 4
    pos = np.searchsorted(need, col_subset // 4)
    return block[:, pos, col_subset % 4]


def rademacher_signs(seed, count, stream, instance=0):
    """+1/-1 per index: the top bit of word 0 set means -1 (the paper's randi(2)*2-3, iid)."""
    w = draw(np.arange(count, dtype=np.uint64), stream, seed, instance)
    return np.where(w[:, 0] >> np.uint32(31), -1.0, 1.0)


def countsketch_hash(seed, m, s, instance=0):
    """Count-sketch bucket h(i) in [0, s) and sign g(i) for rows i < m (Algorithm 3.1, Sec. 3.2.3).

    Bucket: floor(word0 * s / 2^32) (the high half of the 64-bit product), sign: top bit of word 1.
    """
    w = draw(np.arange(m, dtype=np.uint64), STREAM_COUNTSKETCH, seed, instance)
    bucket = ((w[:, 0].astype(np.uint64) * np.uint64(s)) >> np.uint64(32)).astype(np.int64)
    sign = np.where(w[:, 1] >> np.uint32(31), -1.0, 1.0)
    return bucket, sign


def srht_keys(seed, N, instance=0):
    """64-bit sample key per index j < N: (word0 << 32) | word1 of stream 3."""
    w = draw(np.arange(N, dtype=np.uint64), STREAM_SRHT_KEY, seed, instance).astype(np.uint64)
    return (w[:, 0] << np.uint64(32)) | w[:, 1]


def srht_sample(seed, N, s, instance=0):
    """s distinct indices of [0, N), uniformly at random without replacement, returned in ascending order
    (the paper's sort(randsample(n, s)), Sec. 3.2.2): the indices of the s smallest keys, ties to the
    smaller index."""
    keys = srht_keys(seed, N, instance)
    order = np.lexsort((np.arange(N), keys))      # primary: key, secondary: index
    return np.sort(order[:s])


def unit_interval16(half):
    """Map a 16-bit value to (0, 1): (half + 1/2) * 2^-16 (exact in FP32 and FP64)."""
    return (np.asarray(half, dtype=np.float64) + 0.5) * 2.0 ** -16


def sketch_gaussian_matrix(seed, rows, cols, instance=0, col_subset=None):
    """The entries of the Gaussian sketching matrix G (rows x cols) of Sec. 3.2.1, from stream 4, in FP64.

    Entry (i, j) comes from the Philox block at index i * ceil(cols / 8) + j // 8.  Its four words give eight
    16-bit halves, h[2w] = low half and h[2w + 1] = high half of word w; pair t = 0..3 of halves gives columns
    8b + 2t and 8b + 2t + 1 by Box-Muller on u = (h + 1/2) 2^-16: r = sqrt(-2 ln u(h[2t])),
    (r cos 2 pi u(h[2t+1]), r sin 2 pi u(h[2t+1])).  Eight normals per block instead of four (half the Philox
    work per entry); the uniforms' 2^-16 resolution is finer than the 2^-11 of the TF32 operands the sketch
    feeds, and |G_ij| <= sqrt(-2 ln 2^-17) ~ 4.85.
    ``col_subset`` restricts the returned columns (every row is still drawn).
    """
    groups = (cols + 7) // 8
    if col_subset is None:
        col_subset = np.arange(cols)
    col_subset = np.asarray(col_subset, dtype=np.int64)
    need = np.unique(col_subset // 8)
    idx = (np.arange(rows, dtype=np.uint64)[:, None] * np.uint64(groups) + need.astype(np.uint64)[None, :]).ravel()
    w = draw(idx, STREAM_GAUSS_SKETCH, seed, instance).astype(np.uint64).reshape(rows, need.size, 4)
    halves = np.empty((rows, need.size, 8), dtype=np.uint64)
    halves[..., 0::2] = w & np.uint64(0xFFFF)
    halves[..., 1::2] = w >> np.uint64(16)
    out = np.empty((rows, need.size, 8))
    for t in range(4):
        r = np.sqrt(-2.0 * np.log(unit_interval16(halves[..., 2 * t])))
        ang = 2.0 * np.pi * unit_interval16(halves[..., 2 * t + 1])
        out[..., 2 * t] = r * np.cos(ang)
        out[..., 2 * t + 1] = r * np.sin(ang)
    pos = np.searchsorted(need, col_subset // 8)
    return out[:, pos, col_subset % 8]
