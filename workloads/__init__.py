"""Seeded synthetic inputs shaped like the paper's workloads, shared by the tests, the benchmark and the
oracle checks.

This module holds NO arithmetic of the method (no sketching, no QR of a sketch, no SVD of the result): it
only makes input matrices and right-hand sides.  Everything is deterministic given the seed.  Small inputs
are drawn on the CPU with NumPy's PCG64 stream (identical on every machine); large inputs are drawn on
the device with a seeded torch generator, and the oracle reads back the same FP32 bits.

The paper prints no datasets (it is a tutorial), so these stand in for its problem statements:
  * ``lowrank``      A = U diag(sigma) V^T + noise with Haar U, V (the low-rank setting of Ch. 5);
  * ``tall_lsr``     a tall regression problem with non-uniform row leverage (the n >> d setting of Ch. 4);
  * ``factor_rank``  A = G1 diag(sigma) G2^T with Gaussian factors (a large rank-r matrix, Ch. 5);
  * ``batch_sizes``  uneven problem sizes for the batched and served forms.
"""
import math

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def haar(m, k, gen):
    """m x k matrix with orthonormal columns, Haar-distributed: QR of a Gaussian matrix with R's diagonal
    made positive (Mezzadri, "How to generate random matrices from the classical compact groups", 2007)."""
    G = gen.standard_normal((m, k))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def lowrank(m=2048, n=512, decay=0.9, noise_std=1e-3, seed=0, rank=None):
    """A = U diag(sigma) V^T + E, sigma_i = decay^i (i = 1..r), E iid N(0, noise_std^2); returned as FP32.

    The default is the small parity workload: 2048 x 512, sigma_i = 0.9^i, noise variance 1e-6.
    ``rank`` limits r (default min(m, n)); ``noise_std=0`` gives an exactly rank-r matrix up to FP32
    rounding.
    """
    gen = rng(seed)
    r = min(m, n) if rank is None else rank
    U = haar(m, r, gen)
    V = haar(n, r, gen)
    sigma = decay ** np.arange(1, r + 1, dtype=np.float64)
    A = (U * sigma) @ V.T
    if noise_std:
        A = A + noise_std * gen.standard_normal((m, n))
    return A.astype(np.float32)


def exact_rank(m, n, k, seed=0, sigma=None, dtype=np.float32):
    """A matrix of rank k (exactly in FP64, up to rounding in FP32): A = U diag(sigma) V^T with Haar U, V;
    sigma defaults to 1, 1/2, ..., 1/k."""
    gen = rng(seed)
    U = haar(m, k, gen)
    V = haar(n, k, gen)
    if sigma is None:
        sigma = 1.0 / np.arange(1, k + 1)
    return ((U * np.asarray(sigma)) @ V.T).astype(dtype)


def gaussian(m, n, seed=0, scale=1.0):
    return (scale * rng(seed).standard_normal((m, n))).astype(np.float32)


def tall_lsr_numpy(m, n, seed=0, noise_std=math.sqrt(1e-3)):
    """Tall least-squares problem on the CPU: A_ij ~ N(0,1) times a per-row lognormal(0,1) factor (so row
    leverage is non-uniform), x* ~ N(0,1), b = A x* + N(0, noise_std^2).  Returns FP32 A, b and FP64 x*."""
    gen = rng(seed)
    A = gen.standard_normal((m, n)) * np.exp(gen.standard_normal((m, 1)))
    A = A.astype(np.float32)
    x = gen.standard_normal(n)
    b = (A.astype(np.float64) @ x + noise_std * gen.standard_normal(m)).astype(np.float32)
    return A, b, x


def tall_lsr_torch(m=1 << 20, n=256, seed=0, noise_std=math.sqrt(1e-3), device="cuda"):
    """The same recipe drawn with a seeded torch generator on ``device`` (the full-size regression workload:
    1,048,576 x 256).  Returns torch FP32 A (m x n, row-major), b (m,) and x* (n,) on the device."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    A = torch.randn(m, n, generator=g, device=device, dtype=torch.float32)
    A.mul_(torch.exp(torch.randn(m, 1, generator=g, device=device, dtype=torch.float32)))
    x = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    b = (A.double() @ x + noise_std * torch.randn(m, generator=g, device=device, dtype=torch.float64)).float()
    return A, b, x


def factor_rank_torch(m=65536, n=16384, rank=2048, seed=0, exponent=1.0, device="cuda"):
    """A = G1 diag(sigma) G2^T with G1 (m x r), G2 (n x r) iid N(0,1) and sigma_i = i^-exponent, built in FP32
    on ``device`` (the large randomized-SVD workload: 65,536 x 16,384, r = 2048, sigma_i = 1/i)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    G1 = torch.randn(m, rank, generator=g, device=device, dtype=torch.float32)
    G2 = torch.randn(n, rank, generator=g, device=device, dtype=torch.float32)
    sigma = torch.arange(1, rank + 1, device=device, dtype=torch.float32).pow(-exponent)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        A = (G1 * sigma) @ G2.T
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return A.contiguous()


def factor_rank_numpy(m, n, rank, seed=0, exponent=1.0):
    gen = rng(seed)
    G1 = gen.standard_normal((m, rank))
    G2 = gen.standard_normal((n, rank))
    sigma = np.arange(1, rank + 1, dtype=np.float64) ** (-exponent)
    return ((G1 * sigma) @ G2.T).astype(np.float32)


def batch_sizes(count=4096, seed=0, m_range=(512, 32768), n_range=(16, 256)):
    """Uneven problem sizes: m log-uniform on m_range, n uniform on n_range (integers, inclusive).
    Even positions are rsvd instances, odd positions sketch-and-solve instances."""
    gen = rng(seed)
    lo, hi = math.log(m_range[0]), math.log(m_range[1])
    m = np.exp(gen.uniform(lo, hi, count)).astype(np.int64)
    n = gen.integers(n_range[0], n_range[1] + 1, count)
    return m, n


def batch_specs(count=4096, seed=0, m_range=(512, 32768), n_range=(16, 256), k=16, p=8, q=1, s_factor=4):
    """The batched workload: ``count`` problems with m log-uniform and n uniform (``batch_sizes``); even
    positions are randomized k-SVD problems (k, p, q; oversampling cut to p = n - k where n < k + p, since
    l = k + p may not exceed n), odd positions count-sketch least squares with s = s_factor * n.  Each
    problem has its own seed.  Returns a list of dicts."""
    m, n = batch_sizes(count, seed, m_range, n_range)
    specs = []
    for i in range(count):
        mi, ni = int(m[i]), int(n[i])
        pseed = seed * 1000003 + i
        if i % 2 == 0:
            ki = min(k, ni)
            specs.append(dict(kind="rsvd", m=mi, n=ni, k=ki, p=max(0, min(p, ni - ki)), q=q, seed=pseed))
        else:
            specs.append(dict(kind="lsr", m=mi, n=ni, s=s_factor * ni, seed=pseed))
    return specs


def batch_problem_numpy(spec, exponent=1.5, noise_std=math.sqrt(1e-3)):
    """Inputs of one batched problem on the CPU (FP32).  rsvd: A = U diag(i^-exponent) V^T with Haar U
    (m x r), V (n x r), r = min(m, n).  lsr: A iid N(0, 1), b = A x* + N(0, noise_std^2) with x* ~ N(0, 1).
    Returns (A, b) with b None for rsvd."""
    gen = rng(spec["seed"])
    m, n = spec["m"], spec["n"]
    if spec["kind"] == "rsvd":
        r = min(m, n)
        U = haar(m, r, gen)
        V = haar(n, r, gen)
        sigma = np.arange(1, r + 1, dtype=np.float64) ** (-exponent)
        return ((U * sigma) @ V.T).astype(np.float32), None
    A = gen.standard_normal((m, n)).astype(np.float32)
    x = gen.standard_normal(n)
    b = (A.astype(np.float64) @ x + noise_std * gen.standard_normal(m)).astype(np.float32)
    return A, b


def batch_problem_torch(spec, exponent=1.5, noise_std=math.sqrt(1e-3), device="cuda"):
    """The same recipe drawn on ``device`` with a seeded torch generator (for the full-size batch).  Haar
    factors come from the Q of a Cholesky QR of a Gaussian matrix, in FP64."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(spec["seed"])
    m, n = spec["m"], spec["n"]
    if spec["kind"] == "rsvd":
        r = min(m, n)

        def orth(rows):
            G = torch.randn(rows, r, generator=g, device=device, dtype=torch.float64)
            R = torch.linalg.cholesky(G.T @ G, upper=True)
            return torch.linalg.solve_triangular(R, G, upper=True, left=False)

        U, V = orth(m), orth(n)
        sigma = torch.arange(1, r + 1, device=device, dtype=torch.float64).pow(-exponent)
        return ((U * sigma) @ V.T).float().contiguous(), None
    A = torch.randn(m, n, generator=g, device=device, dtype=torch.float32)
    x = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    b = (A.double() @ x + noise_std * torch.randn(m, generator=g, device=device, dtype=torch.float64)).float()
    return A, b


def serve_pool(count=48, seed=0, m_range=(1000, 200000), n_range=(32, 1024)):
    """Resident problems of the served stream: m and n log-uniform on their ranges.  Returns (m, n) lists."""
    gen = rng(seed)
    m = np.exp(gen.uniform(math.log(m_range[0]), math.log(m_range[1]), count)).astype(np.int64)
    n = np.exp(gen.uniform(math.log(n_range[0]), math.log(n_range[1]), count)).astype(np.int64)
    return [int(v) for v in m], [int(v) for v in n]


def serve_arrivals(rate, window_s, pool_size, seed=0, lsr_share=0.6, ks=(8, 32, 64), p=8, q=1, s_factor=4):
    """A Poisson request stream over ``window_s`` seconds at ``rate`` requests/s: each request picks a resident
    problem uniformly, is least squares with probability lsr_share (count sketch, s = s_factor n) and a
    randomized k-SVD otherwise (k uniform on ks, oversampling p, q power iterations; k is cut so that k + p
    <= n).  Returns a list of dicts with the arrival time 't'."""
    gen = rng(seed)
    out, t = [], 0.0
    while True:
        t += gen.exponential(1.0 / rate)
        if t >= window_s:
            return out
        j = int(gen.integers(pool_size))
        if gen.uniform() < lsr_share:
            out.append(dict(t=t, pool=j, kind="lsr", s_factor=s_factor, seed=len(out)))
        else:
            out.append(dict(t=t, pool=j, kind="rsvd", k=int(gen.choice(ks)), p=p, q=q, seed=len(out)))
