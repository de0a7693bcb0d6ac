"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, step by step and end to end.

Tolerances (from the stated targets): hashes, signs, sample indices and Philox words bit-exact; FP32 sketches
within 1e-5 relative Frobenius error; rsvd top-k singular values within 1e-4 relative error and
||A - U S V^T||_F within 1% of the oracle's.
"""
import numpy as np
import pytest

from oracle import linalg, lsr, philox, rsvd, sketch
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    import paper_1505_07570_gb300 as rmc
    return rmc


def relfro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# ------------------------------------------------------------------------------------------------ a1 draws

@pytest.mark.parametrize("stream,instance,first,count", [(0, 0, 0, 1000), (2, 7, 2**32 - 3, 17), (3, 1, 123456789, 4096)])
def test_philox_words_bit_exact(R, stream, instance, first, count):
    seed = 0x0123456789ABCDEF
    got = R.rmc_philox(seed, stream, instance, first, count).cpu().numpy().astype(np.uint64)
    ref = philox.draw(np.arange(first, first + count, dtype=np.uint64), stream, seed, instance).astype(np.uint64)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("rows,cols", [(33, 7), (512, 256), (5, 1)])
def test_gaussian_matrix(R, rows, cols):
    got = R.rmc_gaussian_matrix(99, 3, rows, cols).cpu().numpy()
    ref = philox.gaussian_matrix(99, rows, cols, instance=3)
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=2e-6)


@pytest.mark.parametrize("m,s", [(1000, 7), (4096, 256), (3, 1), (70000, 4096)])
def test_countsketch_hash_bit_exact(R, m, s):
    b, g = R.rmc_countsketch_hash(5, 0, m, s)
    rb, rg = philox.countsketch_hash(5, m, s)
    np.testing.assert_array_equal(b.cpu().numpy(), rb)
    np.testing.assert_array_equal(g.cpu().numpy(), rg)


@pytest.mark.parametrize("N,s", [(16, 16), (16, 1), (2048, 256), (1 << 16, 1000), (1 << 20, 4096), (1000, 999)])
def test_srht_sample_bit_exact(R, N, s):
    got = R.rmc_srht_sample(77, 0, N, s).cpu().numpy()
    np.testing.assert_array_equal(got, philox.srht_sample(77, N, s))


# ------------------------------------------------------------------------------------------ a2-a4 sketches

SKETCH_CASES = [
    # (m, n, s, lda_pad): the small low-rank workload, ragged sizes, leading dimension > n, tiny corners
    (2048, 512, 256, 0),
    (1000, 37, 100, 3),
    (4097, 65, 300, 0),
    (5000, 1, 17, 0),
    (1, 4, 1, 0),
    (70000, 20, 128, 4),
    (20000, 9, 5000, 0),   # SRHT with s > 4096: one 4096-row block per work unit (no folding)
]


@pytest.mark.parametrize("kind", ["countsketch", "srht", "gaussian"])
@pytest.mark.parametrize("m,n,s,pad", SKETCH_CASES)
def test_sketch_parity(R, kind, m, n, s, pad):
    A = workloads.gaussian(m, n, seed=m + n)
    if m == 2048 and n == 512:
        A = workloads.lowrank()
    if kind == "srht" and s > sketch.next_pow2(m):
        pytest.skip("s > N")
    Ad = torch.zeros(m, n + pad, device="cuda")
    Ad[:, :n] = dev(A)
    C = R.rmc_sketch(Ad[:, :n], s, kind, seed=11)
    R.rmc_sync()
    ref = sketch.sketch(A, s, kind, 11)
    assert relfro(C.cpu().numpy(), ref) < 1e-5


def test_countsketch_deterministic(R):
    A = dev(workloads.gaussian(50000, 64, seed=1))
    C1 = R.rmc_sketch(A, 512, "countsketch", 3).clone()
    C2 = R.rmc_sketch(A, 512, "countsketch", 3)
    R.rmc_sync()
    assert torch.equal(C1, C2)


def test_srht_full_sample_orthogonal(R):
    """s = N: the SRHT is orthogonal, column norms are preserved."""
    A = workloads.gaussian(4096, 8, seed=4)
    C = R.rmc_sketch(dev(A), 4096, "srht", 1)
    R.rmc_sync()
    np.testing.assert_allclose(np.linalg.norm(C.cpu().numpy(), axis=0), np.linalg.norm(A, axis=0), rtol=1e-5)


def test_invalid_arguments(R):
    A = torch.zeros(100, 10, device="cuda")
    for args in [(A, 0, "gaussian", 1), (A, 129, "srht", 1)]:
        with pytest.raises(R.RmcError) as e:
            R.rmc_sketch(*args)
        assert e.value.status == R.RMC_EINVAL


# --------------------------------------------------------------------------------------------- a10 LSR

@pytest.mark.parametrize("kind", ["countsketch", "srht", "gaussian"])
@pytest.mark.parametrize("m,n,s", [(4000, 20, 200), (3000, 7, 3000), (20000, 64, 1024), (20000, 300, 1200)])
def test_lsr_parity(R, kind, m, n, s):
    A, b, _ = workloads.tall_lsr_numpy(m, n, seed=m + n)
    if kind == "srht" and s > sketch.next_pow2(m):
        pytest.skip("s > N")
    x = R.rmc_lsr_sketch(dev(A), dev(b), s, kind, seed=5)
    R.rmc_sync()
    xo = lsr.lsr_sketch(A, b, s, kind, 5)
    assert relfro(x.cpu().numpy(), xo) < 1e-4
    # The fit is as good as the oracle's.  In these high signal-to-noise regressions ||A x - b|| is small next
    # to ||A|| ||x||, so the FP32 rounding of S^T A (the Gaussian sketch sums m products per entry) moves the
    # residual ratio by up to ~1e-4 at n = 300 even with x within 1e-4 of the oracle's; stated as 1e-3.
    xs = lsr.lsr_exact(A, b)
    assert lsr.residual_ratio(A, b, x.cpu().numpy(), xs) <= lsr.residual_ratio(A, b, xo, xs) * (1 + 1e-3)


@pytest.mark.parametrize("n", [317, 700, 1024])
def test_lsr_large_n(R, n):
    """n above the shared-memory packed factor: the blocked multi-CTA FP32 factorization and refinement."""
    m, s = 6 * n, 4 * n
    A, b, _ = workloads.tall_lsr_numpy(m, n, seed=n)
    x = R.rmc_lsr_sketch(dev(A), dev(b), s, "countsketch", seed=8)
    R.rmc_sync()
    xo = lsr.lsr_sketch(A, b, s, "countsketch", 8)
    assert relfro(x.cpu().numpy(), xo) < 1e-4


@pytest.mark.parametrize("n", [33, 250, 256])
def test_lsr_single_cta_factor(R, n):
    """n <= 256: the factorization, R^-1 and M = R^-1 R^-T in one CTA's shared memory (ragged and full last
    32-column block)."""
    m, s = 8 * n, 4 * n
    A, b, _ = workloads.tall_lsr_numpy(m, n, seed=n + 1)
    x = R.rmc_lsr_sketch(dev(A), dev(b), s, "countsketch", seed=11)
    R.rmc_sync()
    xo = lsr.lsr_sketch(A, b, s, "countsketch", 11)
    assert relfro(x.cpu().numpy(), xo) < 1e-4


def test_lsr_noise_free_exact(R):
    A, _, xt = workloads.tall_lsr_numpy(5000, 12, seed=3, noise_std=0.0)
    b = (A.astype(np.float64) @ xt).astype(np.float32)
    x = R.rmc_lsr_sketch(dev(A), dev(b), 400, "countsketch", 9)
    R.rmc_sync()
    assert relfro(x.cpu().numpy(), xt) < 1e-5


# -------------------------------------------------------------------------------- a5-a9 rsvd and its steps

@pytest.mark.parametrize("m,n,l", [(2048, 512, 20), (1000, 300, 33), (70000, 200, 120)])
def test_matmuls(R, m, n, l):
    A = workloads.gaussian(m, n, 1)
    X1 = workloads.gaussian(n, l, 2)
    X2 = workloads.gaussian(m, l, 3)
    Y = R.rmc_matmul_an(dev(A), dev(X1))
    W = R.rmc_matmul_at(dev(A), dev(X2))
    R.rmc_sync()
    A64 = A.astype(np.float64)
    assert relfro(Y.cpu().numpy(), A64 @ X1) < 1e-5
    assert relfro(W.cpu().numpy(), X2.astype(np.float64).T @ A64) < 1e-5


@pytest.mark.parametrize("m,l", [(2048, 20), (5000, 33), (65536, 120), (300, 256)])
def test_cholqr2(R, m, l):
    Y = workloads.gaussian(m, l, 7) * np.linspace(1, 100, l).astype(np.float32)
    Yd = dev(Y)
    Rg = R.rmc_cholqr2(Yd)
    R.rmc_sync()
    Q = Yd.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(Q.T @ Q, np.eye(l), atol=5e-6)
    assert relfro(Q @ Rg.cpu().numpy(), Y) < 1e-5
    _, Rh = linalg.householder_qr(Y.astype(np.float64))
    Rh = Rh * np.sign(np.diag(Rh))[:, None]
    assert relfro(Rg.cpu().numpy(), Rh) < 1e-5


@pytest.mark.parametrize("l,n", [(20, 512), (24, 100), (120, 4000)])
def test_svd_wide(R, l, n):
    B = workloads.gaussian(l, n, 8) * np.linspace(0.1, 10, l).astype(np.float32)[:, None]
    Ub, s, Vb = R.rmc_svd_wide(dev(B))
    R.rmc_sync()
    _, so, _ = linalg.jacobi_svd(B.astype(np.float64))
    np.testing.assert_allclose(s.cpu().numpy(), so, rtol=1e-5)
    rec = (Ub.cpu().numpy().astype(np.float64) * s.cpu().numpy()) @ Vb.cpu().numpy().T
    # l > 32 rotates in FP32 (orthogonality tolerance 4 eps sqrt(l)), l <= 32 in FP64
    assert relfro(rec, B) < (3e-5 if l > 32 else 1e-5)


def test_rsvd_lowrank_workload(R):
    """The small workload: 2048 x 512, sigma_i = 0.9^i + noise, k = 10, p = 10, q = 2."""
    A = workloads.lowrank()
    U, s, V = R.rmc_rsvd(dev(A), 10, 10, 2, seed=0)
    R.rmc_sync()
    Uo, so, Vo, _ = rsvd.rsvd(A, 10, 10, 2, 0)
    np.testing.assert_allclose(s.cpu().numpy(), so, rtol=1e-4)
    A64 = A.astype(np.float64)
    err = np.linalg.norm(A64 - (U.cpu().numpy() * s.cpu().numpy()) @ V.cpu().numpy().T)
    erro = np.linalg.norm(A64 - (Uo * so) @ Vo.T)
    assert abs(err - erro) <= 0.01 * erro
    # same singular subspaces (the spectrum is well separated at the top)
    assert np.all(np.abs(np.sum(U.cpu().numpy() * Uo, axis=0)) > 0.999)


@pytest.mark.parametrize("q", [0, 1])
def test_rsvd_exact_rank(R, q):
    """A rank-k matrix is recovered (Sec. 5.2 derivation: range(A Omega) = range(A)) up to FP32 rounding."""
    A = workloads.exact_rank(3000, 400, 8, seed=2, sigma=np.linspace(5, 1, 8))
    U, s, V = R.rmc_rsvd(dev(A), 8, 0, q, seed=4)
    R.rmc_sync()
    np.testing.assert_allclose(s.cpu().numpy(), np.linspace(5, 1, 8), rtol=1e-4)


# --------------------------------------------------------------------------- a2 on the tensor cores (TF32)
# TF32 keeps 10 mantissa bits: the sketch is compared at 2e-3 relative Frobenius error (the truncation of A
# to TF32 alone shrinks entries by ~2^-11 on average), and least squares at the accuracy that implies.

# n = 257 and 513: the column past the last full 256-column tile is folded in by the drawing warps
@pytest.mark.parametrize("m,n,s,pad", [(2048, 512, 256, 0), (4097, 65, 300, 0), (70000, 20, 128, 4),
                                       (1000, 37, 100, 3), (1, 4, 1, 0), (300000, 256, 1024, 0),
                                       (5000, 257, 600, 3), (3001, 513, 256, 3)])
def test_gaussian_tf32_parity(R, m, n, s, pad):
    A = workloads.lowrank() if (m, n) == (2048, 512) else workloads.gaussian(m, n, seed=m + n)
    Ad = torch.zeros(m, n + pad, device="cuda")
    Ad[:, :n] = dev(A)
    C = R.rmc_sketch(Ad[:, :n], s, "gaussian", seed=11, prec="tf32")
    R.rmc_sync()
    ref = sketch.sketch(A, s, "gaussian", 11)
    assert relfro(C.cpu().numpy(), ref) < 2e-3


def test_gaussian_tf32_unaligned_rows_take_fp32_kernel(R):
    """Rows that are not 16-byte aligned (n = 5) cannot be streamed by TMA: the FP32 kernel runs instead and
    meets the FP32 tolerance."""
    A = workloads.gaussian(3000, 5, seed=2)
    C = R.rmc_sketch(dev(A), 300, "gaussian", 1, prec="tf32")
    R.rmc_sync()
    assert relfro(C.cpu().numpy(), sketch.sketch(A, 300, "gaussian", 1)) < 1e-5


@pytest.mark.parametrize("m,n,s", [(20000, 64, 1024), (4000, 20, 200)])
def test_lsr_gaussian_tf32(R, m, n, s):
    A, b, _ = workloads.tall_lsr_numpy(m, n, seed=m + n)
    x = R.rmc_lsr_sketch(dev(A), dev(b), s, "gaussian", seed=5, prec="tf32")
    R.rmc_sync()
    xo = lsr.lsr_sketch(A, b, s, "gaussian", 5)
    assert relfro(x.cpu().numpy(), xo) < 1e-2
    # In this high signal-to-noise regression the TF32 rounding of S^T A is of the order of the noise, so the
    # residual ratio ||A x - b||^2 / ||A x* - b||^2 is stated within 10% of the FP64 oracle's.
    xs = lsr.lsr_exact(A, b)
    assert lsr.residual_ratio(A, b, x.cpu().numpy(), xs) <= lsr.residual_ratio(A, b, xo, xs) * 1.10


# ------------------------------------------------ BF16 operands (kind::f16): the sketch and the products with A
# BF16 keeps 8 mantissa bits: rounding both operands of every product gives a relative error of about
# 2^-9 sqrt(2/3) = 1.6e-3, also for a sum of random-sign products; sketches and products are tested at 5e-3.

@pytest.mark.parametrize("m,n,s,pad", [(2048, 512, 256, 0), (4097, 64, 300, 0), (70000, 20, 128, 4),
                                       (1000, 36, 100, 4), (1, 4, 1, 0), (300000, 256, 1024, 0), (130, 260, 513, 0),
                                       (5000, 257, 600, 3)])
def test_gaussian_bf16_parity(R, m, n, s, pad):
    A = workloads.lowrank() if (m, n) == (2048, 512) else workloads.gaussian(m, n, seed=m + n)
    Ad = torch.zeros(m, n + pad, device="cuda")
    Ad[:, :n] = dev(A)
    C = R.rmc_sketch(Ad[:, :n], s, "gaussian", seed=11, prec="bf16")
    R.rmc_sync()
    ref = sketch.sketch(A, s, "gaussian", 11)
    assert relfro(C.cpu().numpy(), ref) < 5e-3


@pytest.mark.parametrize("m,n,s", [(20000, 64, 1024), (4000, 20, 200)])
def test_lsr_gaussian_bf16(R, m, n, s):
    """An FP64 emulation of these sketches with both operands rounded to BF16 gives x within 7e-4 of the
    oracle's and a residual ratio ||A x - b||^2 / ||A x* - b||^2 of 1.30 and 1.14 against the oracle's 1.08 and
    1.10 (BF16's rounding of S^T A is several times this regression's noise): stated as x within 1e-2 and the
    ratio within 1.5 times the oracle's."""
    A, b, _ = workloads.tall_lsr_numpy(m, n, seed=m + n)
    x = R.rmc_lsr_sketch(dev(A), dev(b), s, "gaussian", seed=5, prec="bf16")
    R.rmc_sync()
    xo = lsr.lsr_sketch(A, b, s, "gaussian", 5)
    assert relfro(x.cpu().numpy(), xo) < 1e-2
    xs = lsr.lsr_exact(A, b)
    assert lsr.residual_ratio(A, b, x.cpu().numpy(), xs) <= lsr.residual_ratio(A, b, xo, xs) * 1.5


@pytest.mark.parametrize("m,n,l", [(2048, 512, 20), (1000, 300, 33), (70000, 200, 120), (4096, 1000, 200),
                                   (333, 4100, 64), (5000, 260, 256), (100, 64, 8)])
def test_matmuls_bf16(R, m, n, l):
    A = workloads.gaussian(m, n, 1)
    X1 = workloads.gaussian(n, l, 2)
    X2 = workloads.gaussian(m, l, 3)
    Y = R.rmc_matmul_an(dev(A), dev(X1), prec="bf16")
    W = R.rmc_matmul_at(dev(A), dev(X2), prec="bf16")
    R.rmc_sync()
    A64 = A.astype(np.float64)
    assert relfro(Y.cpu().numpy(), A64 @ X1) < 5e-3
    assert relfro(W.cpu().numpy(), X2.astype(np.float64).T @ A64) < 5e-3


def test_rsvd_bf16_factor_rank_workload(R):
    """An FP64 emulation of this rSVD with every product's operands rounded to BF16 puts sigma within 1.0e-4
    (q = 1) of the oracle's; the tensor core's truncating FP32 accumulation adds to it: stated as 2e-3, and the
    projection error ||A - U S V^T||_F within 1% of the oracle's."""
    A = workloads.factor_rank_numpy(4096, 2048, 256, seed=3)
    k, p, q = 20, 10, 1
    U, s, V = R.rmc_rsvd(dev(A), k, p, q, seed=7, prec="bf16")
    R.rmc_sync()
    Uo, so, Vo, _ = rsvd.rsvd(A, k, p, q, 7)
    np.testing.assert_allclose(s.cpu().numpy(), so, rtol=2e-3)
    A64 = A.astype(np.float64)
    err = np.linalg.norm(A64 - (U.cpu().numpy() * s.cpu().numpy()) @ V.cpu().numpy().T)
    erro = np.linalg.norm(A64 - (Uo * so) @ Vo.T)
    assert abs(err - erro) <= 0.01 * erro


@pytest.mark.parametrize("m,s", [(100, 64), (333, 1000)])
def test_gaussian_draw_floor_draws_the_sketch_operator(R, m, s):
    """The drawing-bound kernel draws exactly the normals of the sketch's operator: their sum matches the
    oracle's FP64 matrix up to the TF32 rounding (2^-11 relative) and the approximate special functions."""
    got = float(R.rmc_gaussian_draw_floor(m, s, 21).item())
    R.rmc_sync()
    G = philox.sketch_gaussian_matrix(21, m, s)
    assert abs(got - G.sum()) <= 1e-3 * np.abs(G).sum()


def test_lsr_ill_conditioned_falls_back_to_fp64(R):
    """cond(S^T A) ~ 1e5 squares to ~1e10 in the Gram matrix, beyond FP32: the FP32 Cholesky meets a
    non-positive pivot and the FP64 factorization takes over; the fit stays as good as the oracle's."""
    A, b, _ = workloads.tall_lsr_numpy(6000, 10, seed=3, noise_std=1.0)
    A[:, 9] = A[:, 8] + 1e-5 * A[:, 7]
    x = R.rmc_lsr_sketch(dev(A), dev(b), 600, "countsketch", seed=2)
    R.rmc_sync()
    xo = lsr.lsr_sketch(A, b, 600, "countsketch", 2)
    xs = lsr.lsr_exact(A, b)
    assert np.all(np.isfinite(x.cpu().numpy()))
    assert lsr.residual_ratio(A, b, x.cpu().numpy(), xs) <= lsr.residual_ratio(A, b, xo, xs) * (1 + 1e-3)


def test_cholqr2_ill_conditioned_falls_back_to_fp64(R):
    Y = workloads.gaussian(4000, 16, 7) * np.logspace(0, 4.5, 16).astype(np.float32)
    Yd = dev(Y)
    R.rmc_cholqr2(Yd, want_r=False)
    R.rmc_sync()
    Q = Yd.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(Q.T @ Q, np.eye(16), atol=1e-4)


# ------------------------------------------------------------------ a5-a7 on the tensor cores (TF32)

@pytest.mark.parametrize("prec,tol", [("tf32", 2e-3), ("tf32x3", 5e-5)])
@pytest.mark.parametrize("m,n,l", [(2048, 512, 20), (1000, 300, 33), (70000, 200, 120), (4096, 1000, 200),
                                   (333, 4100, 64), (5000, 260, 256)])
def test_matmuls_tf32(R, m, n, l, prec, tol):
    """TF32 keeps 10 mantissa bits (2e-3).  3xTF32 splits every operand into a TF32 head and remainder, so each
    product is good to ~2^-21, but the tensor core adds every k-step into its FP32 accumulator without
    round-to-nearest and that error grows with the chain (capped at 4096 terms): stated as 5e-5."""
    A = workloads.gaussian(m, n, 1)
    X1 = workloads.gaussian(n, l, 2)
    X2 = workloads.gaussian(m, l, 3)
    Y = R.rmc_matmul_an(dev(A), dev(X1), prec=prec)
    W = R.rmc_matmul_at(dev(A), dev(X2), prec=prec)
    R.rmc_sync()
    A64 = A.astype(np.float64)
    assert relfro(Y.cpu().numpy(), A64 @ X1) < tol
    assert relfro(W.cpu().numpy(), X2.astype(np.float64).T @ A64) < tol


@pytest.mark.parametrize("prec", ["fp32", "tf32", "tf32x3"])
def test_rsvd_factor_rank_workload(R, prec):
    """A = G1 diag(1/i) G2^T (Gaussian factors), the large-rSVD recipe at a size the oracle runs."""
    A = workloads.factor_rank_numpy(4096, 2048, 256, seed=3)
    k, p, q = 20, 10, 1
    U, s, V = R.rmc_rsvd(dev(A), k, p, q, seed=7, prec=prec)
    R.rmc_sync()
    _, so, _, _ = rsvd.rsvd(A, k, p, q, 7)
    tol = 2e-3 if prec == "tf32" else 1e-4
    np.testing.assert_allclose(s.cpu().numpy(), so, rtol=tol)
    A64 = A.astype(np.float64)
    err = np.linalg.norm(A64 - (U.cpu().numpy() * s.cpu().numpy()) @ V.cpu().numpy().T)
    Uo, so, Vo, _ = rsvd.rsvd(A, k, p, q, 7)
    erro = np.linalg.norm(A64 - (Uo * so) @ Vo.T)
    assert abs(err - erro) <= 0.01 * erro


# ------------------------------------------------------- the small factorizations: FP32 default, FP64 option

@pytest.fixture
def small_fp64(R):
    R.rmc_set_option(R.RMC_OPT_SMALL_FP64, 1)
    yield
    R.rmc_set_option(R.RMC_OPT_SMALL_FP64, 0)


@pytest.mark.parametrize("l,n", [(120, 4000), (32, 300), (64, 2000)])
def test_svd_wide_fp64_option(R, small_fp64, l, n):
    """RMC_OPT_SMALL_FP64: FP64 Gram products, Cholesky and Jacobi rotations.  The singular values of the FP32
    input are then limited by the FP32 storage of the CholeskyQR2 basis (about 1e-7), not by the rotations."""
    assert R.rmc_get_option(R.RMC_OPT_SMALL_FP64) == 1
    B = workloads.gaussian(l, n, 8) * np.logspace(0, 3, l).astype(np.float32)[:, None]
    Ub, s, Vb = R.rmc_svd_wide(dev(B))
    R.rmc_sync()
    _, so, _ = linalg.jacobi_svd(B.astype(np.float64))
    np.testing.assert_allclose(s.cpu().numpy(), so, rtol=1e-6)
    rec = (Ub.cpu().numpy().astype(np.float64) * s.cpu().numpy()) @ Vb.cpu().numpy().T
    assert relfro(rec, B) < 1e-5


@pytest.mark.parametrize("l,n", [(200, 3000), (240, 2048)])
def test_svd_wide_large_l(R, l, n):
    """l above 128 (block Lanczos bases): the eight-lanes-per-pair Jacobi keeps W in shared memory up to
    l = 240 in FP32.  Each column then takes about l x sweeps FP32 rotations, whose roundings add up to ~2e-5
    relative in sigma at l = 200-240: stated as 5e-5, inside the 1e-4 target of the k-SVD."""
    B = workloads.gaussian(l, n, 9) * np.linspace(0.5, 20, l).astype(np.float32)[:, None]
    Ub, s, Vb = R.rmc_svd_wide(dev(B))
    R.rmc_sync()
    _, so, _ = linalg.jacobi_svd(B.astype(np.float64))
    np.testing.assert_allclose(s.cpu().numpy(), so, rtol=5e-5)
    # Ub = R^T M diag(sigma)^-1: column j is good to about eps * sigma_1 / sigma_j, so the leading half (what a
    # k-SVD keeps) is orthonormal to FP32 level; the reconstruction uses every column
    Ubh = Ub.cpu().numpy().astype(np.float64)
    h = l // 2
    np.testing.assert_allclose(Ubh[:, :h].T @ Ubh[:, :h], np.eye(h), atol=1e-4)
    rec = (Ubh * s.cpu().numpy()) @ Vb.cpu().numpy().T
    assert relfro(rec, B) < 1e-4


def test_rsvd_fp64_option_matches_oracle(R, small_fp64):
    A = workloads.factor_rank_numpy(4096, 2048, 256, seed=3)
    U, s, V = R.rmc_rsvd(dev(A), 100, 20, 1, seed=7, prec="tf32x3")
    R.rmc_sync()
    _, so, _, _ = rsvd.rsvd(A, 100, 20, 1, 7)
    np.testing.assert_allclose(s.cpu().numpy(), so, rtol=1e-4)


def test_cholqr2_fp64_option(R, small_fp64):
    Y = workloads.gaussian(20000, 120, 7) * np.logspace(0, 4, 120).astype(np.float32)
    Yd = dev(Y)
    Rg = R.rmc_cholqr2(Yd)
    R.rmc_sync()
    Q = Yd.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(Q.T @ Q, np.eye(120), atol=5e-6)
    assert relfro(Q @ Rg.cpu().numpy(), Y) < 1e-5


def test_set_option_rejects_unknown(R):
    with pytest.raises(R.RmcError):
        R.rmc_set_option(99, 1)
    with pytest.raises(R.RmcError):
        R.rmc_set_option(R.RMC_OPT_SMALL_FP64, 2)


@pytest.mark.parametrize("q", [0, 1])
def test_rsvd_square_ill_conditioned_omega(R, q):
    """l = n = 33 makes Omega a square Gaussian; with this seed it is ill-conditioned enough that the Gram matrix
    of A Omega with FP32 products is indefinite.  The FP32 Cholesky fails, the Gram matrix is formed again with
    FP64 products and factored in FP64 (a served request once returned RMC_ENUMERIC here).  Q spans range(A), so
    the singular values are A's own."""
    A = workloads.gaussian(20000, 33, seed=77)
    U, s, V = R.rmc_rsvd(dev(A), 25, 8, q, seed=4317)
    R.rmc_sync()
    _, so, _, _ = rsvd.rsvd(A, 25, 8, q, 4317)
    np.testing.assert_allclose(s.cpu().numpy(), so, rtol=1e-4)
    np.testing.assert_allclose(so, np.linalg.svd(A.astype(np.float64), compute_uv=False)[:25], rtol=1e-10)
