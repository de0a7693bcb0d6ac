"""Parity of the CUDA path with the FP64 oracle for the calls beyond the three of the boundary: machine-precision
least squares (Algorithm 4.1) and the block Lanczos k-SVD (Algorithm 5.1).

Tolerances: machine-precision least squares reaches x* = A^+ b of the FP32 inputs within 1e-10 relative (the
point of Algorithm 4.1; its starting point, the sketch-and-solve solution, is compared at the FP32-sketch
tolerance 1e-4 of the sketch-and-solve tests); block Lanczos singular values within 1e-4 relative of the
oracle's and ||A - U S V^T||_F within 1% of the oracle's (the rsvd targets).
"""
import numpy as np
import pytest

from oracle import lsr, rsvd
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


# ------------------------------------------------------------------------------------ Algorithm 4.1

@pytest.mark.parametrize("kind", ["countsketch", "srht", "gaussian"])
@pytest.mark.parametrize("m,n,s", [(4000, 20, 400), (20000, 64, 1024), (20001, 37, 600), (12000, 256, 4096)])
def test_lsr_precise_reaches_the_exact_solution(R, kind, m, n, s):
    A, b, _ = workloads.tall_lsr_numpy(m, n, seed=m + n)
    x, it = R.rmc_lsr_precise(dev(A), dev(b), s, kind, seed=5, max_iters=60, tol=1e-15, want_iters=True)
    R.rmc_sync()
    xs = lsr.lsr_exact(A, b)
    assert relfro(x.cpu().numpy(), xs) < 1e-10
    assert 1 <= int(it.item()) <= 60


@pytest.mark.parametrize("kind", ["countsketch", "srht", "gaussian"])
def test_lsr_precise_starts_from_the_sketched_solution(R, kind):
    """Zero steps: x = T z0 = R^-1 Q^T S^T b, the sketch-and-solve solution of Sec. 4.2."""
    A, b, _ = workloads.tall_lsr_numpy(5000, 24, seed=3)
    x = R.rmc_lsr_precise(dev(A), dev(b), 500, kind, seed=7, max_iters=0)
    R.rmc_sync()
    assert relfro(x.cpu().numpy(), lsr.lsr_sketch(A, b, 500, kind, 7)) < 1e-4


def test_lsr_precise_follows_the_oracle_iteration(R):
    """A fixed step and a fixed number of steps, no early exit: the error x_t - x* shrinks as the oracle's does
    (same sketch, same theta; the iterates differ only through the FP32 rounding of the sketch)."""
    A, b, _ = workloads.tall_lsr_numpy(8000, 16, seed=11)
    xs = lsr.lsr_exact(A, b)
    for t in (1, 3, 6):
        x = R.rmc_lsr_precise(dev(A), dev(b), 400, "gaussian", seed=2, theta=0.6, max_iters=t, tol=0.0)
        R.rmc_sync()
        xo = lsr.lsr_precise(A, b, 400, "gaussian", 2, theta=0.6, iters=t)
        eg, eo = relfro(x.cpu().numpy(), xs), relfro(xo, xs)
        assert abs(eg - eo) <= 0.05 * eo + 1e-12, (t, eg, eo)


def test_lsr_precise_strided_rows(R):
    """lda > n (and so the scalar-load pass when the pitch breaks 16-byte alignment)."""
    A, b, _ = workloads.tall_lsr_numpy(9000, 32, seed=4)
    for pad in (3, 4):
        Ad = torch.zeros(9000, 32 + pad, device="cuda")
        Ad[:, :32] = dev(A)
        x = R.rmc_lsr_precise(Ad[:, :32], dev(b), 512, "countsketch", seed=1, max_iters=60)
        R.rmc_sync()
        assert relfro(x.cpu().numpy(), lsr.lsr_exact(A, b)) < 1e-10


def test_lsr_precise_rejects_bad_arguments(R):
    A = torch.zeros(1000, 300, device="cuda")
    b = torch.zeros(1000, device="cuda")
    with pytest.raises(R.RmcError):
        R.rmc_lsr_precise(A, b, 600, "gaussian", 1)          # n > 256
    A = torch.zeros(1000, 30, device="cuda")
    with pytest.raises(R.RmcError):
        R.rmc_lsr_precise(A, b, 20, "gaussian", 1)           # s < n


# ------------------------------------------------------------------------------------ Algorithm 5.1

@pytest.mark.parametrize("prec", ["fp32", "tf32", "tf32x3"])
@pytest.mark.parametrize("m,n,k,s,q", [(3000, 800, 10, 20, 3), (2048, 512, 10, 12, 4), (5001, 301, 8, 16, 2)])
def test_block_lanczos_parity(R, prec, m, n, k, s, q):
    A = workloads.factor_rank_numpy(m, n, 200, seed=m + q)
    U, sg, V = R.rmc_block_lanczos(dev(A), k, s, q, seed=3, prec=prec)
    R.rmc_sync()
    Uo, so, Vo, _ = rsvd.block_lanczos(A, k, s, q, 3)
    tol = 2e-3 if prec == "tf32" else 1e-4
    np.testing.assert_allclose(sg.cpu().numpy(), so, rtol=tol)
    A64 = A.astype(np.float64)
    err = np.linalg.norm(A64 - (U.cpu().numpy() * sg.cpu().numpy()) @ V.cpu().numpy().T)
    erro = np.linalg.norm(A64 - (Uo * so) @ Vo.T)
    assert abs(err - erro) <= 0.01 * erro
    Ug = U.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(Ug.T @ Ug, np.eye(k), atol=1e-4)


def test_block_lanczos_recovers_an_exact_rank_matrix(R):
    sig = np.linspace(5, 1, 8)
    A = workloads.exact_rank(3000, 400, 8, seed=2, sigma=sig)
    U, s, V = R.rmc_block_lanczos(dev(A), 8, 4, 2, seed=4)
    R.rmc_sync()
    np.testing.assert_allclose(s.cpu().numpy(), sig, rtol=1e-4)


def test_block_lanczos_one_block_is_rsvd(R):
    A = workloads.lowrank(2048, 512)
    _, s1, _ = R.rmc_block_lanczos(dev(A), 10, 20, 1, seed=0)
    _, s2, _ = R.rmc_rsvd(dev(A), 10, 10, 0, seed=0)
    R.rmc_sync()
    np.testing.assert_allclose(s1.cpu().numpy(), s2.cpu().numpy(), rtol=1e-5)


def test_block_lanczos_converges_toward_lapack(R):
    """Block Lanczos reaches the top singular values to FP32 accuracy with a few blocks (Sec. 5.1)."""
    A = workloads.factor_rank_numpy(3000, 600, 300, seed=8)
    sv = np.linalg.svd(A.astype(np.float64), compute_uv=False)[:10]
    _, s, _ = R.rmc_block_lanczos(dev(A), 10, 20, 6, seed=1)
    R.rmc_sync()
    np.testing.assert_allclose(s.cpu().numpy(), sv, rtol=1e-4)


# ---------------------------------------------------------------------- Sec. 3.2.4 and Algorithm 5.3

@pytest.mark.parametrize("m,n,s,pad", [(300, 2000, 64, 0), (1000, 1030, 200, 3), (17, 5, 3, 0), (2049, 4096, 256, 0)])
def test_countsketch_columns_parity(R, m, n, s, pad):
    from oracle import sketch
    A = workloads.gaussian(m, n, seed=n)
    Ad = torch.zeros(m, n + pad, device="cuda")
    Ad[:, :n] = dev(A)
    C = R.rmc_countsketch_columns(Ad[:, :n], s, seed=13, instance=1)
    R.rmc_sync()
    assert relfro(C.cpu().numpy(), sketch.countsketch_columns(A, s, 13, instance=1)) < 1e-6


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
@pytest.mark.parametrize("m,n,k,s,p_cs,p", [(3000, 800, 10, 40, 600, 160), (4096, 2048, 20, 64, 1500, 300)])
def test_rsvd_fast_parity(R, prec, m, n, k, s, p_cs, p):
    A = workloads.factor_rank_numpy(m, n, 300, seed=m + k)
    U, sg, V = R.rmc_rsvd_fast(dev(A), k, s, p_cs, p, seed=9, prec=prec)
    R.rmc_sync()
    Uo, so, Vo = rsvd.faster_rsvd(A, k, s, p_cs, p, 9)
    tol = 1e-4 if prec == "fp32" else 3e-3
    np.testing.assert_allclose(sg.cpu().numpy(), so, rtol=tol)
    A64 = A.astype(np.float64)
    err = np.linalg.norm(A64 - (U.cpu().numpy() * sg.cpu().numpy()) @ V.cpu().numpy().T)
    erro = np.linalg.norm(A64 - (Uo * so) @ Vo.T)
    assert abs(err - erro) <= 0.01 * erro
    if prec == "fp32":
        np.testing.assert_allclose(np.abs(np.sum(V.cpu().numpy() * Vo, axis=0)), 1.0, atol=1e-3)


def test_rsvd_fast_recovers_an_exact_rank_matrix(R):
    """rank(A) = k = s: C = A S spans range(A) and D = P^T C has full column rank, so R_D is invertible (the GPU
    form inverts R_D where the listing takes pinv; a sketch of exactly deficient rank reports RMC_ENUMERIC)."""
    sig = np.linspace(5, 1, 8)
    A = workloads.exact_rank(3000, 400, 8, seed=2, sigma=sig)
    U, s, V = R.rmc_rsvd_fast(dev(A), 8, 8, 256, 64, seed=4)
    R.rmc_sync()
    np.testing.assert_allclose(s.cpu().numpy(), sig, rtol=1e-4)


# -------------------------------------------------------------------------------------------- Sec. 6.4

@pytest.mark.parametrize("n1,n2,d,sigma", [(300, 70, 5, 1.3), (1000, 256, 33, 4.0), (65, 1, 1, 0.5)])
def test_rbf_parity(R, n1, n2, d, sigma):
    from oracle import kernel
    g = np.random.default_rng(n1)
    X = g.standard_normal((n1, d)).astype(np.float32)
    Y = g.standard_normal((n2, d)).astype(np.float32)
    K = R.rmc_rbf(dev(X), dev(Y), sigma)
    R.rmc_sync()
    np.testing.assert_allclose(K.cpu().numpy(), kernel.rbf(X, Y, sigma), rtol=2e-5, atol=1e-6)


@pytest.mark.parametrize("n,d,s,sigma", [(500, 8, 40, 2.0), (20000, 16, 128, 4.0), (3001, 3, 25, 1.0)])
def test_nystrom_parity(R, n, d, s, sigma):
    """L against the oracle's (each column's sign is a reproducibility rule only, so columns are compared up to
    sign), the landmark eigenvalues, and L L^T against the oracle's C W_k^+ C^T on sampled entries."""
    from oracle import kernel
    X = np.random.default_rng(n).standard_normal((n, d)).astype(np.float32)
    L, lam, idx = R.rmc_nystrom(dev(X), sigma, s, seed=21)
    R.rmc_sync()
    Lo, So, lamo, _ = kernel.nystrom(X, sigma, s, 21)
    np.testing.assert_array_equal(idx.cpu().numpy(), So)
    np.testing.assert_allclose(lam.cpu().numpy(), lamo, rtol=1e-4, atol=1e-6 * lamo[0])
    Lg = L.cpu().numpy().astype(np.float64)
    sgn = np.sign(np.sum(Lg * Lo, axis=0))
    # the small eigenvalues of W carry the FP32 rounding of W divided by lam: compare relative to the column norm
    err = np.linalg.norm(Lg * sgn - Lo, axis=0) / np.linalg.norm(Lo, axis=0)
    assert np.all(err < 2e-3 * np.sqrt(lamo[0] / lamo)), err
    rows = np.random.default_rng(1).choice(n, 50, replace=False)
    np.testing.assert_allclose(Lg[rows] @ Lg[rows].T, Lo[rows] @ Lo[rows].T, atol=1e-3)
