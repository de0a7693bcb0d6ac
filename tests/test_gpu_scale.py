"""Parity at the benchmark sizes, in the configuration bench.py times.

* The tall regression workload (A 1,048,576 x 256 FP32 with lognormal row scales, b = A x* + noise), sketched
  to s = 4096 by each kind: sampled rows of C against the oracle's row-by-row forms (the Gaussian rows from
  their own Philox draws, the SRHT rows from the definition (H_N)[r, i] = (-1)^popcount(r & i)), the whole
  count sketch against the oracle's count sketch.  The sketch-and-solve x of every kind against the FP64
  least-squares solution of the same FP32 sketch [S^T A, S^T b] (read back from rmc_sketch of [A, b]); with
  the sketch itself pinned row by row above, that closes the chain to the oracle without an FP64 Gaussian
  sketch of the whole matrix (2^20 x 4096 normals).
* The large randomized-SVD workload (A = G1 diag(1/i) G2^T, 65,536 x 16,384, rank 2048; k = 100, p = 20,
  q = 0, 1, 2) against the oracle's rsvd on the same FP32 bits: top-k singular values within 1e-4 relative
  (FP32 products) and ||A - Q Q^T A||_F within 1% of the oracle's.
Tolerances: 1e-5 relative Frobenius for FP32 sketches, 2e-3 for TF32 (each operand keeps 10 mantissa bits).
"""
import numpy as np
import pytest

from oracle import linalg, philox, rsvd, sketch
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SEED = 20150527          # the benchmark's seed
M, N = 1 << 20, 256


@pytest.fixture(scope="module")
def R():
    import paper_1505_07570_gb300 as rmc
    return rmc


def relfro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def tall():
    """The benchmark's inputs (rank 0 of bench.py) on the device and their FP32 bits on the host."""
    A, b, _ = workloads.tall_lsr_torch(M, N, seed=SEED)
    Ab = torch.cat([A, b[:, None]], dim=1).contiguous()      # [A, b]: 257 columns
    return A, b, Ab, Ab.cpu().numpy()


# rows of the s = 4096 sketch checked one by one: four Philox groups of the Gaussian (16 rows), spread SRHT rows
GAUSS_ROWS = [4 * g + j for g in (0, 317, 640, 1023) for j in range(4)]
SRHT_POS = [0, 1, 777, 2048, 3000, 4095]


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("tf32", 2e-3), ("bf16", 5e-3)])
def test_gaussian_sketch_full_size_sampled_rows(R, tall, prec, tol):
    _, _, Ab, Ab_h = tall
    C = R.rmc_sketch(Ab, 4096, "gaussian", SEED, prec=prec)
    R.rmc_sync()
    got = C[GAUSS_ROWS].cpu().numpy()
    ref = sketch.gaussian_sketch_rows(Ab_h, 4096, SEED, GAUSS_ROWS)
    assert relfro(got, ref) < tol
    assert bool(torch.isfinite(C).all())


def test_srht_sketch_full_size_sampled_rows(R, tall):
    _, _, Ab, Ab_h = tall
    C = R.rmc_sketch(Ab, 4096, "srht", SEED)
    R.rmc_sync()
    got = C[SRHT_POS].cpu().numpy()
    ref = sketch.srht_sketch_rows(Ab_h, 4096, SEED, SRHT_POS)
    assert relfro(got, ref) < 1e-5
    # every row: the SRHT at s <= N keeps column norms in expectation; at s = 4096 within a few percent
    norms = np.linalg.norm(C.cpu().numpy(), axis=0) / np.linalg.norm(Ab_h.astype(np.float64), axis=0)
    assert np.all(np.abs(norms - 1) < 0.1)


def test_countsketch_full_size_whole(R, tall):
    _, _, Ab, Ab_h = tall
    C = R.rmc_sketch(Ab, 4096, "countsketch", SEED)
    R.rmc_sync()
    assert relfro(C.cpu().numpy(), sketch.countsketch(Ab_h, 4096, SEED)) < 1e-5


@pytest.mark.parametrize("kind,prec", [("countsketch", "fp32"), ("srht", "fp32"), ("gaussian", "tf32"),
                                       ("gaussian", "fp32"), ("gaussian", "bf16")])
@pytest.mark.parametrize("s", [1024, 4096])
def test_lsr_full_size_solves_its_sketch(R, tall, kind, prec, s):
    """x of rmc_lsr_sketch is the FP64 least-squares solution of the FP32 sketch [S^T A, S^T b] (the same
    operator rmc_sketch applies to [A, b], pinned against the oracle row by row above).  The tensor-core
    Gaussian form folds b in with FP32 FMAs, so its S^T b is compared with the FP32 form's (1e-5: the two
    draw the normals with different special-function approximations)."""
    A, b, Ab, _ = tall
    x = R.rmc_lsr_sketch(A, b, s, kind, SEED, prec=prec)
    C = R.rmc_sketch(Ab, s, kind, SEED, prec="fp32" if kind == "gaussian" else prec)
    SA = R.rmc_sketch(A, s, kind, SEED, prec=prec) if prec != "fp32" else None
    R.rmc_sync()
    C = C.cpu().numpy().astype(np.float64)
    SA = C[:, :N] if SA is None else SA.cpu().numpy().astype(np.float64)
    xo = linalg.lstsq_qr(SA, C[:, N])
    assert relfro(x.cpu().numpy(), xo) < (1e-6 if prec == "fp32" else 1e-5)


@pytest.fixture(scope="module")
def big():
    A = workloads.factor_rank_torch(65536, 16384, 2048, seed=SEED)
    return A, A.cpu().numpy()


@pytest.mark.parametrize("q", [0, 1, 2])
def test_rsvd_full_size(R, big, q):
    A, A_h = big
    k, p = 100, 20
    Uo, so, Vo, Qo = rsvd.rsvd(A_h, k, p, q, SEED)
    A64 = A_h.astype(np.float64)
    a2 = float(np.sum(A64 * A64))

    def proj_residual(U):
        """||A - Q Q^T A||_F for Q an orthonormal basis of span(U): ||A||^2 - ||Q^T A||^2 (the residual is
        ~0.6% of ||A||^2 here, far above FP64 cancellation)."""
        Q, _ = np.linalg.qr(np.asarray(U, dtype=np.float64))
        P = Q.T @ A64
        return np.sqrt(a2 - float(np.sum(P * P)))

    res_k = proj_residual(Uo)
    for prec, tol in (("fp32", 1e-4), ("tf32x3", 1e-4), ("tf32", 2e-3), ("bf16", 5e-3)):
        U, s, V = R.rmc_rsvd(A, k, p, q, SEED, prec=prec)
        R.rmc_sync()
        np.testing.assert_allclose(s.cpu().numpy(), so, rtol=tol, err_msg=prec)
        # ||A - U U^T A||_F (the top-k directions) against the oracle's
        res_g = proj_residual(U.cpu().numpy())
        assert abs(res_g - res_k) <= 0.01 * res_k, (prec, res_g, res_k)


@pytest.mark.parametrize("kind", ["countsketch", "srht", "gaussian"])
def test_lsr_precise_full_size(R, tall, kind):
    """Algorithm 4.1 on the full regression workload reaches LAPACK's least-squares solution of the FP32
    inputs (numpy.linalg.lstsq in FP64 on the host) within 1e-10 relative."""
    A, b, _, Ab_h = tall
    x = R.rmc_lsr_precise(A, b, 4096, kind, SEED, prec="tf32" if kind == "gaussian" else "fp32", max_iters=60)
    R.rmc_sync()
    xs = _lapack_solution(Ab_h)
    assert relfro(x.cpu().numpy(), xs) < 1e-10


_XSTAR = {}


def _lapack_solution(Ab_h):
    if "x" not in _XSTAR:
        A64 = Ab_h[:, :N].astype(np.float64)
        _XSTAR["x"] = np.linalg.lstsq(A64, Ab_h[:, N].astype(np.float64), rcond=None)[0]
    return _XSTAR["x"]
