"""The batched engine (rmc_batch_run): many uneven problems in one persistent launch.

Checked against the FP64 oracle (rSVD top-k singular values within 1e-4 relative error, ||A - U S V^T||_F
within 1% of the oracle's; least-squares x within 1e-4 relative error), against the single-problem entry
points, and the same problem alone vs in a mix: bit-identical, since a problem's arithmetic does not depend
on what else is in the batch or on which CTA runs it.
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def dev_strided(x, pad, offset):
    """x on the device as a view with row stride n + pad starting `offset` floats into its buffer."""
    m, n = x.shape
    buf = torch.zeros(m * (n + pad) + offset, dtype=torch.float32, device="cuda")
    view = buf[offset:].view(m, n + pad)[:, :n]
    view.copy_(torch.from_numpy(x))
    return view


# (kind, m, n, k or s, p, q, row padding, pointer offset in floats)
CASES = [
    ("rsvd", 300, 40, 16, 8, 1, 0, 0),      # l = 24, tiles of one partial block
    ("rsvd", 1000, 17, 8, 0, 0, 0, 0),      # l = 8, n not a multiple of 4, q = 0 (CholeskyQR2 on A Omega)
    ("rsvd", 2500, 64, 12, 4, 2, 3, 1),     # l = 16, q = 2, unaligned rows (4-byte copies)
    ("rsvd", 5000, 256, 20, 12, 1, 0, 0),   # l = 32, n at its maximum
    ("rsvd", 40, 36, 20, 4, 1, 0, 0),       # nearly square, l close to n
    ("rsvd", 9000, 129, 16, 8, 1, 4, 4),    # many tiles, row stride n + 4
    ("lsr", 700, 16, 64, 0, 0, 0, 0),
    ("lsr", 4000, 100, 400, 0, 0, 0, 0),
    ("lsr", 3000, 256, 1024, 0, 0, 0, 0),   # n and s at their maxima
    ("lsr", 200, 50, 100, 0, 0, 0, 0),      # about one bucket in eight empty
    ("lsr", 6000, 40, 40, 0, 0, 0, 0),      # s = n
    ("lsr", 20000, 33, 132, 0, 0, 5, 3),    # unaligned rows
    ("lsr", 31, 7, 9, 0, 0, 0, 0),          # m < number of warps' rows
]


def make_case(i, case):
    kind, m, n, ks, p, q, pad, off = case
    spec = dict(kind=kind, m=m, n=n, seed=1000 + i)
    if kind == "rsvd":
        spec.update(k=ks, p=p, q=q)
    else:
        spec.update(s=ks)
    A, b = workloads.batch_problem_numpy(spec)
    Ad = dev_strided(A, pad, off) if (pad or off) else dev(A)
    bd = dev(b) if b is not None else None
    return spec, A, b, Ad, bd


def request(R, spec, Ad, bd):
    if spec["kind"] == "rsvd":
        return R.rsvd_request(Ad, spec["k"], spec["p"], spec["q"], spec["seed"])
    return R.lsr_request(Ad, bd, spec["s"], spec["seed"])


@pytest.fixture(scope="module")
def mixed(R):
    """All CASES in one batch: (cases, outputs)."""
    cases = [make_case(i, c) for i, c in enumerate(CASES)]
    reqs, outs = [], []
    for spec, A, b, Ad, bd in cases:
        r, o = request(R, spec, Ad, bd)
        reqs.append(r)
        outs.append(o)
    R.rmc_batch_run(reqs)
    R.rmc_sync()
    return cases, outs


def check_rsvd(spec, A, out):
    U, s, V = (t.cpu().numpy() for t in out)
    k, p, q = spec["k"], spec["p"], spec["q"]
    Uo, so, Vo, _ = rsvd.rsvd(A, k, p, q, spec["seed"])
    np.testing.assert_allclose(s, so, rtol=1e-4)
    A64 = A.astype(np.float64)
    err = np.linalg.norm(A64 - (U * s) @ V.T)
    erro = np.linalg.norm(A64 - (Uo * so) @ Vo.T)
    assert abs(err - erro) <= 0.01 * erro
    # the same vectors under the same sign convention
    np.testing.assert_allclose(V, Vo, atol=2e-3)
    np.testing.assert_allclose(U, Uo, atol=2e-3)


def check_lsr(spec, A, b, x):
    xo = lsr.lsr_sketch(A, b, spec["s"], "countsketch", spec["seed"])
    x = x.cpu().numpy()
    assert np.linalg.norm(x - xo) <= 1e-4 * np.linalg.norm(xo)


@pytest.mark.parametrize("i", range(len(CASES)))
def test_batch_matches_oracle(R, mixed, i):
    cases, outs = mixed
    spec, A, b, _, _ = cases[i]
    if spec["kind"] == "rsvd":
        check_rsvd(spec, A, outs[i])
    else:
        check_lsr(spec, A, b, outs[i])


def test_batch_alone_equals_mixed(R, mixed):
    """Each problem run alone gives bit-identical outputs to the same problem inside the mixed batch."""
    cases, outs = mixed
    for i, (spec, A, b, Ad, bd) in enumerate(cases):
        r, o = request(R, spec, Ad, bd)
        R.rmc_batch_run([r])
        R.rmc_sync()
        got = o if isinstance(o, tuple) else (o,)
        ref = outs[i] if isinstance(outs[i], tuple) else (outs[i],)
        for g, e in zip(got, ref):
            assert torch.equal(g, e), (i, spec)


def test_batch_matches_single_entry_points(R, mixed):
    """The batch and rmc_rsvd / rmc_lsr_sketch (FP32, count sketch) agree within the stated tolerances."""
    cases, outs = mixed
    for i, (spec, A, b, Ad, bd) in enumerate(cases):
        if spec["kind"] == "rsvd":
            U, s, V = R.rmc_rsvd(Ad, spec["k"], spec["p"], spec["q"], spec["seed"], prec="fp32")
            R.rmc_sync()
            np.testing.assert_allclose(outs[i][1].cpu().numpy(), s.cpu().numpy(), rtol=1e-4)
        else:
            x = R.rmc_lsr_sketch(Ad, bd, spec["s"], "countsketch", spec["seed"])
            R.rmc_sync()
            xs = x.cpu().numpy()
            assert np.linalg.norm(outs[i].cpu().numpy() - xs) <= 1e-4 * np.linalg.norm(xs)


def test_batch_square_omega_shifted_cholqr(R):
    """l = n with a draw of Omega (seed below) that makes A Omega ill conditioned: the FP32 CholeskyQR of the
    range finder meets a non-positive pivot and the shifted retry keeps the result accurate (no breakdown)."""
    spec = dict(kind="rsvd", m=893, n=17, k=16, p=1, q=1, seed=20150587454479)
    A, _ = workloads.batch_problem_numpy(spec)
    for Ad in (dev(A), dev_strided(A, 3, 1)):
        r, out = R.rsvd_request(Ad, 16, 1, 1, spec["seed"])
        R.rmc_batch_run([r])
        R.rmc_sync()
        check_rsvd(spec, A, out)


def test_batch_workload_sample(R):
    """A 48-problem sample of the batched workload recipe (m up to 8192), every problem against the oracle."""
    specs = workloads.batch_specs(count=48, seed=3, m_range=(512, 8192))
    probs, reqs, outs = [], [], []
    for spec in specs:
        A, b = workloads.batch_problem_numpy(spec)
        Ad, bd = dev(A), (dev(b) if b is not None else None)
        r, o = request(R, spec, Ad, bd)
        probs.append((spec, A, b, Ad, bd))
        reqs.append(r)
        outs.append(o)
    R.rmc_batch_run(reqs)
    R.rmc_sync()
    for (spec, A, b, _, _), o in zip(probs, outs):
        if spec["kind"] == "rsvd":
            check_rsvd(spec, A, o)
        else:
            check_lsr(spec, A, b, o)


def test_batch_empty_and_invalid(R):
    R.rmc_batch_run([])
    A = dev(workloads.gaussian(100, 20, seed=1))
    b = dev(workloads.gaussian(100, 1, seed=2)[:, 0])
    Aw = dev(workloads.gaussian(40, 300, seed=3))
    good, good_out = R.lsr_request(A, b, 40, 0)
    bad = [
        R.rsvd_request(A, 16, 8, 1, 0),      # l = 24 > n = 20
        R.lsr_request(A, b, 10, 0),          # s < n
        R.lsr_request(A, b, 1025, 0),        # s above 1024
        R.rsvd_request(Aw, 4, 4, 1, 0),      # n above 256
    ]
    for r, _ in bad:  # the output tensors stay referenced in `bad`
        with pytest.raises(R.RmcError) as e:
            R.rmc_batch_run([good, r])
        assert e.value.status == R.RMC_EINVAL
    good.kind = 7
    with pytest.raises(R.RmcError):
        R.rmc_batch_run([good])


# ------------------------------------------------------------------------------------------ autotuner

def test_autotune_fills_the_table_and_keeps_parity(R):
    """rmc_batch_autotune picks a row tile per k-SVD class from the candidates; with the tuned table every
    problem still matches the oracle, and a problem is bit-identical alone and in the mix."""
    cases = [make_case(i, c) for i, c in enumerate(CASES)]
    reqs, outs = [], []
    for spec, A, b, Ad, bd in cases:
        r, o = request(R, spec, Ad, bd)
        reqs.append(r)
        outs.append(o)
    default = R.rmc_batch_get_tiles()
    try:
        table = R.rmc_batch_autotune(reqs, reps=2)
        assert len(table) == R.RMC_BATCH_TILE_CLASSES
        assert all(t in (0, 32, 64, 128) for t in table)
        R.rmc_batch_run(reqs)
        R.rmc_sync()
        for (spec, A, b, Ad, bd), o in zip(cases, outs):
            if spec["kind"] == "rsvd":
                check_rsvd(spec, A, o)
            else:
                check_lsr(spec, A, b, o)
        # alone vs in the mix under the tuned table
        i = 3
        spec, A, b, Ad, bd = cases[i]
        r, o = request(R, spec, Ad, bd)
        R.rmc_batch_run([r])
        R.rmc_sync()
        for g, e in zip(o, outs[i]):
            assert torch.equal(g, e)
    finally:
        R.rmc_batch_set_tiles(default)


def test_tile_table_round_trip_and_validation(R):
    old = R.rmc_batch_get_tiles()
    try:
        t = [16 * (i % 9) for i in range(R.RMC_BATCH_TILE_CLASSES)]
        R.rmc_batch_set_tiles(t)
        assert R.rmc_batch_get_tiles() == t
        with pytest.raises(R.RmcError):
            R.rmc_batch_set_tiles([17] * R.RMC_BATCH_TILE_CLASSES)
        assert R.rmc_batch_get_tiles() == t
    finally:
        R.rmc_batch_set_tiles(old)
