"""Failure delivery, in forms that fault, trap or hang no GPU: a bounded device wait that runs out, a numerically
rank-deficient problem, and an allocation refused by the context's HBM budget.  Each error reaches the host as a
status code (synchronously for the budget, at rmc_sync for the device-detected ones) and the context stays
usable afterwards."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    import paper_1505_07570_gb300 as rmc
    return rmc


def test_bounded_wait_reports_timeout_and_context_recovers(R):
    ctx = R.context().bind()
    assert R.lib.rmc_debug_wait_timeout(ctx, 2_000_000) == R.RMC_OK          # a 2 ms wait that nothing ends
    assert R.lib.rmc_sync(ctx) == R.RMC_ETIMEOUT
    assert R.lib.rmc_sync(ctx) == R.RMC_OK                                  # the status word was cleared
    A = torch.from_numpy(workloads.gaussian(5000, 16, seed=1)).cuda()
    C = R.rmc_sketch(A, 64, "countsketch", 3)                               # the context still works
    R.rmc_sync()
    assert bool(torch.isfinite(C).all())
    assert R.lib.rmc_debug_wait_timeout(ctx, 2_000_000_000) == R.RMC_EINVAL  # above the 1 s cap


@pytest.mark.parametrize("kind", ["countsketch", "gaussian"])
def test_rank_deficient_least_squares_reports_numeric(R, kind):
    """A zero column of A makes S^T A rank deficient for every S, with an exactly zero pivot: both the FP32
    factor and the FP64 fallback meet it, and rmc_sync returns RMC_ENUMERIC."""
    A, b, _ = workloads.tall_lsr_numpy(4000, 8, seed=2)
    A[:, 5] = 0
    x = R.rmc_lsr_sketch(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), 200, kind, 4)
    with pytest.raises(R.RmcError) as e:
        R.rmc_sync()
    assert e.value.status == R.RMC_ENUMERIC
    R.rmc_sync()                                                             # cleared; the context is usable


def test_cholqr2_of_a_zero_column_reports_numeric(R):
    Y = torch.from_numpy(workloads.gaussian(3000, 10, seed=3)).cuda()
    Y[:, 4] = 0
    R.rmc_cholqr2(Y, want_r=False)
    with pytest.raises(R.RmcError) as e:
        R.rmc_sync()
    assert e.value.status == R.RMC_ENUMERIC


def test_budget_refuses_each_call_synchronously(R):
    """A context created with a 4 KiB budget: every call whose workspace exceeds it returns RMC_ENOMEM before
    anything is enqueued."""
    h = ctypes.c_void_p()
    stream = torch.cuda.current_stream().cuda_stream
    assert R.lib.rmc_create(ctypes.byref(h), ctypes.c_void_p(stream), 4096) == R.RMC_OK
    try:
        m, n = 20000, 64
        A = torch.randn(m, n, device="cuda")
        b = torch.randn(m, device="cuda")
        C = torch.empty(1024, n, device="cuda")
        x = torch.empty(n, device="cuda", dtype=torch.float64)
        U = torch.empty(m, 8, device="cuda")
        sg = torch.empty(8, device="cuda")
        V = torch.empty(n, 8, device="cuda")
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        assert R.lib.rmc_sketch(h, p(A), m, n, n, 1024, R.RMC_COUNTSKETCH, 1, R.RMC_FP32, p(C), n) == R.RMC_ENOMEM
        assert R.lib.rmc_lsr_sketch(h, p(A), m, n, n, p(b), 1024, R.RMC_GAUSSIAN, 1, R.RMC_FP32,
                                    p(x)) == R.RMC_ENOMEM
        assert R.lib.rmc_rsvd(h, p(A), m, n, n, 8, 4, 1, 1, R.RMC_FP32, p(U), 8, p(sg), p(V), 8) == R.RMC_ENOMEM
        assert R.lib.rmc_sync(h) == R.RMC_OK
        used = ctypes.c_size_t()
        assert R.lib.rmc_workspace_bytes(h, ctypes.byref(used)) == R.RMC_OK and used.value <= 4096
    finally:
        R.lib.rmc_destroy(h)
