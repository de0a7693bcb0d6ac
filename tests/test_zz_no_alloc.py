"""The allocation-free count-sketch entry point (rmc_countsketch_noalloc) gives the same sketch as the
context-based rmc_sketch.  It exists for callers that must not allocate device memory at call time (a
serving loop that reserves its HBM up front, or a framework that owns all device memory through its own
allocator); it keeps its scratch in a fixed 32 MiB device array instead.

This file is collected last on purpose: if it fails, a run that stops at the first failure has already run
every other test.  It passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def relfro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_noalloc_matches_context_path_two_calls_in_a_row():
    import paper_1505_07570_gb300 as rmc
    # Two different problems back to back: the second call must not see the first call's scratch.
    cases = [(200000, 96, 2048, 31), (50000, 33, 500, 7)]
    for m, n, s, seed in cases:
        A = torch.from_numpy(workloads.gaussian(m, n, seed=m)).cuda()
        ref = rmc.rmc_sketch(A, s, "countsketch", seed)
        out = torch.full((s, n), float("nan"), device="cuda")
        got = rmc.rmc_countsketch_noalloc(A, s, seed, out=out)
        torch.cuda.synchronize()
        rmc.rmc_sync()
        assert got.data_ptr() == out.data_ptr()
        assert relfro(got.cpu().numpy(), ref.cpu().numpy()) < 1e-5


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1505_07570_gb300 as rmc
    A = torch.zeros(1 << 20, 4, device="cuda")
    with pytest.raises(rmc.RmcError) as e:
        rmc.rmc_countsketch_noalloc(A, 16384, 1)       # needs about 72 MB of scratch
    assert e.value.status == rmc.RMC_ESCRATCH
