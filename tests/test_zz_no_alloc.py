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
    # Two different problems back to back: the second call must not see the first call's scratch.  Both
    # paths run the same deterministic kernels in the same order, so the sketches are bit-identical.
    cases = [(200000, 96, 2048, 31), (50000, 33, 500, 7)]
    for m, n, s, seed in cases:
        A = torch.from_numpy(workloads.gaussian(m, n, seed=m)).cuda()
        ref = rmc.rmc_sketch(A, s, "countsketch", seed)
        out = torch.full((s, n), float("nan"), device="cuda")
        got = rmc.rmc_countsketch_noalloc(A, s, seed, out=out)
        torch.cuda.synchronize()
        rmc.rmc_sync()
        assert got.data_ptr() == out.data_ptr()
        assert torch.equal(got, ref)


def test_noalloc_padded_strides_on_a_side_stream_match_the_oracle():
    """lda > n and ldc > n, enqueued on a stream of its own, against the oracle's count sketch."""
    import paper_1505_07570_gb300 as rmc
    from oracle import sketch
    m, n, s, seed = 3000, 21, 64, 5
    A = workloads.gaussian(m, n, seed=9)
    Ad = torch.zeros(m, n + 3, device="cuda")
    Ad[:, :n] = torch.from_numpy(A).cuda()
    Cd = torch.full((s, n + 5), float("nan"), device="cuda")
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        rmc.rmc_countsketch_noalloc(Ad[:, :n], s, seed, out=Cd[:, :n])
    side.synchronize()
    got = Cd.cpu().numpy()
    assert np.all(np.isnan(got[:, n:]))            # the padding of C is untouched
    assert relfro(got[:, :n], sketch.countsketch(A, s, seed)) < 1e-6


def test_noalloc_rejects_an_output_of_the_wrong_size():
    import paper_1505_07570_gb300 as rmc
    A = torch.zeros(1000, 8, device="cuda")
    with pytest.raises(ValueError):
        rmc.rmc_countsketch_noalloc(A, 64, 1, out=torch.empty(63, 8, device="cuda"))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1505_07570_gb300 as rmc
    A = torch.zeros(1 << 20, 4, device="cuda")
    with pytest.raises(rmc.RmcError) as e:
        rmc.rmc_countsketch_noalloc(A, 16384, 1)       # needs about 72 MB of scratch
    assert e.value.status == rmc.RMC_ESCRATCH
