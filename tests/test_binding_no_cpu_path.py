"""The Python binding has no CPU path: every entry point that takes a matrix refuses a host tensor (or a
matrix of the wrong dtype or layout) with ValueError before any CUDA call, so nothing computes silently on the
host.  Runs without a GPU."""
import pytest
import torch

rmc = pytest.importorskip("paper_1505_07570_gb300")

A = torch.zeros(64, 8, dtype=torch.float32)
b = torch.zeros(64, dtype=torch.float32)

CALLS = {
    "rmc_sketch": lambda M: rmc.rmc_sketch(M, 16, "gaussian", 1),
    "rmc_lsr_sketch": lambda M: rmc.rmc_lsr_sketch(M, b, 16, "countsketch", 1),
    "rmc_rsvd": lambda M: rmc.rmc_rsvd(M, 2, 2, 1, 1),
    "rmc_lsr_precise": lambda M: rmc.rmc_lsr_precise(M, b, 16, "srht", 1),
    "rmc_block_lanczos": lambda M: rmc.rmc_block_lanczos(M, 2, 4, 1, 1),
    "rmc_rsvd_fast": lambda M: rmc.rmc_rsvd_fast(M, 2, 4, 16, 8, 1),
    "rmc_countsketch_columns": lambda M: rmc.rmc_countsketch_columns(M, 4, 1),
    "rmc_nystrom": lambda M: rmc.rmc_nystrom(M, 1.0, 8, 1),
    "rmc_rbf": lambda M: rmc.rmc_rbf(M, M, 1.0),
    "rmc_cholqr2": lambda M: rmc.rmc_cholqr2(M),
    "rmc_svd_wide": lambda M: rmc.rmc_svd_wide(M),
    "rmc_matmul_an": lambda M: rmc.rmc_matmul_an(M, torch.zeros(8, 4)),
    "rmc_matmul_at": lambda M: rmc.rmc_matmul_at(M, torch.zeros(64, 4)),
    "rmc_countsketch_noalloc": lambda M: rmc.rmc_countsketch_noalloc(M, 16, 1),
}


@pytest.mark.parametrize("name", sorted(CALLS))
def test_host_matrix_is_refused(name):
    with pytest.raises(ValueError, match="CUDA float32 matrix"):
        CALLS[name](A)


@pytest.mark.parametrize("bad", [A.double(), A.t(), A[:, 0]], ids=["float64", "column-major", "vector"])
def test_wrong_dtype_or_layout_is_refused(bad):
    with pytest.raises(ValueError):
        rmc.rmc_sketch(bad, 16, "countsketch", 1)


def test_every_matrix_entry_point_is_covered():
    """A new public entry point that takes a matrix first gets a line in CALLS."""
    import inspect
    takes_matrix = {n for n, f in vars(rmc).items()
                    if n.startswith("rmc_") and inspect.isfunction(f)
                    and list(inspect.signature(f).parameters)[:1] in (["A"], ["X"], ["Y"], ["B"])}
    assert takes_matrix <= set(CALLS), sorted(takes_matrix - set(CALLS))
