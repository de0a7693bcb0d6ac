"""Host-side checks of the index schedules two kernels rely on (run without a GPU).  Each test restates a
kernel's formula in Python and checks the invariant its correctness or speed depends on.

- transpose_tile_tf32 (tc_gemm.cu): the lane -> unit mapping covers every 4 x 4 unit of the staged tile
  exactly once, stays inside the tile, and each 8-lane group's 16-byte reads and writes fall on 8 distinct
  bank groups (the swizzled layout a 32 x 32 TMA box with 128-byte swizzle writes).
- jacobi_oe_kernel (dense.cu): the odd-even schedule with one column kept per group meets every pair of
  columns exactly once per sweep of l' rounds, and the output order returns every real column once (the zero
  padding column of an odd l sits at position 0 after an odd number of sweeps, else at l' - 1).
"""
import itertools

import pytest


def swz_off(r, q):
    """Byte offset of (row r, 16-byte chunk q) in a tile of 128-byte rows with 128-byte swizzle."""
    return r * 128 + ((q ^ (r & 7)) << 4)


@pytest.mark.parametrize("atoms,halves,threads", [(8, 1, 64), (8, 2, 128), (4, 2, 128)])
def test_transposer_units_cover_the_tile_without_bank_conflicts(atoms, halves, threads):
    units = {}
    banks = {}
    for tl in range(threads):
        lq, gl, gh = tl & 7, (tl >> 3) & 7, tl >> 6
        c0 = (gl + lq) & 7
        for i in range(atoms // halves):
            atom = gh + halves * i
            cq = c0 + 8 * atom
            units[(lq, cq)] = units.get((lq, cq), 0) + 1
            for t in range(4):
                read = atom * 4096 + swz_off(4 * lq + t, c0)      # staged: row 4 lq + t, columns 4 cq .. +3
                write = atom * 4096 + swz_off(4 * c0 + t, lq)     # operand: row 4 cq + t, K chunk lq
                assert write == swz_off(4 * cq + t, lq)
                assert 0 <= read < atoms * 4096 and 0 <= write < atoms * 4096
                banks.setdefault(("r", tl >> 3, i, t), set()).add((read >> 4) & 7)
                banks.setdefault(("w", tl >> 3, i, t), set()).add((write >> 4) & 7)
    assert len(units) == 8 * 8 * atoms and set(units.values()) == {1}
    assert all(len(v) == 8 for v in banks.values())


def odd_even_sweeps(l, sweeps):
    """The data flow of jacobi_oe_kernel with column labels: returns the pairs met in each sweep and the
    output column order."""
    lp = l + (l & 1)
    last = lp // 2 - 1
    slot = list(range(lp))
    arr = [slot[2 * g] for g in range(lp // 2)]
    keep = [slot[2 * g + 1] for g in range(lp // 2)]
    met = []
    for _ in range(sweeps):
        pairs = []
        for _ in range(0, lp, 2):
            for g in range(lp // 2):                 # even round: (2g, 2g+1) = (arr, keep), then swap
                pairs.append(frozenset((arr[g], keep[g])))
                slot[2 * g] = keep[g]
                keep[g] = arr[g]
            for g in range(last):
                arr[g] = slot[2 * g + 2]
            for g in range(last):                    # odd round: (2g+1, 2g+2) = (keep, arr), then swap
                pairs.append(frozenset((keep[g], arr[g])))
                slot[2 * g + 2] = keep[g]
                keep[g] = arr[g]
            for g in range(lp // 2):
                arr[g] = slot[2 * g]
        met.append(pairs)
    for g in range(lp // 2):
        slot[2 * g + 1] = keep[g]
    pad = -1 if lp == l else (0 if sweeps & 1 else lp - 1)
    out = [slot[c + 1] if 0 <= pad <= c else slot[c] for c in range(l)]
    return met, out


@pytest.mark.parametrize("l", [2, 3, 7, 33, 40, 72, 99, 120, 127, 128])
@pytest.mark.parametrize("sweeps", [1, 2, 3, 10, 11])
def test_odd_even_schedule_meets_every_pair_once_per_sweep(l, sweeps):
    met, out = odd_even_sweeps(l, sweeps)
    lp = l + (l & 1)
    every = {frozenset(p) for p in itertools.combinations(range(lp), 2)}
    for pairs in met:
        assert len(pairs) == len(every) and set(pairs) == every
    assert sorted(out) == list(range(l))
