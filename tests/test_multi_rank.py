"""The multi-GPU form is replicas (independent problems per rank, no data-path collective): bench.py takes the
maximum time over ranks and the total bytes over ranks.  These tests run that host logic as two gloo ranks on
the CPU (127.0.0.1), and check that the reference arm does its work on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
dist.init_process_group("gloo", rank=int(os.environ["RANK"]), world_size=int(os.environ["WORLD_SIZE"]))
import bench
rank = dist.get_rank()
seconds, nbytes = bench.combine_over_ranks(0.25 + 0.5 * rank, 1000 * (rank + 1), dist.get_world_size())
print(json.dumps({"rank": rank, "seconds": seconds, "bytes": nbytes}))
dist.destroy_process_group()
"""


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(code, world, extra_args=(), timeout=120):
    port = free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", code, ROOT, *extra_args], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=timeout)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_combine_over_ranks_two_gloo_ranks():
    outs = run_ranks(RANK_SCRIPT, 2)
    lines = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(l["rank"] for l in lines) == [0, 1]
    for l in lines:  # every rank sees the slowest rank's time and the bytes of all ranks
        assert l["seconds"] == pytest.approx(0.75)
        assert l["bytes"] == pytest.approx(3000.0)


def test_combine_over_ranks_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_over_ranks(1.5, 42, 1) == (1.5, 42)


REFERENCE_SCRIPT = r"""
import os, sys
sys.path.insert(0, sys.argv[1])
sys.argv = ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
import bench
bench.ORACLE_SAMPLE_ROWS = 256  # a tiny sample: this checks the control flow, not the timing
sys.exit(bench.main())
"""


def test_reference_arm_runs_on_rank_zero_only():
    outs = run_ranks(REFERENCE_SCRIPT, 2, timeout=300)
    printed = [o.strip() for o in outs]
    assert printed[1] == ""  # rank 1 exits 0 without work
    line = json.loads(printed[0].splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


def test_union_of_launch_intervals():
    """The roofline's device time for launches that overlap on several streams: the union of their intervals."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.union_ms([]) == 0.0
    assert bench.union_ms([(0.0, 2.0), (1.0, 3.0)]) == pytest.approx(3.0)      # overlapping
    assert bench.union_ms([(5.0, 6.0), (0.0, 1.0)]) == pytest.approx(2.0)      # disjoint, unsorted
    assert bench.union_ms([(0.0, 4.0), (1.0, 2.0), (3.0, 5.0)]) == pytest.approx(5.0)  # nested + chained
