"""The oracle's Philox4x32-10 against an independent implementation that ships with PyTorch: ATen's
``at::philox_engine`` (ATen/core/PhiloxRNGEngine.h, an open-source header), compiled here on the host.

ATen's engine takes key = (seed mod 2^32, seed div 2^32), counter words 2-3 = the 64-bit "subsequence" and
counter words 0-1 = the 64-bit "offset", and returns the four words of one block in order; so the block at
(index, stream, instance) of the library's layout is ATen's block at offset = index and subsequence =
stream + 2^32 instance.  A mistake the statistical pins cannot see (swapped output words, hi and lo exchanged
in a round, a wrong Weyl constant) fails here.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import philox

PROBE = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdlib>
int main(int argc, char **argv) {
  for (int a = 1; a + 2 < argc; a += 3) {
    const unsigned long long seed = strtoull(argv[a], 0, 0), sub = strtoull(argv[a + 1], 0, 0),
                             off = strtoull(argv[a + 2], 0, 0);
    at::philox_engine e(seed, sub, off);
    const unsigned w0 = e(), w1 = e(), w2 = e(), w3 = e();
    printf("%u %u %u %u\n", w0, w1, w2, w3);
  }
  return 0;
}
"""

# (seed, stream, instance, index): zero key and counter, every counter word non-zero, the top bits of the
# index and of the seed, each stream of the layout, large instances
CASES = [
    (0, 0, 0, 0),
    (0x0123456789ABCDEF, 2, 0, 5),
    (0xFFFFFFFFFFFFFFFF, 3, 0xFFFFFFFF, 0xFFFFFFFFFFFFFFFF),
    (20150527, 0, 0, 262143),
    (20150527, 1, 0, (1 << 32) + 7),
    (7, 2, 123456, 1 << 40),
    (1 << 63, 3, 1, 987654321),
    (0xDEADBEEFCAFEF00D, 8, 42, 31),
]


@pytest.fixture(scope="module")
def aten_probe(tmp_path_factory):
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("ATen headers not installed")
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("aten_philox")
    src, exe = d / "probe.cpp", d / "probe"
    src.write_text(PROBE)
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I" + inc, str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    if r.returncode != 0:
        pytest.skip("ATen Philox header does not compile here: " + r.stderr[-400:])
    return str(exe)


def test_oracle_philox_matches_aten(aten_probe):
    args = []
    for seed, stream, instance, index in CASES:
        args += [str(seed), str(stream + (instance << 32)), str(index)]
    out = subprocess.run([aten_probe] + args, capture_output=True, text=True, check=True).stdout.split("\n")
    for (seed, stream, instance, index), line in zip(CASES, out):
        ref = np.array([int(v) for v in line.split()], dtype=np.uint64)
        got = philox.draw(np.array([index], dtype=np.uint64), stream, seed, instance)[0].astype(np.uint64)
        np.testing.assert_array_equal(got, ref, err_msg=str((seed, stream, instance, index)))
