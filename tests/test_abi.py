"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point include/rmc.h
declares.  No compute calls (those need a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"^\s*(?:const\s+)?(?:int|char\s*\*|const\s+char\s*\*|void)\s*\*?\s*(rmc_\w+)\s*\(",
                                text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    return ctypes.CDLL(path)


def test_header_declares_the_three_calls():
    names = declared_functions()
    for f in ["rmc_create", "rmc_destroy", "rmc_sync", "rmc_sketch", "rmc_rsvd", "rmc_lsr_sketch"]:
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    lib.rmc_status_string.restype = ctypes.c_char_p
    seen = set()
    for code in range(9):
        s = lib.rmc_status_string(code)
        assert s and s not in seen
        seen.add(s)


def test_argument_errors_need_no_gpu(lib):
    """Argument checks run before any CUDA call: a NULL context is rejected synchronously."""
    lib.rmc_sketch.restype = ctypes.c_int
    assert lib.rmc_sketch(None, None, 0, 0, 0, 0, 0, 0, 0, None, 0) == 1     # RMC_EINVAL
    assert lib.rmc_create(None, None, 0) == 1
    assert lib.rmc_destroy(None) == 0


def test_profile_hooks_reject_bad_arguments_without_gpu(lib):
    lib.rmc_profile_reference.restype = ctypes.c_int
    lib.rmc_profile_spans.restype = ctypes.c_int
    n = ctypes.c_int(-1)
    assert lib.rmc_profile_reference(None) == 1                                 # RMC_EINVAL
    assert lib.rmc_profile_spans(None, 3, None, None, 0, ctypes.byref(n)) == 1  # RMC_EINVAL
    assert lib.rmc_profile_begin(None) == 1


def test_header_is_plain_c(tmp_path):
    """include/*.h is a C ABI: every header compiles as C99 on its own (no C++ or CUDA types leak in)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    for h in HEADERS:
        src = tmp_path / "use.c"
        src.write_text('#include "%s"\nint main(void) { return 0; }\n' % h)
        r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-fsyntax-only", str(src)], capture_output=True,
                           text=True)
        assert r.returncode == 0, r.stderr
