"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every function declared in include/afieti.h; status strings."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "afieti.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "return")))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300 import afieti
    return afieti.load()


def test_header_lists_entry_points():
    names = declared_functions()
    for n in ("af_ieti_setup", "fd_apply", "ieti_solve", "ieti_solve_adjoint", "afi_lame_grad",
              "afi_sizes", "af_ieti_destroy", "afi_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_status_strings(lib):
    from paper_2001_09626_gb300 import afieti
    assert afieti.afi_status_string(0) == "ok"
    assert "converged" in afieti.afi_status_string(afieti.AFI_ENOT_CONVERGED)
    assert afieti.afi_status_string(99) == "unknown status"


def test_setup_rejects_invalid_problem_without_touching_the_device(lib):
    import ctypes as C
    from paper_2001_09626_gb300 import afieti
    prob = afieti.afi_problem(5, 1, None, None, None, None, None)
    opt = afieti.afi_options(0, 1e-8, 100, 0, 0)
    h = C.c_void_p()
    st = lib.af_ieti_setup(C.byref(prob), C.byref(opt), C.byref(h))
    assert st == afieti.AFI_EINVAL and not h.value
    assert "invalid" in afieti.afi_last_error()


def test_selftest_rejects_out_of_range_polls_without_touching_the_device(lib):
    from paper_2001_09626_gb300 import afieti
    for polls in (0, -5, (1 << 22) + 1):
        status, used = afieti.afi_selftest_bounded_wait(polls)
        assert status == afieti.AFI_EINVAL and used == 0
    assert "polls" in afieti.afi_last_error()


def test_no_oracle_on_product_path():
    """The package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2001_09626_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
