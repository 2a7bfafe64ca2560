"""The C-ABI library loads and exports every symbol include/pjac.h declares
(no GPU needed; no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pjac.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pjac_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_23187_b300 import build_lib
    build_lib.build()
    from paper_2607_23187_b300 import pjac
    return pjac.load()


def test_header_declares_the_api():
    names = declared_functions()
    for must in ("pjac_precondition", "pjac_solve", "pjac_solve_preconditioned", "pjac_solve_batched",
                 "pjac_serve_submit", "pjac_serve_poll", "pjac_create", "pjac_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2607_23187_b300 import pjac
    assert set(pjac.EXPORTS) == set(declared_functions())


def test_status_strings_and_default_opts(lib):
    from paper_2607_23187_b300 import pjac
    assert lib.pjac_status_string(0) == b"PJAC_OK"
    assert b"ENOCONV" in lib.pjac_status_string(pjac.PJAC_ENOCONV)
    o = pjac.default_opts()
    assert o.tol == 1e-15 and o.ns_steps == 3 and o.stop == 0
    s = pjac.ServeOpts()
    lib.pjac_serve_default_opts(ctypes.byref(s))


def test_struct_sizes_match_header():
    """The ctypes mirrors have the C layout (offsets checked by a C compile)."""
    import subprocess
    import tempfile
    from paper_2607_23187_b300 import pjac
    src = '#include <stdio.h>\n#include <stddef.h>\n#include "pjac.h"\nint main(){printf("%zu %zu %zu %zu\\n", sizeof(pjac_opts), sizeof(pjac_info), sizeof(pjac_serve_opts), sizeof(pjac_serve_stats));return 0;}\n'
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    assert [int(x) for x in out] == [ctypes.sizeof(pjac.Opts), ctypes.sizeof(pjac.Info),
                                     ctypes.sizeof(pjac.ServeOpts), ctypes.sizeof(pjac.ServeStats)]
