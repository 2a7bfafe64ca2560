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


def test_arguments_rejected_before_any_device_work(lib):
    """Every entry point checks its arguments before it touches the device,
    so these run without a GPU: invalid options, NULL handles and servers,
    out-of-range sizes.  Each returns PJAC_EINVAL with a message and crashes
    nothing; the pointers passed are never dereferenced."""
    from paper_2607_23187_b300 import pjac
    EINVAL = pjac.PJAC_EINVAL
    bad_opts = {"ns_steps": 11, "cluster_size": 3, "tol": -1.0, "max_rotations": -1, "check_every": -2,
                "stop": 7, "transform": 5}
    for field, value in bad_opts.items():
        h = ctypes.c_void_p(1234)
        st = lib.pjac_create(ctypes.byref(h), ctypes.byref(pjac.default_opts(**{field: value})))
        assert st == EINVAL and h.value is None, field
        assert lib.pjac_last_error(), field
    d1 = ctypes.c_double(1e-15)
    fake = ctypes.c_void_p(4096)    # a device address that is never used
    assert lib.pjac_set_opts(None, None) == EINVAL
    assert lib.pjac_solve(None, fake, 4, 4, 0, 1e-15, fake, None, 4, None, None) == EINVAL
    assert lib.pjac_precondition(None, fake, 4, 4, None, fake, 4, fake, 4, None) == EINVAL
    assert lib.pjac_solve_preconditioned(None, fake, 4, 4, None, 4, 0, 1e-15, fake, None, 4, None, None) == EINVAL
    assert lib.pjac_solve_batched(None, 1, None, None, None, None, None, None, None, 0, 1e-15, None, None) == EINVAL
    assert lib.pjac_product(None, 0, 0, 4, 4, 4, 1.0, fake, 4, fake, 4, 0.0, fake, 4, None) == EINVAL
    assert lib.pjac_product_symmetric(None, 0, 0, 4, 4, 1.0, fake, 4, fake, 4, 0.0, fake, 4, None) == EINVAL
    noalloc = lib.pjac_solve_preconditioned_noalloc
    assert noalloc(None, 4, 4, None, 4, 0, d1, fake, None, 4, None, None) == EINVAL
    assert noalloc(fake, 0, 4, None, 4, 0, d1, fake, None, 4, None, None) == EINVAL
    # beyond the fixed scratch array of the allocation-free entry point
    assert noalloc(fake, 513, 513, None, 513, 0, d1, fake, None, 513, None, None) == EINVAL
    assert b"allocation-free limit" in lib.pjac_last_error()
    assert noalloc(fake, 4, 4, None, 4, 9, d1, fake, None, 4, None, None) == EINVAL
    assert noalloc(fake, 4, 4, None, 4, 0, ctypes.c_double(-1.0), fake, None, 4, None, None) == EINVAL
    # serving
    assert lib.pjac_serve_create(None, None) == EINVAL
    so = pjac.ServeOpts()
    lib.pjac_serve_default_opts(ctypes.byref(so))
    assert so.max_slots == 8 and so.max_queue == 1 << 16 and so.hbm_budget_bytes == 8 << 30
    so.max_slots = 65
    s = ctypes.c_void_p()
    assert lib.pjac_serve_create(ctypes.byref(s), ctypes.byref(so)) == EINVAL and s.value is None
    t = ctypes.c_uint64()
    assert lib.pjac_serve_submit(None, fake, 4, 4, 0, 1e-15, fake, None, 4, ctypes.byref(t)) == EINVAL
    assert lib.pjac_serve_poll(None, ctypes.c_uint64(1), None) == EINVAL
    assert lib.pjac_serve_progress(None) == EINVAL
    assert lib.pjac_serve_get_stats(None, None) == EINVAL
    # NULL is a no-op for the destructors; the counts report -1
    assert lib.pjac_destroy(None) == 0 and lib.pjac_serve_destroy(None) == 0
    assert lib.pjac_solve_launch_count(None, 4) == -1
    assert lib.pjac_product_launch_count(None, 4, 4, 4) == -1
    # every status has its own text
    texts = [lib.pjac_status_string(c) for c in range(-7, 2)]
    assert len(set(texts)) == len(texts) and all(texts)
    assert lib.pjac_status_string(-99) == b"unknown status"
