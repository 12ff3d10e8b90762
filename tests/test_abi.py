"""The C-ABI library loads and exports every entry point include/grtx.h declares; host-side
argument checks return their documented status without touching a GPU. CPU only."""
import ctypes as C
import os
import re

import pytest

from paper_2601_20429_gb300 import native as N

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "grtx.h")


def declared_symbols():
    src = open(HEADER).read()
    return re.findall(r"GRTX_API\s+[\w\s\*]+?\b(grtx_\w+)\s*\(", src)


@pytest.fixture(scope="module")
def lib():
    N.build()
    return N.lib()


def test_header_declares_the_boundary():
    names = set(declared_symbols())
    for core in ("grtx_build_bvh", "grtx_trace_forward", "grtx_trace_backward", "grtx_render_requests",
                 "grtx_server_create", "grtx_server_destroy", "grtx_scene_destroy", "grtx_status_string"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(N.SYMBOLS)


def test_status_strings_and_version(lib):
    assert lib.grtx_version() == 1
    assert lib.grtx_status_string(0) == b"ok"
    assert lib.grtx_status_string(1) == b"invalid argument"
    assert lib.grtx_status_string(999) == b"unknown status"


def test_host_side_argument_errors(lib):
    p = N.make_params(k=3)
    assert lib.grtx_build_bvh(None, C.byref(p), 0, None, C.byref(C.c_void_p())) == 1
    g = N.grtx_gaussians()
    g.n, g.sh_degree = 10, 5
    assert lib.grtx_prep_gaussians(C.byref(g), 0.01, None, None, None) == 1
    assert b"sh_degree" in lib.grtx_last_error()
    g.sh_degree = 0
    assert lib.grtx_prep_gaussians(C.byref(g), 0.01, None, None, None) == 1     # NULL arrays
    assert lib.grtx_trace_forward(None, None, None, None, None) == 1
    nb = C.c_size_t(0)
    assert lib.grtx_sort_pairs(None, None, 1000, 64, None, C.byref(nb), None) == 0 and nb.value > 8 * 1000
    assert lib.grtx_sort_pairs(None, None, 10, 65, None, C.byref(nb), None) == 1
    assert lib.grtx_radix_tree(None, 1, None, None, None, None) == 1
    assert lib.grtx_server_submit(None, None, 0) == 1
    assert lib.grtx_server_create(None, 0, None, 0, 0, None, None) == 1
