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
    assert lib.grtx_server_create(None, 0, None, 0, 0, 0, None, None) == 1
    assert lib.grtx_server_release(None, None) == 1
    assert lib.grtx_server_get_info(None, None) == 1
    assert lib.grtx_server_set_linger(None, 0) == 1
    assert lib.grtx_server_set_order(None, 0.0) == 1
    assert lib.grtx_server_set_append_guard(None, 1) == 1


def test_host_side_errors_of_the_extensions(lib):
    """Argument checks of the builder, world, template and secondary-ray entry points return
    GRTX_ERR_INVALID_ARG before any device work."""
    it = C.c_int(0)
    assert lib.grtx_ploc_tree(None, 1, None, None, None, C.byref(it), None) == 1       # n < 2
    assert lib.grtx_ploc_tree(None, 10, None, None, None, C.byref(it), None) == 1      # NULL arrays
    assert lib.grtx_morton_codes_sized(None, -1, None, None, None, None) == 1
    n = C.c_int(0)
    assert lib.grtx_template_mesh(0, None, C.byref(n)) == 1                            # not an icosphere form
    assert lib.grtx_template_mesh(2, None, C.byref(n)) == 0 and n.value == 20
    assert lib.grtx_template_mesh(3, None, C.byref(n)) == 0 and n.value == 80
    w = C.c_void_p()
    assert lib.grtx_world_create(None, 0, None, C.byref(w)) == 1 and not w.value
    inst = (N.grtx_instance * 1)()
    assert lib.grtx_world_create(inst, 1, None, C.byref(w)) == 1                        # NULL scene
    assert b"scene is NULL" in lib.grtx_last_error()
    assert lib.grtx_world_update(None, inst, 1, None) == 1
    assert lib.grtx_memory_trim(-1) == 1                                                 # no device work
    assert lib.grtx_trace_forward_batch(None, None, 1, None, None, None) == 1
    assert lib.grtx_trace_forward_batch(None, N.grtx_camera(), 0, None, (N._fp * 1)(), None) == 1
    rebuilt = C.c_int(5)
    assert lib.grtx_scene_update(None, None, 0, None, C.byref(rebuilt)) == 1 and rebuilt.value == 0
    assert b"scene is NULL" in lib.grtx_last_error()
    assert lib.grtx_world_trace_forward(None, None, None, None, None) == 1
    lib.grtx_world_destroy(None)
    cam = N.grtx_camera()
    cam.type, cam.width, cam.height, cam.fov, cam.t_far = 0, 4, 4, 1.0, 1e30
    mirrors = (N.grtx_mirror * 1)()
    glass = (N.grtx_glass * 1)()
    nulls = [None] * 10
    assert lib.grtx_secondary_rays(C.byref(cam), mirrors, 17, glass, 0, *nulls, None) == 1   # too many objects
    assert lib.grtx_secondary_rays(C.byref(cam), mirrors, 0, glass, 1, *nulls, None) == 1    # radius 0
    assert b"glass" in lib.grtx_last_error()
    p = N.make_params(bvh_builder=7)
    g = N.grtx_gaussians()
    assert lib.grtx_build_bvh(C.byref(g), C.byref(p), 0, None, C.byref(C.c_void_p())) == 1


def header_structs():
    """Field names of every `typedef struct name { ... } name;` in the header, in order."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    out = {}
    for name, body in re.findall(r"typedef\s+struct\s+(\w+)\s*\{(.*?)\}\s*\1\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            first, *more = decl.split(",")
            fields.append(re.findall(r"(\w+)\s*(?:\[[^\]]*\])?\s*$", first)[0])
            fields += [re.findall(r"(\w+)", m)[0] for m in more]
        out[name] = fields
    return out


def test_binding_structs_match_the_header():
    """The binding's ctypes mirrors name the header's fields in the header's order (a field
    added on one side only would shift every later one)."""
    structs = header_structs()
    assert {"grtx_stats", "grtx_params", "grtx_trace_outputs", "grtx_saved"} <= set(structs)
    checked = 0
    for name, fields in structs.items():
        mirror = getattr(N, name, None)
        if mirror is None:
            continue
        assert [f for f, *_ in mirror._fields_] == fields, name
        checked += 1
    assert checked >= 6
    assert N.STATS_FIELDS[-1] == "bounds_errors"
