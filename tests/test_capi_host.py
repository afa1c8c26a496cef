"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol declared in include/cem.h, and rejects malformed input on the host."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "cem.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(cem_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_04076_gb300 import load_library
    return load_library()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n


def test_binding_binds_every_declared_symbol(lib):
    # the Python binding sets return and argument types for exactly the header's entry points
    from paper_2508_04076_gb300.binding import EXPORTED
    assert sorted(EXPORTED) == _declared()
    for n in EXPORTED:
        assert getattr(lib, n).argtypes is not None, n


def _desc(X, tets, notch_tet=(), notch_side=(), precision=0):
    from paper_2508_04076_gb300.binding import MeshDesc, ALLOC_FN, FREE_FN
    X = np.ascontiguousarray(X, np.float64)
    tets = np.ascontiguousarray(tets, np.int32)
    nt = np.ascontiguousarray(notch_tet, np.int32)
    ns = np.ascontiguousarray(notch_side, np.uint8)
    d = MeshDesc()
    d.n_nodes, d.n_tets = len(X), len(tets)
    d.X = X.ctypes.data_as(C.POINTER(C.c_double))
    d.tets = tets.ctypes.data_as(C.POINTER(C.c_int32))
    d.n_notch = len(nt)
    d.notch_tet = nt.ctypes.data_as(C.POINTER(C.c_int32)) if len(nt) else None
    d.notch_side = ns.ctypes.data_as(C.POINTER(C.c_uint8)) if len(ns) else None
    d.precision = precision
    d.split_enabled = 1
    d.alloc, d.free = ALLOC_FN(), FREE_FN()
    return d, (X, tets, nt, ns)


UNIT = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])


@pytest.mark.parametrize("case,expect", [
    ("node_out_of_range", "out of range"),
    ("repeated_node", "repeated node"),
    ("zero_volume", "zero-volume"),
    ("bad_notch_mask", "side mask"),
    ("notch_out_of_range", "out of range"),
    ("bad_precision", "CEM_FP64"),
    ("bad_split_mode", "split_mode"),
    ("bad_g_variant", "g_variant"),
    ("dir_twice", "prescribed twice"),
    ("dir_component", "out of range"),
    ("dir_node", "out of range"),
    ("dir_missing", "dir_node"),
    ("bad_elem_type", "elem_type"),
    ("bad_tface_nodes", "tface_nodes"),
    ("hex_with_splitting", "fixed topology"),
    ("hex_zero_volume", "positive volume"),
    ("empty_mesh", "required"),
    ("no_nodes", "required"),
])
def test_host_validation_rejects(lib, case, expect):
    X, tets, nt, ns, prec = UNIT, [[0, 1, 2, 3]], [], [], 0
    dirichlet = None
    if case == "node_out_of_range":
        tets = [[0, 1, 2, 4]]
    elif case == "repeated_node":
        tets = [[0, 1, 1, 3]]
    elif case == "zero_volume":
        X = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 0, 1.0]])
    elif case == "bad_notch_mask":
        nt, ns = [0], [15]
    elif case == "notch_out_of_range":
        nt, ns = [3], [1]
    elif case == "bad_precision":
        prec = 7
    elif case == "empty_mesh":
        tets = np.zeros((0, 4), np.int32)
    elif case == "no_nodes":
        X = np.zeros((0, 3))
    elif case == "dir_twice":
        dirichlet = ([1, 2, 1], [0, 0, 0], [0.0, 0.0, 1.0])
    elif case == "dir_component":
        dirichlet = ([1], [3], [0.0])
    elif case == "dir_node":
        dirichlet = ([4], [0], [0.0])
    hexX = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1.0]])
    if case == "hex_with_splitting":
        X, tets = hexX, [list(range(8))]
    elif case == "hex_zero_volume":
        X, tets = hexX, [[0, 3, 2, 1, 4, 7, 6, 5]]   # mirrored: negative volume
    d, keep = _desc(X, tets, nt, ns, prec)
    if case in ("hex_with_splitting", "hex_zero_volume"):
        d.elem_type = 1
        d.split_enabled = 1 if case == "hex_with_splitting" else 0
    if case == "bad_elem_type":
        d.elem_type = 5
    elif case == "bad_tface_nodes":
        d.tface_nodes = 5
    if case == "bad_split_mode":
        d.split_mode = 2
    elif case == "bad_g_variant":
        d.g_variant = -1
    elif case == "dir_missing":
        d.n_dirichlet = 1
    if dirichlet is not None:
        dn = np.ascontiguousarray(dirichlet[0], np.int32)
        dc = np.ascontiguousarray(dirichlet[1], np.uint8)
        dv = np.ascontiguousarray(dirichlet[2], np.float64)
        keep = keep + (dn, dc, dv)
        d.n_dirichlet = dn.size
        d.dir_node = dn.ctypes.data_as(C.POINTER(C.c_int32))
        d.dir_comp = dc.ctypes.data_as(C.POINTER(C.c_uint8))
        d.dir_v0 = dv.ctypes.data_as(C.POINTER(C.c_double))
    ctx = C.c_void_p()
    rc = lib.cem_mesh_create(C.byref(d), C.byref(ctx))
    assert rc == -1
    assert not ctx.value
    assert expect in lib.cem_last_error(None).decode()


def test_null_arguments(lib):
    assert lib.cem_mesh_create(None, None) == -1
    assert lib.cem_destroy(None) == 0
    assert lib.cem_step(None, 1) == -1
