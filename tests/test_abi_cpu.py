"""Host-side checks of the C ABI: the library builds, loads without a GPU,
exports every function the header declares, and rejects bad arguments on the
host before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2208_12795_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


def _declared(header="fempic_env.h"):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fempic_\w+)\s*\(", txt)))


def test_header_declares_what_binding_exports():
    assert sorted(capi.EXPORTS) == _declared()
    assert sorted(capi.DS_EXPORTS) == _declared("fempic_downshift.h")


def test_every_header_is_covered():
    assert sorted(os.listdir(os.path.join(ROOT, "include"))) == ["fempic_downshift.h", "fempic_env.h"]


def test_library_exports_every_declared_symbol(lib):
    for name in _declared() + _declared("fempic_downshift.h"):
        assert hasattr(lib, name), name


def test_debug_build_exports_the_same_symbols(lib):
    """The bounds-checked debug build (FEMPIC_BOUNDS_CHECK) is built beside
    the release library and loads without a GPU."""
    dbg = C.CDLL(build.DEBUG_LIB)
    for name in _declared() + _declared("fempic_downshift.h"):
        assert hasattr(dbg, name), name


def test_downshift_plane_layout_matches_header():
    txt = open(os.path.join(ROOT, "include", "fempic_downshift.h")).read()
    got = {k: int(v) for k, v in re.findall(r"#define FEMPIC_DS_(\w+) (\d+)", txt)}
    assert got == {"VH": capi.FEMPIC_DS_VH, "F": capi.FEMPIC_DS_F, "VN": capi.FEMPIC_DS_VN,
                   "U": capi.FEMPIC_DS_U, "PLANES": capi.FEMPIC_DS_PLANES}
    # 3 velocity levels + 2 complex E~, B~ sample levels + 2 scratch vectors
    assert got["F"] == 9 and got["VN"] == 9 + 24 and got["PLANES"] == got["U"] + 3


def test_downshift_null_arguments_rejected_on_host(lib):
    assert lib.fempic_downshift_create(None, None) == capi.FEMPIC_EINVAL
    assert "NULL" in capi.fempic_downshift_last_error()
    assert lib.fempic_push_step_downshift(None, None, None, None, None, 0.0, 0.0, 1e-9, 1, None) == \
        capi.FEMPIC_EINVAL
    w = (C.c_double * 24)()
    assert lib.fempic_downshift_weights(0.0, -1.0, 1.0, w) == capi.FEMPIC_EINVAL
    assert lib.fempic_downshift_weights(float("nan"), 1.0, 1.0, w) == capi.FEMPIC_EINVAL
    assert lib.fempic_downshift_debug_set_table(None, capi.FEMPIC_TABLE_EDGE, 0, 0) == capi.FEMPIC_EINVAL
    lib.fempic_downshift_destroy(None)   # safe on NULL


def test_null_arguments_rejected_on_host(lib):
    assert lib.fempic_env_create(None, None, None) == capi.FEMPIC_EINVAL
    assert "NULL" in capi.fempic_last_error()
    assert lib.fempic_locate(None, None, None) == capi.FEMPIC_EINVAL
    assert lib.fempic_push_step(None, None, None, 0.0, 0.0, 1e-9, None) == capi.FEMPIC_EINVAL
    assert lib.fempic_deposit(None, 0.0, 0.0, None, None, None, None) == capi.FEMPIC_EINVAL
    assert lib.fempic_stats(None, None, None) == capi.FEMPIC_EINVAL
    lib.fempic_env_destroy(None)   # safe on NULL


def test_bad_options_rejected_before_device(lib):
    nodes = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    tets = np.array([[0, 1, 2, 3]], np.int32)
    d = capi.fempic_mesh_desc(4, 1, nodes.ctypes.data, tets.ctypes.data, (C.c_double * 3)(0, 0, 0),
                              (C.c_double * 3)(1, 1, 1))
    h = C.c_void_p()
    for opt in (capi.fempic_options(7, 10, 0, 0), capi.fempic_options(0, -1, 0, 0),
                capi.fempic_options(0, 10, 5, 0), capi.fempic_options(0, 10, 0, 3)):
        assert lib.fempic_env_create(C.byref(d), C.byref(opt), C.byref(h)) == capi.FEMPIC_EINVAL
        assert not h.value


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(capi.FempicError):
        capi._lib_backup = capi._lib
        try:
            capi._lib = None
            capi.load(str(tmp_path / "nope.so"))
        finally:
            capi._lib = capi._lib_backup


def _desc(nodes, tets):
    nodes = np.ascontiguousarray(nodes, float)
    tets = np.ascontiguousarray(tets, np.int32)
    d = capi.fempic_mesh_desc(nodes.shape[0], tets.shape[0], nodes.ctypes.data, tets.ctypes.data,
                              (C.c_double * 3)(0, 0, 0), (C.c_double * 3)(1, 1, 1))
    return d, (nodes, tets)


@pytest.mark.parametrize("what,nodes,tets,code,msg", [
    ("zero volume", [[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], [[0, 1, 2, 3]], capi.FEMPIC_EMESH, "zero-volume"),
    ("repeated node", [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], [[0, 0, 1, 2]], capi.FEMPIC_EMESH, "repeated"),
    ("face in three tets", [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.2, 0.2, 1], [0.2, 0.2, -1], [0.3, 0.3, 0.5]],
     [[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]], capi.FEMPIC_EMESH, "non-conforming"),
    ("node id out of range", [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], [[0, 1, 2, 7]], None, "out of range"),
])
def test_bad_meshes_rejected_by_the_host_builder(lib, what, nodes, tets, code, msg):
    """The library's host mesh builder (shared by fempic_env_create and
    fempic_downshift_create) rejects degenerate and non-conforming meshes
    with an error code and a message, before any device work."""
    d, keep = _desc(nodes, tets)
    h = C.c_void_p()
    rc = lib.fempic_downshift_create(C.byref(d), C.byref(h))
    assert rc != capi.FEMPIC_OK and not h.value, what
    if code is not None:
        assert rc == code, (what, rc)
    assert msg in capi.fempic_downshift_last_error(), capi.fempic_downshift_last_error()
