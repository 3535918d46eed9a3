"""The C-ABI library loads without a GPU and exports every function include/lpdf.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lpdf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lpdf_\w+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for n in ("lpdf_mesh_load", "lpdf_particles_init", "lpdf_pdf_step", "lpdf_grid_statistics", "lpdf_sort",
              "lpdf_pdf_step_static", "lpdf_elliptic_relax_solve"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1006_0549_gb300 import _build, lpdf
    try:
        path = _build.build()
    except RuntimeError as e:          # no nvcc on this machine
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(lpdf.EXPORTS) == set(declared_functions())


def test_params_struct_layout_matches_header():
    """The binding's Params mirrors lpdf_params field by field (checked through the library's
    own defaults: lpdf_params_default needs no GPU)."""
    from paper_1006_0549_gb300 import _build, lpdf
    try:
        _build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    p = lpdf.Params()
    lpdf.lib().lpdf_params_default(ctypes.byref(p))
    assert (p.C3, p.C4, p.Cphi, p.C0, p.Comega1, p.Comega2) == (5.0, 0.25, 2.0, 2.1, 0.5, 0.73)
    assert p.ns == 1 and p.n_sources == 0 and p.seed == 1


def test_params_struct_size_matches_header():
    """lpdf_params_default writes exactly sizeof(Params) bytes: a sentinel after the struct stays
    untouched and the last field is written (so the library's struct is neither larger nor smaller)."""
    from paper_1006_0549_gb300 import _build, lpdf
    try:
        _build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    n = ctypes.sizeof(lpdf.Params)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    lpdf.lib().lpdf_params_default(ctypes.cast(buf, ctypes.c_void_p))
    assert all(b == 0xAB for b in bytes(buf)[n:])
    p = lpdf.Params.from_buffer_copy(bytes(buf)[:n])
    assert p.dpdx0 == 0.0 and p.dpdy0 == 0.0 and p.gmodel == 0 and p.pressure_solve == 0
