"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header declares.

No compute call is made here (no GPU in this environment)."""
import ctypes as C
import os
import re

import pytest

from paper_1301_5914_gb300 import build, hobi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "hobi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(?:int|void|const char\s*\*)\s+(hobi_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_binding_exports():
    assert sorted(hobi.EXPORTS) == _declared_functions()


def test_library_builds_loads_and_exports():
    path = build.build()
    assert os.path.exists(path)
    lib = C.CDLL(path)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    # host-only calls that need no GPU
    hobi.load_library(path)
    opt = hobi.Options()
    hobi._lib.hobi_default_options(C.byref(opt))
    assert opt.precision == hobi.HOBI_FP32_BULK and opt.restart == 50 and opt.use_graph == 1
    assert opt.fast_degree == 0 and abs(opt.fast_theta - 0.7) < 1e-15
    assert opt.gmres_scaling == 1  # GMRES on the diagonally scaled unknowns by default
    assert isinstance(hobi._lib.hobi_last_error(), bytes)  # thread-local message of the last failing call


def test_null_arguments_rejected_without_gpu():
    hobi.load_library()
    h = C.c_void_p()
    rc = hobi._lib.hobi_setup(None, 0, None, 0, None, None, 0, 1.0, 80.0, 0.0, None, C.byref(h))
    assert rc == hobi.HOBI_ERR_ARG
    assert b"non-NULL" in hobi._lib.hobi_last_error()
    assert hobi._lib.hobi_matvec(None, None, None) == hobi.HOBI_ERR_ARG
    assert hobi._lib.hobi_energy(None, None) == hobi.HOBI_ERR_ARG
    assert hobi._lib.hobi_reaction_field(None, None, 0, None) == hobi.HOBI_ERR_ARG
    assert hobi._lib.hobi_reaction_forces(None, None) == hobi.HOBI_ERR_ARG
    assert hobi._lib.hobi_reaction_forces_batch(None, None) == hobi.HOBI_ERR_ARG
