"""The C-ABI library builds, loads and exports every entry point that
include/vdwnl.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vdwnl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vdw_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_0812_0244_gb300 import build, vdwnl
    build.build()
    return vdwnl.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("vdw_kernel_table", "vdw_create", "vdw_plan", "vdw_energy_potential",
                     "vdw_energy_potential_host", "vdw_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_0812_0244_gb300 import vdwnl
    assert set(declared_functions()) <= set(vdwnl.EXPORTS)


def test_host_only_entry_points(lib):
    from paper_0812_0244_gb300 import vdwnl
    p = vdwnl._Params()
    assert lib.vdw_params_default(ctypes.byref(p)) == 0
    d = vdwnl.Params()
    assert (p.Nq, p.m_c, p.na, p.Nr, p.Nk) == (d.Nq, d.m_c, d.na, d.Nr, d.Nk)
    assert abs(p.q_c - d.q_c) == 0 and abs(p.lambda_ - d.lam) == 0 and p.k_max == d.k_max
    assert lib.vdw_error_string(-2) == b"unsupported grid size"
    assert lib.vdw_params_default(None) == -1
    assert lib.vdw_destroy(None) == -1
    assert lib.vdw_plan(None, 8, 8, 8, None) == -1
    assert lib.vdw_plan_cell(None, 8, 8, 8, None) == -1


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_0812_0244_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), f
                assert "vdw_oracle" not in txt, f
