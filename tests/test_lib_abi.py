"""The C-ABI library loads and exports every function include/wcmg.h declares
(no compute calls: runs without a GPU)."""
import ctypes

import pytest


def test_library_exports_every_header_symbol():
    wcmg = pytest.importorskip("paper_1904_08678_gb300.wcmg")
    names = wcmg.header_functions()
    assert len(names) >= 20
    missing = [n for n in names if not wcmg.exported(n)]
    assert not missing, missing


def test_struct_layout_matches_header_defaults():
    wcmg = pytest.importorskip("paper_1904_08678_gb300.wcmg")
    p = wcmg.default_params()
    assert list(p.dims) == [4, 4, 4, 4] and p.n_levels == 2 and p.nvec[0] == 8
    assert p.outer_tol == 1e-10 and p.coarse_tol == 0.05 and p.smoother_steps == 4


def test_invalid_params_rejected_without_gpu_work():
    wcmg = pytest.importorskip("paper_1904_08678_gb300.wcmg")
    p = wcmg.default_params(dims=(4, 4, 4, 6), blocks=[(4, 4, 4, 4)])
    h = ctypes.c_void_p()
    assert wcmg.wcmg_create(ctypes.byref(p), ctypes.byref(h)) == wcmg.ERR_ARG
    p = wcmg.default_params(n_levels=7)
    assert wcmg.wcmg_create(ctypes.byref(p), ctypes.byref(h)) == wcmg.ERR_ARG
