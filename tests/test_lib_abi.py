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


def test_graph_and_autotune_params_validated_without_gpu_work():
    wcmg = pytest.importorskip("paper_1904_08678_gb300.wcmg")
    p = wcmg.default_params()
    assert p.use_graphs == 0 and p.autotune == 0 and p.profile == 0 and p.max_rhs == 1
    h = ctypes.c_void_p()
    for field, bad in (("use_graphs", 2), ("autotune", 2), ("smoother", 3), ("kcycle", 2), ("kcycle_steps", 0),
                       ("kcycle_tol", -1.0), ("sap_cycles", 0), ("sap_cycles", 17), ("sap_eo", 2), ("smoother_steps", 65)):
        q = wcmg.default_params(**{field: bad})
        assert wcmg.wcmg_create(ctypes.byref(q), ctypes.byref(h)) == wcmg.ERR_ARG, field
    q = wcmg.default_params()
    assert q.kcycle == 0 and q.kcycle_steps == 5 and q.kcycle_tol == 0.1 and q.smoother == wcmg.SMOOTHER_MR
    assert q.sap_cycles == 1 and q.sap_eo == 0 and wcmg.SMOOTHER_SAP == 2
    # even-odd block solves need fine aggregates with an even x extent and <= 256 sites
    for blk in ((3, 2, 2, 2), (4, 4, 4, 8)):
        q = wcmg.default_params(dims=(12, 8, 8, 8), blocks=[blk], nvec=[4], sap_eo=1, smoother=wcmg.SMOOTHER_SAP)
        assert wcmg.wcmg_create(ctypes.byref(q), ctypes.byref(h)) == wcmg.ERR_ARG, blk


def test_batch_solve_rejects_empty_batch_without_gpu_work():
    wcmg = pytest.importorskip("paper_1904_08678_gb300.wcmg")
    assert wcmg.wcmg_solve_batch(None, 0, None, None, None, wcmg.DEVICE, None, None) == wcmg.ERR_ARG


def test_tile_and_stats_structs_match_header_sizes():
    """wcmg_tile: 8 ints + 2 doubles; wcmg_stats ends with the kernel-class array."""
    wcmg = pytest.importorskip("paper_1904_08678_gb300.wcmg")
    assert ctypes.sizeof(wcmg.wcmg_tile) == 8 * 4 + 2 * 8
    assert wcmg.wcmg_stats.k.offset % 8 == 0
    assert ctypes.sizeof(wcmg.wcmg_stats) == wcmg.wcmg_stats.k.offset + wcmg.NKCLASS * ctypes.sizeof(wcmg.wcmg_kstat)


def test_new_boundary_calls_reject_null_context_without_gpu_work():
    """set_clover / set_clover_raw / solve_ex / save_net / load_net check their context
    before any device work; wcmg_solve_opts is four ints."""
    wcmg = pytest.importorskip("paper_1904_08678_gb300.wcmg")
    assert ctypes.sizeof(wcmg.wcmg_solve_opts) == 16
    assert wcmg.wcmg_set_clover(None, 1.0, None) == wcmg.ERR_ARG
    assert wcmg.wcmg_set_clover_raw(None, None, wcmg.DEVICE, None) == wcmg.ERR_ARG
    o = wcmg.wcmg_solve_opts(zero_guess=1)
    assert wcmg.wcmg_solve_ex(None, None, None, 1, ctypes.byref(o), wcmg.DEVICE, None, None) == wcmg.ERR_ARG
    assert wcmg.wcmg_save_net(None, b"x") == wcmg.ERR_ARG
    assert wcmg.wcmg_load_net(None, b"x") == wcmg.ERR_ARG


def test_even_odd_coarsest_solve_needs_even_coarse_extents_without_gpu_work():
    """coarse_eo is rejected when the coarsest lattice has an odd extent (a hop across its
    periodic boundary would join sites of equal parity)."""
    wcmg = pytest.importorskip("paper_1904_08678_gb300.wcmg")
    h = ctypes.c_void_p()
    p = wcmg.default_params(dims=(4, 4, 4, 6), blocks=[(2, 2, 2, 2)], nvec=[4], coarse_eo=1)  # coarse t = 3
    assert wcmg.wcmg_create(ctypes.byref(p), ctypes.byref(h)) == wcmg.ERR_ARG
    p = wcmg.default_params(coarse_eo=2)
    assert wcmg.wcmg_create(ctypes.byref(p), ctypes.byref(h)) == wcmg.ERR_ARG
