"""The C-ABI library builds, loads and exports every symbol include/hmc.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2210_06874_gb300 import build_lib, hmc

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "hmc.h")


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return hmc.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hmc_[A-Za-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("hmc_ctx_create", "hmc_ctx_destroy", "hmc_apply_M", "hmc_apply_Mdag",
                 "hmc_cg_solve", "hmc_force", "hmc_trajectory", "hmc_rng_draw"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in hmc.SIGNATURES, name


def test_version(lib):
    assert b"sm_103a" in lib.hmc_version()


def bad(**kw):
    p = hmc.Params(L=3, Nt=8).to_c()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("field,value", [("L", 0), ("Nt", 0), ("U", 0.0), ("beta", -1.0),
                                         ("n_md", 0), ("cg_tol", 0.0), ("cg_max_iter", 0),
                                         ("precision", 7), ("ru_delta", 1.5),
                                         ("L", 30000), ("operand_mode", 6),
                                         ("cluster_mode", 3), ("cluster_mode", -1),
                                         ("integrator", 2), ("integrator", -1),
                                         ("mu", float("nan")), ("mu", 100.0),
                                         ("traj_length", 0.0), ("kappa", float("inf")),
                                         ("team_ctas", -1), ("inner_ctas", 2000),
                                         ("tile_slices", 12), ("tile_slices", 64)])
def test_ctx_create_rejects_bad_params(lib, field, value):
    h = ctypes.c_void_p()
    p = bad(**{field: value})
    assert lib.hmc_ctx_create(ctypes.byref(p), ctypes.byref(h)) == hmc.HMC_ERR_BAD_ARG
    assert not h.value


@pytest.mark.parametrize("kw,ok", [(dict(operand_mode=4, tile_slices=64), True),
                                   (dict(operand_mode=4, tile_slices=65), False),
                                   (dict(operand_mode=1, tile_slices=32), True),
                                   (dict(mu=4.9 * 8 / 2.0), True),      # |delta mu| = 4.9
                                   (dict(mu=5.1 * 8 / 2.0), False)])
def test_ctx_create_limits(lib, kw, ok):
    """Parameters at the edge of what the kernels take pass the host checks
    (then the context is created, or the missing device is reported);
    just beyond the edge they are refused before any CUDA call."""
    h = ctypes.c_void_p()
    p = bad(**kw)
    code = lib.hmc_ctx_create(ctypes.byref(p), ctypes.byref(h))
    if ok:
        assert code in (hmc.HMC_OK, hmc.HMC_ERR_CUDA)
        if code == hmc.HMC_OK:
            lib.hmc_ctx_destroy(h)
    else:
        assert code == hmc.HMC_ERR_BAD_ARG and not h.value


def test_null_arguments_rejected(lib):
    assert lib.hmc_ctx_create(None, None) == hmc.HMC_ERR_BAD_ARG
    assert lib.hmc_ctx_destroy(None) == hmc.HMC_OK
    assert lib.hmc_apply_M(None, None, None, None, 0, None) == hmc.HMC_ERR_BAD_ARG
    assert lib.hmc_apply_Mdag(None, None, None, None, 0, None) == hmc.HMC_ERR_BAD_ARG
    st = hmc.hmc_cg_stats()
    assert lib.hmc_cg_solve(None, None, None, None, 1e-10, 10, 0, ctypes.byref(st),
                            None) == hmc.HMC_ERR_BAD_ARG
    assert lib.hmc_force(None, None, None, None, None) == hmc.HMC_ERR_BAD_ARG
    out = hmc.hmc_traj_out()
    assert lib.hmc_trajectory(None, None, 0, 0, 0, ctypes.byref(out), None) == \
        hmc.HMC_ERR_BAD_ARG
    assert lib.hmc_rng_draw(0, 0, 0, 0, -1, None, None, None, None) == hmc.HMC_ERR_BAD_ARG
    assert lib.hmc_get_transfer_matrix(None, None, 0) == hmc.HMC_ERR_BAD_ARG
    assert lib.hmc_spin_traces(None, None, 1, 0, 0, 1e-10, 10, 0, None, None, ctypes.byref(st),
                               None) == hmc.HMC_ERR_BAD_ARG
