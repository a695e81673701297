"""The C-ABI library builds, loads without a GPU and exports every function
that include/*.h declares; host-side argument checks return error codes."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(dnnmg_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_07687_gb300 import build
    return ctypes.CDLL(build.build())


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "dnnmg_setup" in names and "dnnmg_vcycle" in names and "dnnmg_step" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_config_and_argument_errors(lib):
    from paper_2106_07687_gb300 import dnnmg
    dnnmg.load()
    cfg = dnnmg.default_config()
    assert ctypes.sizeof(cfg) == 168
    assert (cfg.nu, cfg.level_solve, cfg.level_coarse, cfg.gmres_m) == (0.01, 3, 1, 20)
    # fields late in the struct, written by the library: the ctypes layout matches the header
    assert (cfg.hidden, cfg.gru_layers, cfg.mlp_width, cfg.lps_mode) == (64, 2, 128, 0)
    assert (cfg.stream_pass, cfg.net_bias, cfg.net_inputs) == (0, 1, 0)
    assert (cfg.obstacle_i0, cfg.obstacle_j0, cfg.obstacle_level) == (2, 1, 0)
    L = dnnmg.load()
    assert L.dnnmg_default_config(None) == dnnmg.ERR_ARG
    out = ctypes.c_void_p(1)
    assert L.dnnmg_setup(None, None, ctypes.byref(out)) == dnnmg.ERR_ARG
    assert out.value is None
    for bad in (dict(level_coarse=0), dict(level_solve=12), dict(nu=-1.0), dict(gmres_m=0),
                dict(precision=7), dict(replaced_levels=5), dict(obstacle_i0=20),
                dict(coarse_refresh=0), dict(persistent_mode=3), dict(lps_mode=3), dict(lps_mode=-1),
                dict(obstacle_level=2), dict(obstacle_level=1, obstacle_i0=30),
                dict(obstacle_level=1, obstacle_j0=6), dict(obstacle_level=1, level_solve=1),
                dict(obstacle_level=1, obstacle_i0=1, obstacle_j0=2),
                dict(obstacle_level=1, obstacle_i0=6, obstacle_j0=1)):
        c = dnnmg.default_config(**bad)
        assert L.dnnmg_setup(ctypes.byref(c), None, ctypes.byref(out)) == dnnmg.ERR_ARG, bad
        assert out.value is None
        assert len(L.dnnmg_last_error(None)) > 0
    assert L.dnnmg_destroy(None) == dnnmg.OK
    assert L.dnnmg_step(None, 0, None) == dnnmg.ERR_ARG


def test_batch_argument_errors(lib):
    """Batch setup rejects bad inputs before touching the device: no configs,
    an invalid configuration, and problems that differ in a shared field."""
    from paper_2106_07687_gb300 import dnnmg
    L = dnnmg.load()
    out = ctypes.c_void_p(1)
    assert L.dnnmg_batch_setup(None, 0, None, ctypes.byref(out)) == dnnmg.ERR_ARG
    assert out.value is None
    assert len(L.dnnmg_batch_last_error(None)) > 0
    a = dnnmg.default_config()
    b = dnnmg.default_config(nu=-1.0)
    arr = (dnnmg.Config * 2)(a, b)
    assert L.dnnmg_batch_setup(arr, 2, None, ctypes.byref(out)) == dnnmg.ERR_ARG
    assert b"problem 1" in L.dnnmg_batch_last_error(None)
    c = dnnmg.default_config(gmres_m=10, level_solve=4)
    arr = (dnnmg.Config * 2)(a, c)
    assert L.dnnmg_batch_setup(arr, 2, None, ctypes.byref(out)) == dnnmg.ERR_ARG
    assert out.value is None
    # the obstacle snapped to level-1 cells is for single contexts only
    d = dnnmg.default_config(obstacle_level=1, obstacle_i0=5, obstacle_j0=3)
    arr = (dnnmg.Config * 2)(a, d)
    assert L.dnnmg_batch_setup(arr, 2, None, ctypes.byref(out)) == dnnmg.ERR_ARG
    assert b"level-0 obstacle" in L.dnnmg_batch_last_error(None)
    assert out.value is None
    assert L.dnnmg_batch_destroy(None) == dnnmg.OK
    assert L.dnnmg_batch_step(None, 0, None) == dnnmg.ERR_ARG
    n, length = ctypes.c_int(), ctypes.c_int64()
    assert L.dnnmg_batch_size(None, ctypes.byref(n), ctypes.byref(length)) == dnnmg.ERR_ARG
