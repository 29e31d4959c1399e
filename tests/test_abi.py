"""The C-ABI library builds, loads and exports every symbol include/qg.h
declares, and validates its arguments, all without a GPU (no compute call
is made here)."""
import ctypes
import os
import re

import pytest

from paper_1308_3290_gb300 import build, qg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "qg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qg_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return qg.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(qg.EXPORTS) == names


def test_status_strings(lib):
    assert qg.qg_status_string(0) == "ok"
    assert qg.qg_status_string(2) == "unsupported grid shape"
    assert qg.qg_status_string(99) == "unknown status"


def _basin(nx=64, ny=128, dt=1e-4):
    return qg.qg_basin(nx, ny, 0.0, 1.0, -1.0, 1.0, 1.0, 0.2, 0.0, dt, 0)


def _create(b, layers=1, Re=200.0, Ro=0.0016, Fr=0.0, levels=1, dtype=0):
    h = ctypes.c_void_p()
    st = qg.load().qg_create(ctypes.byref(b), layers, Re, Ro, Fr, levels, dtype, None,
                             ctypes.byref(h))
    if st == 0:
        qg.load().qg_destroy(h)
    return st


def test_argument_validation(lib):
    assert _create(_basin(48, 128)) == 2          # not a power of two
    assert _create(_basin(4, 128)) == 2           # too small
    assert _create(_basin(64, 128), levels=4) == 2  # coarse grid below 8 intervals
    assert _create(_basin(), layers=3) == 1
    assert _create(_basin(), Re=-1.0) == 1
    assert _create(_basin(dt=0.0)) == 1
    assert _create(_basin(), dtype=7) == 1
    b = _basin()
    b.flags = 1
    assert _create(b) == 1
    assert lib.qg_create(None, 1, 1.0, 1.0, 0.0, 0, 0, None, None) == 1


def test_calls_on_null_handle(lib):
    assert lib.qg_destroy(None) == 0
    assert lib.qg_step(None, 1) == 1
    assert lib.qg_set_state(None, None, 0) == 1
    assert lib.qg_synchronize(None) == 1
    assert lib.qg_inject_fault(None, 1) == 1
    assert lib.qg_set_solver(None, 1, 4) == 1
    assert lib.qg_set_cfl(None, 0.5) == 1
    assert lib.qg_stats_begin(None) == 1
    assert lib.qg_stats_end(None) == 1
    assert lib.qg_tape_begin(None, 1, 10) == 1
    assert lib.qg_adjoint_step(None, 1, None, None) == 1
    assert lib.qg_get_time(None, None, None) == 1
    assert lib.qg_set_timing_mask(None, 1) == 1
    assert lib.qg_solve_engine(None, None) == 1
    assert lib.qg_ensemble_step(None, 1) == 1
    assert lib.qg_ensemble_destroy(None) == 0
    e = ctypes.c_void_p()
    assert lib.qg_ensemble_create(None, None, None, None, 0, 0, None, ctypes.byref(e)) == 1


def test_no_device_is_reported():
    """On a machine without a GPU a valid request returns QG_ERR_NO_DEVICE."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    qg.load()
    assert _create(_basin()) == 9
