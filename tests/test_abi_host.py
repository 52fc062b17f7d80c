"""The C-ABI library loads and exports every entry point that include/rd.h declares, and the
host-side argument checks answer without touching a GPU (no compute call here)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2308_07403_gb300 import build, rd

    build.build()
    return rd.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rd_[a-z_]+)\s*\(", text)))


def test_header_and_binding_agree(lib):
    from paper_2308_07403_gb300 import rd

    decl = declared_functions()
    assert decl, "no declarations found"
    assert sorted(rd.exported_symbols()) == decl


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2308_07403_gb300",
                                                                     "_build", "librd.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rd_[a-z_]+)\b", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        getattr(lib, f)


def test_host_side_errors_without_gpu(lib):
    from paper_2308_07403_gb300 import rd

    h = ctypes.c_void_p()
    A = np.zeros((4, 4), dtype=np.uint8)
    pa = A.ctypes.data_as(ctypes.c_void_p)
    assert lib.rd_create(None, 4, 0.1, ctypes.byref(h)) == rd.RD_ERR_ARG
    assert lib.rd_create(pa, 0, 0.1, ctypes.byref(h)) == rd.RD_ERR_ARG
    assert lib.rd_create(pa, 4, 1.5, ctypes.byref(h)) == rd.RD_ERR_GAMMA
    assert lib.rd_create(pa, 4, 0.0, ctypes.byref(h)) == rd.RD_ERR_GAMMA
    assert lib.rd_create(pa, 4, float("nan"), ctypes.byref(h)) == rd.RD_ERR_GAMMA
    assert lib.rd_create(pa, 4, 0.1, None) == rd.RD_ERR_ARG
    assert b"gamma" in lib.rd_last_error(None) or b"NULL" in lib.rd_last_error(None)
    assert lib.rd_create_weighted(pa, None, 4, 0.1, ctypes.byref(h)) == rd.RD_ERR_ARG
    assert lib.rd_apsp(None, None, None) == rd.RD_ERR_ARG
    assert lib.rd_goal_solve(None, None, 1, None) == rd.RD_ERR_ARG
    assert lib.rd_greedy_next(None, None, 1, None, None) == rd.RD_ERR_ARG
    assert lib.rd_set_tau(None, 1e-9) == rd.RD_ERR_ARG
    assert lib.rd_set_precision(None, 0, 0) == rd.RD_ERR_ARG
    assert lib.rd_sync(None) == rd.RD_ERR_ARG
    lib.rd_destroy(None)
    for s in range(9):
        assert lib.rd_status_string(s).startswith(b"RD_")


def test_binding_raises_typed_errors(lib):
    from paper_2308_07403_gb300 import rd

    with pytest.raises(rd.RDError) as ei:
        rd.rd_create(np.zeros((3, 3), np.uint8), 3, 2.0)
    assert ei.value.status == rd.RD_ERR_GAMMA
