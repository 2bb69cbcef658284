"""The C-ABI library loads on a machine without a GPU and exports every
function that include/dsbcg.h declares (no compute calls here)."""
import ctypes
import os

import pytest

from paper_1205_0359_gb300 import dsbcg


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(dsbcg.LIB_PATH):
        from paper_1205_0359_gb300 import build
        build.build()
    return dsbcg.lib()


def test_header_symbols_exported(L):
    names = dsbcg.header_symbols()
    assert "dsbcg_solve" in names and "dsbcg_create" in names and "dsbcg_force" in names
    raw = ctypes.CDLL(dsbcg.LIB_PATH)
    for nm in names:
        assert hasattr(raw, nm), f"{nm} not exported"


def test_host_only_calls(L):
    assert L.dsbcg_version().startswith(b"dsbcg")
    p = dsbcg.Params()
    L.dsbcg_params_default(ctypes.byref(p))
    assert p.storage == 1 and p.freeze_converged == 1 and p.max_restarts > 0
    for code in (0, 1, -1, -2, -3, -4, -5, -6):
        assert len(L.dsbcg_error_string(code)) > 0
    # argument validation happens before any device work
    ctx = ctypes.c_void_p()
    bad = (ctypes.c_int * 4)(4, 4, 1, 4)
    assert L.dsbcg_create(ctypes.byref(ctx), bad, ctypes.c_void_p(1), 0.1, 1, None) == -1
    assert L.dsbcg_solve(None, 1, None, 1, None, 1e-8, None, None, None) == -1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(dsbcg, "_lib_handle", None)
    monkeypatch.setattr(dsbcg, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError):
        dsbcg.lib()
