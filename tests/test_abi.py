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
    assert p.fp64_residuals == 1            # IEEE FP64 reliable updates by default
    for code in (0, 1, -1, -2, -3, -4, -5, -6):
        assert len(L.dsbcg_error_string(code)) > 0
    # argument validation happens before any device work
    ctx = ctypes.c_void_p()
    bad = (ctypes.c_int * 4)(4, 4, 1, 4)
    assert L.dsbcg_create(ctypes.byref(ctx), bad, ctypes.c_void_p(1), 0.1, 1, None) == -1
    assert L.dsbcg_solve(None, 1, None, 1, None, 1e-8, None, None, None) == -1
    assert L.dsbcg_solve_rational(None, 1, None, 1, None, 0.0, None, 1e-8, None, None, None, None) == -1
    assert L.dsbcg_backward(None, 1, None, 1, None, None, None, None, 0.0, 1e-8, None, None, None, None, None,
                            None) == -1
    assert L.dsbcg_debug_shift_chunk(None, 1) == -1
    assert L.dsbcg_debug_first_wait(None, 0) == -1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(dsbcg, "_lib_handle", None)
    monkeypatch.setattr(dsbcg, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError):
        dsbcg.lib()


_LAYOUT_C = r"""
#include <stddef.h>
#include <stdio.h>
#include "dsbcg.h"
#define OFF(T, f) printf(#T " " #f " %zu\n", offsetof(T, f))
int main(void) {
    printf("dsbcg_params sizeof %zu\n", sizeof(dsbcg_params));
    OFF(dsbcg_params, storage); OFF(dsbcg_params, dtol); OFF(dsbcg_params, max_block_steps);
    OFF(dsbcg_params, max_restarts); OFF(dsbcg_params, restart_drop); OFF(dsbcg_params, poll_every);
    OFF(dsbcg_params, freeze_converged); OFF(dsbcg_params, refine); OFF(dsbcg_params, fp64_residuals);
    OFF(dsbcg_params, x0);
    printf("dsbcg_stats sizeof %zu\n", sizeof(dsbcg_stats));
    OFF(dsbcg_stats, block_steps); OFF(dsbcg_stats, mvms); OFF(dsbcg_stats, deflations);
    OFF(dsbcg_stats, restarts); OFF(dsbcg_stats, final_rank); OFF(dsbcg_stats, seconds);
    OFF(dsbcg_stats, true_relres); OFF(dsbcg_stats, conv_step); OFF(dsbcg_stats, kernel_ms);
    OFF(dsbcg_stats, kernel_launches); OFF(dsbcg_stats, kernel_bytes); OFF(dsbcg_stats, kernel_flops);
    printf("prec fp64 %d\nprec fp32 %d\nprec bf16 %d\nprec fp16 %d\nprec df32 %d\n", DSBCG_PREC_FP64,
           DSBCG_PREC_FP32, DSBCG_PREC_BF16, DSBCG_PREC_FP16, DSBCG_PREC_DF32);
    printf("op D %d\nop Ddag %d\nop A %d\n", DSBCG_OP_D, DSBCG_OP_DDAG, DSBCG_OP_A);
    printf("status OK %d\nstatus NOT_CONVERGED %d\nstatus ERR_ARG %d\nstatus ERR_NOT_HPD %d\n"
           "status ERR_CUDA %d\nstatus ERR_OOM %d\nstatus ERR_NONFINITE %d\nstatus ERR_UNSUPPORTED %d\n",
           DSBCG_OK, DSBCG_NOT_CONVERGED, DSBCG_ERR_ARG, DSBCG_ERR_NOT_HPD, DSBCG_ERR_CUDA, DSBCG_ERR_OOM,
           DSBCG_ERR_NONFINITE, DSBCG_ERR_UNSUPPORTED);
    printf("kclass dslash %d\nkclass gram %d\nkclass update %d\nkclass shift %d\nkclass small %d\n"
           "kclass residual %d\nkclass other %d\n", DSBCG_KCLASS_DSLASH, DSBCG_KCLASS_GRAM, DSBCG_KCLASS_UPDATE,
           DSBCG_KCLASS_SHIFT, DSBCG_KCLASS_SMALL, DSBCG_KCLASS_RESIDUAL, DSBCG_KCLASS_OTHER);
    return 0;
}
"""


def test_binding_matches_header_layout(tmp_path):
    """The ctypes structures and name tables of the binding agree with the C
    header: struct offsets and sizes (compiled with the host C compiler) and
    every enum and class constant."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            a, b, v = ln.split()
            got[(a, b)] = int(v)
    for T, name in ((dsbcg.Params, "dsbcg_params"), (dsbcg.Stats, "dsbcg_stats")):
        assert ctypes.sizeof(T) == got[(name, "sizeof")], name
        for f, _ in T._fields_:
            assert getattr(T, f).offset == got[(name, f)], (name, f)
    for k, v in dsbcg.PREC.items():
        assert got[("prec", k)] == v
    for k, v in dsbcg.OPS.items():
        assert got[("op", k)] == v
    for code, nm in dsbcg.STATUS.items():
        assert got[("status", nm)] == code
    for q, nm in enumerate(dsbcg.KCLASS[:7]):
        assert got[("kclass", nm)] == q


def test_product_never_reaches_the_oracle():
    """The library, its binding and the input generators import, include or
    name no module of oracle/ (the oracle is test infrastructure), and the
    oracle imports nothing of the product package (its inputs are passed in)."""
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_1205_0359_gb300")
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|#\s*include\s*[<\"][^>\"]*oracle", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, f)) as fh:
                    assert not pat.search(fh.read()), f
    with open(os.path.join(root, "include", "dsbcg.h")) as fh:
        assert "oracle" not in fh.read()
    opat = re.compile(r"^\s*(from|import)\s+paper_1205_0359_gb300\b", re.M)
    for f in os.listdir(os.path.join(root, "oracle")):
        if f.endswith(".py"):
            with open(os.path.join(root, "oracle", f)) as fh:
                assert not opat.search(fh.read()), f
