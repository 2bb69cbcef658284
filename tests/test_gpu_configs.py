"""GPU solves of the two largest workloads, checked through the oracle.

The oracle's solver cannot run at these sizes, so every check is one it can
make at any size: residuals b_i - (sigma_j + A) x_ij recomputed with the
oracle's own FP64 Wilson operator (tests/oracle_check.py), against the
tolerance of the solve.

* 24^3 x 48, m = s = 8: the storage precision ladder FP64, FP32, BF16, FP16
  (FP32/16-bit storage inside the FP64 reliable-update loop).  The FP64-
  storage solution is certified by the oracle for all 64 (rhs, shift)
  systems; every other storage meets 10 tol on all 64 systems too, and its
  per-(rhs, shift) error against the certified FP64-storage solution is
  bounded.
* 32^3 x 64, m = 16, s = 8, b_16 = b_1 + 1e-9 noise: FP32 storage, the
  near-dependent right-hand side is deflated, x_16 stays next to x_1; every
  right-hand side of the smallest and of the largest shift is certified by
  the oracle.
"""
import numpy as np
import pytest
import torch

from oracle_check import relres_all
from paper_1205_0359_gb300 import dsbcg, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


@pytest.fixture()
def w3():
    wl = synth.make_workload("w3_24x24x24x48")
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(DEV), wl["kappa"])
    yield wl, ctx
    ctx.close()


def _certify(wl, X, st, shifts=None, rows=None):
    """Oracle residuals of the chosen pairs: each <= 10 tol, and the
    library's own FP64 true residual agrees with it to tol / 100."""
    tol = wl["tol"]
    rel = relres_all(wl, X, shifts, rows)
    done = ~np.isnan(rel)
    assert done.any()
    assert (rel[done] <= 10 * tol).all(), (np.argwhere(done & (rel > 10 * tol)), np.nanmax(rel))
    diff = np.abs(rel[done] - st["true_relres"][done])
    assert diff.max() <= 1e-2 * tol, diff.max()
    return rel


def test_w3_precision_ladder(w3):
    wl, ctx = w3
    B = torch.from_numpy(wl["B"]).to(DEV)
    tol = wl["tol"]
    X64, st64 = ctx.solve(B, wl["sigma"], tol, storage="fp64")
    assert st64["code"] == 0 and st64["true_relres"].max() <= tol
    _certify(wl, X64, st64)
    n64 = torch.linalg.vector_norm(X64, dim=-1)
    for storage in ("fp32", "bf16", "fp16"):
        X, st = ctx.solve(B, wl["sigma"], tol, storage=storage)
        assert st["code"] == 0, (storage, st["status"])
        assert st["true_relres"].max() <= tol, storage
        _certify(wl, X, st)
        # per (rhs, shift) error against the certified FP64-storage solution:
        # both meet tol, so it is bounded by the conditioning of sigma_j + A
        err = (torch.linalg.vector_norm(X - X64, dim=-1) / n64).cpu().numpy()
        assert err.max() <= 1e-4, (storage, err.max())
        del X


def test_w5_full_size_near_dependent():
    # the solve's workspace is about 170 GB: give back what earlier tests
    # left in torch's cache
    torch.cuda.empty_cache()
    wl = synth.make_workload("w5_32x32x32x64")
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(DEV), wl["kappa"])
    try:
        B = torch.from_numpy(wl["B"]).to(DEV)
        X, st = ctx.solve(B, wl["sigma"], wl["tol"], storage="fp32")
        assert st["code"] == 0, st["status"]
        assert st["true_relres"].max() <= wl["tol"]
        assert st["deflations"] >= 1
        m, s = wl["B"].shape[0], len(wl["sigma"])
        # every right-hand side of the smallest and of the largest shift
        _certify(wl, X, st, shifts=[0, s - 1])
        # b_16 - b_1 is 1e-9 noise, so x_16 - x_1 is tiny for every shift
        d = torch.linalg.vector_norm(X[:, m - 1] - X[:, 0], dim=-1) / torch.linalg.vector_norm(X[:, 0], dim=-1)
        assert float(d.max()) <= 1e-5, float(d.max())
        del X, B
    finally:
        ctx.close()
