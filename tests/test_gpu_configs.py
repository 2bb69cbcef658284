"""GPU solves of the two largest workloads, checked through the oracle.

The oracle's solver cannot run at these sizes, so every check is one it can
make at any size: residuals b_i - (sigma_j + A) x_ij recomputed with the
oracle's own FP64 Wilson operator for sampled (i, j), against the tolerance
of the solve.

* 24^3 x 48, m = s = 8: the storage precision ladder FP64, FP32, BF16, FP16
  (FP32/16-bit storage inside the reliable-update loop).  Every storage meets
  tol; the per-(rhs, shift) difference to the FP64-storage solution is
  reported and bounded.
* 32^3 x 64, m = 16, s = 8, b_16 = b_1 + 1e-9 noise: FP32 storage, the
  near-dependent right-hand side is deflated, x_16 stays next to x_1.
"""
import numpy as np
import pytest
import torch

from oracle import wilson as W
from paper_1205_0359_gb300 import dsbcg, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


def _oracle_relres(wl, X, j, i):
    x = X[j, i].cpu().numpy()
    r = wl["B"][i] - wl["sigma"][j] * x - W.A_vec(wl["U"], wl["kappa"], wl["dims"], x)
    return np.linalg.norm(r) / np.linalg.norm(wl["B"][i])


@pytest.fixture(scope="module")
def w3():
    wl = synth.make_workload("w3_24x24x24x48")
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(DEV), wl["kappa"])
    yield wl, ctx
    ctx.close()


def test_w3_precision_ladder(w3):
    wl, ctx = w3
    B = torch.from_numpy(wl["B"]).to(DEV)
    tol = wl["tol"]
    X64, st64 = ctx.solve(B, wl["sigma"], tol, storage="fp64")
    assert st64["code"] == 0 and st64["true_relres"].max() <= tol
    assert _oracle_relres(wl, X64, 0, 0) <= 10 * tol
    n64 = torch.linalg.vector_norm(X64, dim=-1)
    for storage in ("fp32", "bf16", "fp16"):
        X, st = ctx.solve(B, wl["sigma"], tol, storage=storage)
        assert st["code"] == 0, (storage, st["status"])
        assert st["true_relres"].max() <= tol, storage
        for (j, i) in [(0, 7), (7, 3)]:
            rel = _oracle_relres(wl, X, j, i)
            assert rel <= 10 * tol, (storage, j, i, rel)
        # per (rhs, shift) difference to the FP64-storage solution: both meet
        # tol, so it is bounded by the conditioning of sigma_j + A
        err = (torch.linalg.vector_norm(X - X64, dim=-1) / n64).cpu().numpy()
        assert err.max() <= 1e-4, (storage, err.max())
        del X


def test_w5_full_size_near_dependent():
    wl = synth.make_workload("w5_32x32x32x64")
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(DEV), wl["kappa"])
    try:
        B = torch.from_numpy(wl["B"]).to(DEV)
        X, st = ctx.solve(B, wl["sigma"], wl["tol"], storage="fp32")
        assert st["code"] == 0, st["status"]
        assert st["true_relres"].max() <= wl["tol"]
        assert st["deflations"] >= 1
        m = wl["B"].shape[0]
        for (j, i) in [(0, 0), (7, m - 1)]:
            rel = _oracle_relres(wl, X, j, i)
            assert rel <= 10 * wl["tol"], (j, i, rel)
        # b_16 - b_1 is 1e-9 noise, so x_16 - x_1 is tiny for every shift
        d = torch.linalg.vector_norm(X[:, m - 1] - X[:, 0], dim=-1) / torch.linalg.vector_norm(X[:, 0], dim=-1)
        assert float(d.max()) <= 1e-5, float(d.max())
        del X, B
    finally:
        ctx.close()
