"""Degenerate right-hand sides through the C ABI.

* A zero right-hand side among others: its direction is deflated at the
  start (its creation norm is zero), x_ij = 0 exactly for every shift, and
  the other systems still meet tol on the oracle's FP64 operator.
* B = 0: no Krylov vector is built and X = 0 is returned as converged.
"""
import numpy as np
import pytest
import torch

from oracle import wilson as W
from paper_1205_0359_gb300 import dsbcg, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


@pytest.fixture(scope="module")
def lat():
    dims = (4, 4, 4, 6)
    rng = np.random.Generator(np.random.PCG64(57))
    U = synth.su3_links(dims, 0.4, rng)
    kappa = 0.12
    n = 12 * synth.volume(dims)
    B = synth.gaussian_rhs(n, 4, rng)
    ctx = dsbcg.Context(dims, torch.from_numpy(U).to(DEV), kappa)
    yield dims, U, kappa, B, ctx
    ctx.close()


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_zero_right_hand_side(lat, storage):
    dims, U, kappa, B, ctx = lat
    Bz = B.copy()
    Bz[2] = 0.0
    sigma = [0.01, 0.1, 1.0]
    tol = 1e-9
    X, st = ctx.solve(torch.from_numpy(Bz).to(DEV), sigma, tol, storage=storage)
    assert st["code"] == 0, st["status"]
    Xc = X.cpu().numpy()
    assert np.all(Xc[:, 2] == 0)
    assert np.all(st["true_relres"][:, 2] == 0)
    for j, sg in enumerate(sigma):
        for i in (0, 1, 3):
            r = Bz[i] - sg * Xc[j, i] - W.A_vec(U, kappa, dims, Xc[j, i])
            assert np.linalg.norm(r) <= 10 * tol * np.linalg.norm(Bz[i]), (storage, j, i)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_all_zero_B(lat, storage):
    dims, U, kappa, B, ctx = lat
    Z = torch.zeros((3, B.shape[1]), dtype=torch.complex128, device=DEV)
    X, st = ctx.solve(Z, [0.01, 0.5], 1e-9, storage=storage)
    assert st["code"] == 0, st["status"]
    assert bool(torch.all(X == 0))
    assert np.all(st["true_relres"] == 0)
