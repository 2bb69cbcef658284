"""dsbcg_update_gauge through the C ABI.

* A context moved to a new gauge field computes bitwise what a fresh context
  on that field computes, in every storage precision, including precisions
  whose links had been packed for the old field; a solve after the update
  meets its tolerance on the new operator (checked with the oracle's FP64
  Wilson operator).
* A field with NaN is rejected (DSBCG_ERR_NONFINITE); the context then holds
  no field and refuses work (DSBCG_ERR_ARG) until the next good update.
"""
import numpy as np
import pytest
import torch

from oracle import wilson as W
from paper_1205_0359_gb300 import dsbcg, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


def test_update_gauge():
    dims = (4, 4, 4, 6)
    rng = np.random.Generator(np.random.PCG64(31))
    U1 = synth.su3_links(dims, 0.4, rng)
    U2 = synth.su3_links(dims, 0.6, rng)
    kappa = 0.12
    n = 12 * synth.volume(dims)
    F = torch.from_numpy(synth.gaussian_rhs(n, 3, rng)).to(DEV)
    B = synth.gaussian_rhs(n, 2, rng)
    sigma = [0.01, 0.1]
    tol = 1e-9
    ctx = dsbcg.Context(dims, torch.from_numpy(U1).to(DEV), kappa)
    fresh = dsbcg.Context(dims, torch.from_numpy(U2).to(DEV), kappa)
    try:
        for st in ("fp64", "fp32"):                     # links of the old field, packed
            ctx.apply("A", F, storage=st)
        X1, st1 = ctx.solve(torch.from_numpy(B).to(DEV), sigma, tol, storage="fp32")
        assert st1["code"] == 0

        ctx.update_gauge(torch.from_numpy(U2).to(DEV))
        for st in ("fp64", "fp32", "bf16"):
            assert torch.equal(ctx.apply("A", F, storage=st), fresh.apply("A", F, storage=st)), st
        Y = ctx.apply("A", F, storage="fp64").cpu().numpy()
        Yo = W.A_vec(U2, kappa, dims, F.cpu().numpy())
        assert np.max(np.abs(Y - Yo)) <= 1e-12 * np.max(np.abs(Yo))

        X2, st2 = ctx.solve(torch.from_numpy(B).to(DEV), sigma, tol, storage="fp32")
        assert st2["code"] == 0 and st2["true_relres"].max() <= tol
        for j in range(len(sigma)):
            for i in range(B.shape[0]):
                x = X2[j, i].cpu().numpy()
                r = B[i] - sigma[j] * x - W.A_vec(U2, kappa, dims, x)
                assert np.linalg.norm(r) <= 10 * tol * np.linalg.norm(B[i]), (j, i)
        # the old field's solution does not solve the new system
        x = X1[0, 0].cpu().numpy()
        r = B[0] - sigma[0] * x - W.A_vec(U2, kappa, dims, x)
        assert np.linalg.norm(r) > 1e-3 * np.linalg.norm(B[0])

        # a host (numpy) field is accepted as well
        ctx.update_gauge(U1)
        Yd = ctx.apply("D", F, storage="fp64").cpu().numpy()
        Ydo = W.D_vec(U1, kappa, dims, F.cpu().numpy())
        assert np.max(np.abs(Yd - Ydo)) <= 1e-12 * np.max(np.abs(Ydo))

        bad = U2.copy()
        bad[1, 2, 3, 0, 2, 1, 1] = np.nan
        with pytest.raises(dsbcg.DSBCGError) as e:
            ctx.update_gauge(torch.from_numpy(bad).to(DEV))
        assert e.value.code == -5
        for call in (lambda: ctx.apply("A", F, storage="fp64"),
                     lambda: ctx.apply_static("A", F, storage="fp64"),
                     lambda: ctx.solve(torch.from_numpy(B).to(DEV), sigma, tol, storage="fp32")):
            with pytest.raises(dsbcg.DSBCGError) as e:
                call()
            assert e.value.code == -1

        ctx.update_gauge(torch.from_numpy(U2).to(DEV))
        for st in ("fp64", "fp32"):
            assert torch.equal(ctx.apply("A", F, storage=st), fresh.apply("A", F, storage=st)), st
    finally:
        ctx.close()
        fresh.close()
