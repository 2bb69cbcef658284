"""GPU force kernel and autograd backward against the oracle's gradients.

The oracle's gradients are pinned by central finite differences
(tests/test_oracle_force.py); here the GPU force kernel (dsbcg_force) is
compared with them element by element, and the autograd wrapper's
gradients w.r.t. B, sigma and the links are compared with the oracle and
with central finite differences of the GPU solve itself (step 1e-6, FP64).
"""
import numpy as np
import pytest
import torch

from oracle import wilson as W
from oracle.dsbcg import dense_solve
from oracle.force import link_gradient, rhmc_gradients, rhmc_loss
from paper_1205_0359_gb300 import dsbcg, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


@pytest.fixture(scope="module")
def w4():
    wl = synth.make_workload("w4_grad_4x4x4x4")
    Ad = W.dense_A(wl["U"], wl["kappa"], wl["dims"])
    X = dense_solve(Ad, wl["B"], wl["sigma"])
    return wl, Ad, X


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_force_kernel_matches_oracle(w4, storage, tol):
    wl, Ad, X = w4
    rng = np.random.Generator(np.random.PCG64(8))
    Lam = synth.gaussian_rhs(X.shape[-1], X.shape[0] * X.shape[1], rng).reshape(X.shape)
    w = np.array([0.3, 1.0, 2.0])
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(DEV), wl["kappa"])
    got = ctx.force(torch.from_numpy(X).to(DEV), torch.from_numpy(Lam).to(DEV), w, storage=storage)
    want = link_gradient(wl["U"], wl["kappa"], wl["dims"], X, Lam, w)
    err = np.linalg.norm(got.cpu().numpy() - want) / np.linalg.norm(want)
    assert err < tol
    ctx.close()


def test_autograd_matches_oracle_and_fd(w4):
    wl, Ad, X = w4
    alpha = torch.tensor(wl["weights"], dtype=torch.float64)
    args = dict(dims=wl["dims"], kappa=wl["kappa"], tol=1e-12, storage="fp64")

    def loss_of(Bt, st, Ut):
        Xt = dsbcg.DSBCGSolve.apply(Bt, st, Ut, args)
        return sum(alpha[j] * torch.real(torch.sum(torch.conj(Bt) * Xt[j])) for j in range(len(alpha)))

    Bt = torch.from_numpy(wl["B"]).to(DEV).requires_grad_(True)
    st = torch.tensor(wl["sigma"], dtype=torch.float64).requires_grad_(True)
    Ut = torch.from_numpy(wl["U"]).to(DEV).requires_grad_(True)
    L = loss_of(Bt, st, Ut)
    L.backward()
    gB, gs, gU = rhmc_gradients(wl["U"], wl["kappa"], wl["dims"], wl["B"], wl["sigma"], wl["weights"], X)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert abs(L.item() - rhmc_loss(wl["B"], X, wl["weights"])) < 1e-9 * abs(L.item())
    assert rel(Bt.grad.cpu().numpy(), gB) < 1e-8
    assert rel(st.grad.numpy(), gs) < 1e-8
    assert rel(Ut.grad.cpu().numpy(), gU) < 1e-8
    # central finite differences of the GPU solve itself
    h = 1e-6
    rng = np.random.Generator(np.random.PCG64(12))
    with torch.no_grad():
        for _ in range(2):
            dU = torch.from_numpy(rng.standard_normal(wl["U"].shape) + 1j * rng.standard_normal(wl["U"].shape)).to(DEV)
            fd = (loss_of(Bt, st, Ut + h * dU) - loss_of(Bt, st, Ut - h * dU)).item() / (2 * h)
            an = torch.sum(torch.real(torch.conj(Ut.grad) * dU)).item()
            assert abs(fd - an) <= 1e-5 * abs(an)
        e = torch.zeros(3, dtype=torch.float64)
        e[0] = 1.0
        fd = (loss_of(Bt, st + h * e, Ut) - loss_of(Bt, st - h * e, Ut)).item() / (2 * h)
        assert abs(fd - st.grad[0].item()) <= 1e-5 * abs(st.grad[0].item())
