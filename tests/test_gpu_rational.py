"""dsbcg_solve_rational: Y = alpha_0 B + sum_j alpha_j (sigma_j + A)^{-1} B
(the rational-approximation use of the shifted solves, Sec. 1) against the
oracle.

* 4^4 workload: Y from the GPU against oracle.dsbcg.rational_combination of
  dense LU solutions, with and without the per-shift solutions written, on
  device and on host buffers, in FP64 and FP32 storage;
* partial fraction of 1/((x+a)(x+b)): Y equals a dense solve with the
  product (A + a)(A + b);
* A^{-1/2} B by an exponentially convergent trapezoidal quadrature
  (shifts e^{2u_k}, weights 2h/pi e^{u_k}) on a 2^4 lattice: within the
  quadrature's own spectral error bound of the exact A^{-1/2} B.
"""
import numpy as np
import pytest
import torch

from oracle import wilson as W
from oracle.dsbcg import dense_solve, rational_combination
from paper_1205_0359_gb300 import dsbcg, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


@pytest.fixture(scope="module")
def w1():
    wl = synth.make_workload("w1_4x4x4x4")
    Ad = W.dense_A(wl["U"], wl["kappa"], wl["dims"])
    Xd = dense_solve(Ad, wl["B"], wl["sigma"])
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(DEV), wl["kappa"])
    yield wl, Ad, Xd, ctx
    ctx.close()


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_rational_matches_oracle(w1, storage):
    wl, Ad, Xd, ctx = w1
    a0, alpha = 0.3, np.array([0.7, -0.2, 1.5, 0.05])
    want = rational_combination(wl["B"], Xd, a0, alpha)
    B = torch.from_numpy(wl["B"]).to(DEV)
    Y, st = ctx.solve_rational(B, wl["sigma"], a0, alpha, 1e-10, storage=storage)
    assert st["code"] == 0 and st["true_relres"].max() <= 1e-10
    assert _rel(Y.cpu().numpy(), want) <= 1e-7
    # with the per-shift solutions written as well: the same Y, and X as dsbcg_solve
    X = torch.empty((len(alpha),) + tuple(B.shape), dtype=torch.complex128, device=DEV)
    Y2, _ = ctx.solve_rational(B, wl["sigma"], a0, alpha, 1e-10, storage=storage, X=X)
    assert _rel(X.cpu().numpy(), Xd) <= 1e-7
    assert torch.equal(Y, Y2)
    # host buffers in and out
    Yh, _ = ctx.solve_rational(wl["B"], wl["sigma"], a0, alpha, 1e-10, storage=storage)
    assert isinstance(Yh, np.ndarray) and _rel(Yh, want) <= 1e-7


def test_rational_partial_fraction(w1):
    """1/((x+a)(x+b)) = (1/(x+a) - 1/(x+b)) / (b-a)."""
    wl, Ad, Xd, ctx = w1
    a, b = 0.01, 0.5
    Y, st = ctx.solve_rational(torch.from_numpy(wl["B"]).to(DEV), [a, b], 0.0, [1 / (b - a), -1 / (b - a)], 1e-11,
                               storage="fp64")
    I = np.eye(Ad.shape[0])
    Yd = np.linalg.solve((Ad + a * I) @ (Ad + b * I), wl["B"].T).T
    assert _rel(Y.cpu().numpy(), Yd) <= 1e-7


def test_rational_inverse_square_root():
    dims = (2, 2, 2, 2)
    rng = np.random.Generator(np.random.PCG64(41))
    U = synth.su3_links(dims, 0.5, rng)
    kappa = 0.12
    n = 12 * synth.volume(dims)
    B = synth.gaussian_rhs(n, 3, rng)
    Ad = W.dense_A(U, kappa, dims)
    lam, Q = np.linalg.eigh(Ad)
    assert lam.min() > 0
    h = 0.5
    u = np.arange(-30, 31) * h                          # 61 shifts (the library takes up to 64)
    sig, alpha = np.exp(2 * u), (2 * h / np.pi) * np.exp(u)
    r = sum(a / (lam + s_) for a, s_ in zip(alpha, sig))
    bound = np.max(np.abs(r - lam ** -0.5))
    assert bound < 1e-4
    ctx = dsbcg.Context(dims, torch.from_numpy(U).to(DEV), kappa)
    try:
        Y, st = ctx.solve_rational(torch.from_numpy(B).to(DEV), sig, 0.0, alpha, 1e-12, storage="fp64")
        assert st["code"] == 0
        Yd = (Q @ ((lam ** -0.5)[:, None] * (Q.conj().T @ B.T))).T
        Yg = Y.cpu().numpy()
        for i in range(B.shape[0]):
            err = np.linalg.norm(Yg[i] - Yd[i])
            assert err <= bound * np.linalg.norm(B[i]) + 1e-8 * np.linalg.norm(Yd[i]), (i, err)
    finally:
        ctx.close()
