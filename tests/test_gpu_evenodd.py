"""The even-odd (Schur) operator on the GPU against oracle/evenodd.py.

* Dhat, Dhat^H and Ahat = Dhat^H Dhat applied by the library's half-lattice
  stencil (dsbcg_apply on a context with DSBCG_OPERATOR_SCHUR) against the
  oracle's definitions, on 2^4, 2 x 4 x 2 x 4 and 8 x 4 x 4 x 6 lattices, in
  FP64 (to 1e-13) and in the reduced storages;
* DSBlockCG on sigma_j + Ahat (FP64 and FP32 storage) against dense LU of
  the oracle's dense Ahat, with an exactly dependent right-hand side;
* D x = b solved through the odd-site system (sigma = 0 solve of
  Ahat y = Dhat^H c, c = b_o + kappa H_oe b_e) plus the even-site
  reconstruction, against dense LU of the full D;
* a lattice with an odd extent is refused; switching back to the normal
  operator restores full-lattice solves.
"""
import numpy as np
import pytest
import torch

from oracle import evenodd as EO
from oracle import wilson as W
from oracle.dsbcg import dense_solve
from paper_1205_0359_gb300 import dsbcg, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _lattice(dims, seed=91, eps=0.5):
    rng = np.random.Generator(np.random.PCG64(seed))
    U = synth.su3_links(dims, eps, rng)
    return U, rng


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 4), (8, 4, 4, 6)])
@pytest.mark.parametrize("storage,tol", [("fp64", 1e-13), ("df32", 1e-12), ("fp32", 1e-6), ("fp16", 5e-3),
                                         ("bf16", 3e-2)])
def test_schur_operators_match_oracle(dims, storage, tol):
    U, rng = _lattice(dims)
    kappa = 0.13
    nh = 6 * synth.volume(dims)
    h = synth.gaussian_rhs(nh, 3, rng)
    ctx = dsbcg.Context(dims, torch.from_numpy(U).to(DEV), kappa)
    try:
        ctx.set_operator("schur")
        assert ctx.n == nh
        ht = torch.from_numpy(h).to(DEV)
        for op, ref in (("D", EO.Dhat_vec), ("Ddag", EO.Dhat_dag_vec), ("A", EO.Ahat_vec)):
            got = ctx.apply(op, ht, storage=storage).cpu().numpy()
            assert _rel(got, ref(U, kappa, dims, h)) <= tol, (op, storage)
    finally:
        ctx.close()


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_schur_solve_against_dense_lu(dims, storage):
    U, rng = _lattice(dims, seed=92)
    kappa = 0.13
    nh = 6 * synth.volume(dims)
    B = synth.gaussian_rhs(nh, 4, rng)
    B[3] = B[0] + B[1]                          # exactly dependent: deflation at the start
    sigma = np.array([1e-3, 1e-2, 1e-1, 1.0])
    Ah = EO.dense_Ahat(U, kappa, dims)
    Xd = dense_solve(Ah, B, sigma)
    ctx = dsbcg.Context(dims, torch.from_numpy(U).to(DEV), kappa)
    try:
        ctx.set_operator("schur")
        X, st = ctx.solve(torch.from_numpy(B).to(DEV), sigma, 1e-10, storage=storage)
        assert st["code"] == 0 and st["true_relres"].max() <= 1e-10
        assert st["deflations"] >= 1
        err = np.linalg.norm(X.cpu().numpy() - Xd, axis=-1) / np.linalg.norm(Xd, axis=-1)
        assert err.max() <= 1e-7, err.max()
    finally:
        ctx.close()


def test_full_solve_through_schur_system():
    dims = (4, 4, 4, 4)
    U, rng = _lattice(dims, seed=93)
    kappa = 0.12
    n = 12 * synth.volume(dims)
    b = synth.gaussian_rhs(n, 2, rng)
    Dd = W.dense_D(U, kappa, dims)
    want = np.linalg.solve(Dd, b.T).T
    ctx = dsbcg.Context(dims, torch.from_numpy(U).to(DEV), kappa)
    try:
        ctx.set_operator("schur")
        # right-hand side of the odd-site system (oracle half-lattice helpers)
        be, bo = EO.pack(b, dims, EO.EVEN), EO.pack(b, dims, EO.ODD)
        c = bo + kappa * EO.pack(EO.hop_vec(U, kappa, dims, EO.unpack(be, dims, EO.EVEN)), dims, EO.ODD)
        rhs = ctx.apply("Ddag", torch.from_numpy(c).to(DEV), storage="fp64")
        xo, st = ctx.solve(rhs, [0.0], 1e-12, storage="fp32")
        assert st["code"] == 0
        xo = xo[0].cpu().numpy()
        xe = be + kappa * EO.pack(EO.hop_vec(U, kappa, dims, EO.unpack(xo, dims, EO.ODD)), dims, EO.EVEN)
        x = EO.unpack(xe, dims, EO.EVEN) + EO.unpack(xo, dims, EO.ODD)
        assert _rel(x, want) <= 1e-8
    finally:
        ctx.close()


def test_schur_refused_on_odd_extent_and_switch_back():
    dims = (4, 4, 4, 5)
    U, rng = _lattice(dims, seed=94)
    ctx = dsbcg.Context(dims, torch.from_numpy(U).to(DEV), 0.12)
    try:
        with pytest.raises(dsbcg.DSBCGError) as e:
            ctx.set_operator("schur")
        assert e.value.code == -1
    finally:
        ctx.close()
    dims = (4, 4, 4, 4)
    U, rng = _lattice(dims, seed=95)
    kappa = 0.12
    B = synth.gaussian_rhs(12 * synth.volume(dims), 2, rng)
    ctx = dsbcg.Context(dims, torch.from_numpy(U).to(DEV), kappa)
    try:
        X1, _ = ctx.solve(B, [0.1], 1e-10, storage="fp64")
        ctx.set_operator("schur")
        with pytest.raises(dsbcg.DSBCGError) as e:          # the force of the normal operator only
            ctx.force(X1, X1, storage="fp64")
        assert e.value.code == -6
        ctx.set_operator("normal")
        X2, st = ctx.solve(B, [0.1], 1e-10, storage="fp64")
        assert st["code"] == 0 and _rel(X2, X1) <= 1e-9
    finally:
        ctx.close()
