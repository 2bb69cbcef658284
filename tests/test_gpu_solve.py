"""GPU DSBlockCG parity against the FP64 oracle, through the C ABI.

* 4^4 workload (b_4 = b_1 + b_2): FP64 and mixed precisions (double-float
  or FP64 reliable updates) against dense LU (relative error <= 1e-7 per
  (rhs, shift)), exact deflation, x_4 = x_1 + x_2;
* fixed number of block steps: the GPU iterate equals the block Galerkin
  iterate of Eq. 3.2 computed by the oracle's definition;
* special cases m = s = 1 (CG), sigma = 0, a ragged lattice whose volume is
  not a multiple of the CTA tiles, compared with the oracle's band-Lanczos
  solver;
* error paths: negative shift, NaN input, iteration cap;
* the 16^3 x 32, m = s = 12 workload in the configuration bench.py times:
  every true residual reported by the library <= tol, and the residual of
  every one of the 144 (rhs, shift) systems recomputed with the oracle's own
  FP64 Wilson operator <= 10 tol and equal to the library's residual (FP64,
  or double-float on request) within tol / 100.
"""
import numpy as np
import pytest
import torch

from oracle import wilson as W
from oracle.dsbcg import dense_solve, dsbcg as oracle_dsbcg, galerkin_iterate
from oracle_check import relres_all
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


def _relerr(X, Xd):
    return np.linalg.norm(X - Xd, axis=-1) / np.linalg.norm(Xd, axis=-1)


@pytest.mark.parametrize("storage,tol,bound,fp64res", [("fp64", 1e-10, 1e-7, False), ("fp32", 1e-10, 1e-7, False),
                                                       ("fp32", 1e-10, 1e-7, True), ("fp16", 1e-10, 1e-7, False),
                                                       ("bf16", 1e-8, 1e-5, False)])
def test_w1_against_dense_lu(w1, storage, tol, bound, fp64res):
    wl, Ad, Xd, ctx = w1
    B = torch.from_numpy(wl["B"]).to(DEV)
    X, st = ctx.solve(B, wl["sigma"], tol, storage=storage, fp64_residuals=fp64res)
    Xg = X.cpu().numpy()
    assert st["code"] == 0, st
    assert st["true_relres"].max() <= tol
    assert _relerr(Xg, Xd).max() <= bound
    assert st["deflations"] >= 1
    dep = np.linalg.norm(Xg[:, 3] - Xg[:, 0] - Xg[:, 1], axis=1) / np.linalg.norm(Xg[:, 3], axis=1)
    assert dep.max() <= 10 * bound


@pytest.mark.parametrize("k", [1, 2, 3])
def test_fixed_k_galerkin_iterate(k):
    dims = (2, 2, 2, 2)
    rng = np.random.Generator(np.random.PCG64(31))
    U = synth.su3_links(dims, 0.5, rng)
    kappa = 0.12
    n = 12 * synth.volume(dims)
    B = synth.gaussian_rhs(n, 3, rng)
    sigma = synth.log_shifts(1e-3, 1.0, 4)
    Ad = W.dense_A(U, kappa, dims)
    ctx = dsbcg.Context(dims, U, kappa)
    X, st = ctx.solve(B, sigma, 0.0, storage="fp64", max_block_steps=k, refine=False, freeze=False,
                      poll_every=1, raise_on_error=False)
    assert st["code"] == 1 and st["block_steps"] == k
    Xg = galerkin_iterate(Ad, B, sigma, k)
    assert _relerr(X, Xg).max() < 1e-9
    ctx.close()


def test_fixed_k_with_deflation(w1):
    wl, Ad, Xd, ctx = w1
    X, st = ctx.solve(wl["B"], wl["sigma"], 0.0, storage="fp64", max_block_steps=2, refine=False,
                      freeze=False, poll_every=1, raise_on_error=False)
    assert st["deflations"] == 1 and st["final_rank"] == 3
    Xg = galerkin_iterate(Ad, wl["B"], wl["sigma"], 2)
    assert _relerr(X, Xg).max() < 1e-9


def test_cg_special_case_and_zero_shift(w1):
    wl, Ad, Xd, ctx = w1
    b = wl["B"][:1]
    for storage in ("fp64", "fp32"):
        X, st = ctx.solve(b, [0.0], 1e-10, storage=storage)
        want = dense_solve(Ad, b, [0.0])
        assert st["code"] == 0 and _relerr(X, want).max() < 1e-7


def test_ragged_lattice_against_oracle_solver():
    dims = (6, 4, 4, 5)                         # 480 sites: 15 CTA tiles of 32
    rng = np.random.Generator(np.random.PCG64(77))
    U = synth.su3_links(dims, 0.5, rng)
    kappa = 0.12
    n = 12 * synth.volume(dims)
    B = synth.gaussian_rhs(n, 5, rng)
    sigma = synth.log_shifts(1e-2, 1.0, 3)
    Aop = lambda v: W.A_vec(U, kappa, dims, v)
    Xo, info = oracle_dsbcg(Aop, B, sigma, tol=1e-12)
    assert info["converged"]
    ctx = dsbcg.Context(dims, torch.from_numpy(U).to(DEV), kappa)
    for storage in ("fp64", "fp32"):
        X, st = ctx.solve(torch.from_numpy(B).to(DEV), sigma, 1e-11, storage=storage)
        assert st["code"] == 0
        assert _relerr(X.cpu().numpy(), Xo).max() < 1e-7
    ctx.close()


def test_error_paths(w1):
    wl, Ad, Xd, ctx = w1
    B = wl["B"]
    with pytest.raises(dsbcg.DSBCGError) as e:
        ctx.solve(B, [0.1, -1.0], 1e-8)
    assert e.value.code == -1
    Bn = B.copy()
    Bn[1, 5] = np.nan
    with pytest.raises(dsbcg.DSBCGError) as e:
        ctx.solve(Bn, [0.1], 1e-8)
    assert e.value.code == -5
    X, st = ctx.solve(B, wl["sigma"], 1e-10, storage="fp64", max_block_steps=3, refine=False,
                      raise_on_error=False)
    assert st["code"] == 1 and st["status"] == "NOT_CONVERGED"
    assert np.all(np.isfinite(X)) and st["true_relres"].max() > 1e-10
    # the library still works after a capped solve
    X, st = ctx.solve(B, wl["sigma"], 1e-10, storage="fp64")
    assert st["code"] == 0


def test_host_buffers_roundtrip(w1):
    wl, Ad, Xd, ctx = w1
    X, st = ctx.solve(wl["B"], wl["sigma"], 1e-10, storage="fp32")   # numpy in/out
    assert isinstance(X, np.ndarray) and st["code"] == 0
    assert _relerr(X, Xd).max() < 1e-7


@pytest.fixture(scope="module")
def w2():
    wl = synth.make_workload("w2_16x16x16x32")
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(DEV), wl["kappa"])
    yield wl, ctx
    ctx.close()


@pytest.mark.parametrize("fp64res", [False, True])
def test_w2_full_size_mixed(w2, fp64res):
    wl, ctx = w2
    B = torch.from_numpy(wl["B"]).to(DEV)
    X, st = ctx.solve(B, wl["sigma"], wl["tol"], storage="fp32", fp64_residuals=fp64res)
    assert st["code"] == 0, st
    assert st["true_relres"].max() <= wl["tol"]
    # every (rhs, shift) system, recomputed with the oracle's operator
    rel = relres_all(wl, X)
    assert not np.isnan(rel).any()
    bad = np.argwhere(rel > 10 * wl["tol"])
    assert bad.size == 0, (bad, rel.max())
    # the library's true residual (FP64, or double-float on request) agrees
    # with the oracle's FP64 recomputation far below tol, for every pair
    diff = np.abs(rel - st["true_relres"])
    assert diff.max() <= 1e-2 * wl["tol"], (np.unravel_index(diff.argmax(), diff.shape), diff.max())


def test_concurrent_restarts_match_serial(w1):
    """The per-shift restarts run concurrently on separate streams, each
    shift handed off as soon as the joint solve freezes it (its residuals
    and restarts then overlap the joint solve of the other shifts); with the
    library's profiling on everything runs one step after another.  Each
    restart only touches its own lane's buffers and a frozen shift's inner
    iterate no longer changes, so X is bitwise the same either way."""
    wl, Ad, Xd, ctx = w1
    B = torch.from_numpy(wl["B"]).to(DEV)
    Xc, stc = ctx.solve(B, wl["sigma"], 1e-10, storage="fp32")
    ctx.set_profiling(True)
    Xs, sts = ctx.solve(B, wl["sigma"], 1e-10, storage="fp32")
    ctx.set_profiling(False)
    assert stc["code"] == 0 and sts["code"] == 0
    assert stc["restarts"] == sts["restarts"] >= len(wl["sigma"])
    assert stc["block_steps"] == sts["block_steps"]
    assert torch.equal(Xc, Xs)
    assert np.array_equal(stc["true_relres"], sts["true_relres"])


def test_paper_comparison_special_cases():
    """The paper's comparison (Sec. 4, Table 1) as special cases of the same
    solver, on a small lattice: every system of every algorithm meets tol,
    DSBlockCG needs the fewest A applications and plain CG the most."""
    import bench
    res = bench.run_comparison(DEV, torch.cuda.current_stream(), name="cmp_16x16x16x16", dims=(8, 8, 8, 8),
                               m=3, s=4)["algorithms"]
    for alg, r in res.items():
        assert r["max_true_relres"] <= 1e-8, (alg, r)
    mv = {alg: r["mvms"] for alg, r in res.items()}
    assert mv["DSBlockCG"] == min(mv.values()), mv
    assert mv["CG"] == max(mv.values()), mv


@pytest.mark.parametrize("m", [20, 32])
@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_wide_block_against_dense_lu(storage, m):
    """m = 20 and 32 right-hand sides (the largest block): widths above 16
    take the untiled Gram kernel, and from 28 on the initial QR needs more
    than 48 KB of shared memory; solutions against dense LU on 4^4."""
    dims = (4, 4, 4, 4)
    rng = np.random.Generator(np.random.PCG64(77))
    U = synth.su3_links(dims, 0.3, rng)
    kappa = 0.12
    n = 12 * synth.volume(dims)
    B = synth.gaussian_rhs(n, m, rng)
    sigma = np.array([1e-2, 1.0])
    Ad = W.dense_A(U, kappa, dims)
    Xd = dense_solve(Ad, B, sigma)
    ctx = dsbcg.Context(dims, torch.from_numpy(U).to(DEV), kappa)
    try:
        X, st = ctx.solve(torch.from_numpy(B).to(DEV), sigma, 1e-10, storage=storage)
        assert st["code"] == 0, st["status"]
        assert st["true_relres"].max() <= 1e-10
        assert _relerr(X.cpu().numpy(), Xd).max() <= 1e-7
    finally:
        ctx.close()


def test_resume_from_initial_guess(w1):
    """dsbcg_params.x0: a solve resumed from X_0.  From the exact solution no
    block step is needed; a loose solve resumed at a tight tolerance reaches
    it and agrees with dense LU."""
    wl, Ad, Xd, ctx = w1
    B = torch.from_numpy(wl["B"]).to(DEV)
    X, st = ctx.solve(B, wl["sigma"], 1e-10, storage="fp32", x0=torch.from_numpy(Xd).to(DEV))
    assert st["code"] == 0 and st["block_steps"] == 0 and st["restarts"] == 0
    assert _relerr(X.cpu().numpy(), Xd).max() <= 1e-12
    X1, st1 = ctx.solve(B, wl["sigma"], 1e-5, storage="fp32", refine=False, raise_on_error=False)
    X2, st2 = ctx.solve(B, wl["sigma"], 1e-10, storage="fp32", x0=X1)
    assert st2["code"] == 0 and st2["true_relres"].max() <= 1e-10
    assert _relerr(X2.cpu().numpy(), Xd).max() <= 1e-7


def test_restart_cap_reports_not_converged(w1):
    """FP32 storage cannot reach 1e-10 without restarts: with max_restarts = 0
    the solve reports NOT_CONVERGED and still returns finite iterates."""
    wl, Ad, Xd, ctx = w1
    X, st = ctx.solve(torch.from_numpy(wl["B"]).to(DEV), wl["sigma"], 1e-10, storage="fp32", max_restarts=0,
                      raise_on_error=False)
    assert st["code"] == 1 and st["restarts"] == 0
    assert st["true_relres"].max() > 1e-10
    assert bool(torch.isfinite(X).all())
