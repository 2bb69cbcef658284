"""Pins for the oracle's DSBlockCG (CPU only).

The oracle's recurrences are checked against
  * dense LU solves of every (sigma_j I + A) x = b (Eq. 1.1) on 2^4 and 4^4,
  * the Galerkin definition X = V (V^H (sigma+A) V)^{-1} V^H B over the block
    Krylov subspace (Eqs. 2.1, 2.2, 3.2), with a basis built by fully
    orthogonalised block Arnoldi, at a fixed number of block steps,
  * textbook CG iterates for m = s = 1, CG per shift for m = 1 (shifted
    CG), and block CG iterates for s = 1,
  * exact deflation when b_4 = b_1 + b_2 (Sec. 3: the deflated subspace has
    smaller dimension and the bandwidth of T drops),
  * the structural statements of Sec. 3: orthonormal V, hermitian banded T
    with semi-bandwidth m, T = V^H A V, B = V rho,
  * the residual statement of Sec. 3: R is orthogonal to the Lanczos vectors
    built so far, and the column norms of C in R = W C (computed from T's
    factors, no product with A) equal the explicit ||b_i - (sigma_j+A) x_ij||,
    at vector counts inside a block and after a deflation; for m = 1 they are
    the textbook CG residual norms,
  * the rational combination alpha_0 B + sum_j alpha_j X_j (Sec. 1) against
    r(A) B through A's eigendecomposition, a closed partial fraction, and a
    quadrature approximation of A^{-1/2} within its spectral error bound.
"""
import numpy as np
import pytest

from oracle import wilson as W
from oracle.dsbcg import (NotHPD, dense_solve, dsbcg, galerkin_iterate, rational_combination,
                          true_relres)
from paper_1205_0359_gb300 import synth


def _problem(dims, m, s, seed, eps=0.4, kappa=0.12, dependent=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    U = synth.su3_links(dims, eps, rng)
    n = 12 * synth.volume(dims)
    B = synth.gaussian_rhs(n, m, rng)
    if dependent:
        B[m - 1] = B[0] + B[1]
    sigma = synth.log_shifts(1e-3, 1.0, s)
    Aop = lambda v: W.A_vec(U, kappa, dims, v)
    return U, kappa, B, sigma, Aop


@pytest.fixture(scope="module")
def small():
    dims = (2, 2, 2, 2)
    U, kappa, B, sigma, Aop = _problem(dims, 3, 4, 21)
    Ad = W.dense_A(U, kappa, dims)
    return dims, Ad, B, sigma, Aop


@pytest.fixture(scope="module")
def w1():
    wl = synth.make_workload("w1_4x4x4x4")
    dims, U, k = wl["dims"], wl["U"], wl["kappa"]
    Ad = W.dense_A(U, k, dims)
    Aop = lambda v: W.A_vec(U, k, dims, v)
    return wl, Ad, Aop


def test_dense_lu_2x2x2x2(small):
    dims, Ad, B, sigma, Aop = small
    X, info = dsbcg(Aop, B, sigma, tol=1e-13)
    Xd = dense_solve(Ad, B, sigma)
    err = np.linalg.norm(X - Xd, axis=2) / np.linalg.norm(Xd, axis=2)
    assert info["converged"]
    assert err.max() < 1e-10


def test_dense_lu_4x4x4x4_workload(w1):
    wl, Ad, Aop = w1
    B, sigma = wl["B"], wl["sigma"]
    X, info = dsbcg(Aop, B, sigma, tol=1e-12)
    Xd = dense_solve(Ad, B, sigma)
    err = np.linalg.norm(X - Xd, axis=2) / np.linalg.norm(Xd, axis=2)
    assert info["converged"]
    assert info["deflations"] >= 1
    assert err.max() < 1e-9
    rr = true_relres(Aop, B, sigma, X)
    assert rr.max() <= 1e-12


@pytest.mark.parametrize("nblocks", [1, 2, 3])
def test_galerkin_definition_fixed_k(small, nblocks):
    dims, Ad, B, sigma, Aop = small
    m = B.shape[0]
    X, info = dsbcg(Aop, B, sigma, tol=0.0, freeze=False, stop_after_vectors=m * nblocks)
    assert info["nvec"] == m * nblocks
    Xg = galerkin_iterate(Ad, B, sigma, nblocks)
    err = np.linalg.norm(X - Xg, axis=2) / np.linalg.norm(Xg, axis=2)
    assert err.max() < 1e-9


def test_galerkin_definition_with_deflation(w1):
    wl, Ad, Aop = w1
    B, sigma = wl["B"], wl["sigma"]
    # b_4 = b_1 + b_2: the block Krylov space has dimension 3 per block
    for nblocks in (1, 2):
        X, info = dsbcg(Aop, B, sigma, tol=0.0, freeze=False, stop_after_vectors=3 * nblocks)
        if nblocks > 1:          # b_4 is examined once v_1..v_3 exist
            assert info["deflations"] == 1 and info["deflated_at"] == [3]
        Xg = galerkin_iterate(Ad, B, sigma, nblocks)
        err = np.linalg.norm(X - Xg, axis=2) / np.linalg.norm(Xg, axis=2)
        assert err.max() < 1e-9


def test_textbook_cg_m1_s1(small):
    """m = s = 1: the iterates are those of plain CG on (sigma + A) x = b."""
    dims, Ad, B, sigma, Aop = small
    b = B[0]
    sg = sigma[1]
    M = Ad + sg * np.eye(Ad.shape[0])
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    for k in range(1, 9):
        Mp = M @ p
        a = np.vdot(r, r).real / np.vdot(p, Mp).real
        x = x + a * p
        rn = r - a * Mp
        beta = np.vdot(rn, rn).real / np.vdot(r, r).real
        p = rn + beta * p
        r = rn
        Xo, _ = dsbcg(Aop, b[None], [sg], tol=0.0, freeze=False, stop_after_vectors=k)
        assert np.linalg.norm(Xo[0, 0] - x) <= 1e-10 * np.linalg.norm(x)


def test_exact_deflation_solution(w1):
    wl, Ad, Aop = w1
    B, sigma = wl["B"], wl["sigma"]
    X, info = dsbcg(Aop, B, sigma, tol=1e-13, freeze=False)
    assert info["deflated_at"][0] == 3
    diff = np.linalg.norm(X[:, 3] - X[:, 0] - X[:, 1], axis=1) / np.linalg.norm(X[:, 3], axis=1)
    assert diff.max() < 1e-11


def test_lanczos_structure(small):
    dims, Ad, B, sigma, Aop = small
    m = B.shape[0]
    X, info = dsbcg(Aop, B, sigma, tol=0.0, freeze=False, stop_after_vectors=5 * m,
                    keep_basis=True)
    V, T, rho = info["V"], info["T"], info["rho"]
    k = V.shape[0]
    assert np.max(np.abs(V.conj() @ V.T - np.eye(k))) < 1e-10
    assert np.max(np.abs(T - T.conj().T)) == 0.0
    i, j = np.nonzero(np.abs(T) > 0)
    assert np.max(np.abs(i - j)) <= m                 # semi-bandwidth m (Sec. 3)
    TA = V.conj() @ Ad @ V.T                           # V^H A V
    assert np.max(np.abs(T - TA)) < 1e-10
    assert np.max(np.abs(V.T @ rho - B.T)) < 1e-12    # B = V rho
    assert np.max(np.abs(np.tril(rho, -1)[m:])) == 0.0


def test_shifted_systems_share_one_lanczos_run(small):
    """One multi-shift run equals separate single-shift runs (Sec. 3, last paragraph)."""
    dims, Ad, B, sigma, Aop = small
    X, _ = dsbcg(Aop, B, sigma, tol=0.0, freeze=False, stop_after_vectors=12)
    for j, sg in enumerate(sigma):
        Xj, _ = dsbcg(Aop, B, [sg], tol=0.0, freeze=False, stop_after_vectors=12)
        assert np.max(np.abs(X[j] - Xj[0])) < 1e-12 * np.max(np.abs(Xj))


def test_not_hpd_is_reported(small):
    dims, Ad, B, sigma, Aop = small
    with pytest.raises(NotHPD):
        dsbcg(Aop, B, [-10.0], tol=1e-10)


@pytest.mark.parametrize("k", [1, 2, 4, 7, 11, 16])
def test_residual_estimate_matches_explicit(small, k):
    """||C[:, i]|| = ||r_i|| (Sec. 3), also when k is not a multiple of m."""
    dims, Ad, B, sigma, Aop = small
    X, info = dsbcg(Aop, B, sigma, tol=0.0, freeze=False, stop_after_vectors=k, estimate=True)
    rr = true_relres(Aop, B, sigma, X)
    assert rr.min() > 1e-4                            # not yet converged: a real test
    assert np.max(np.abs(info["est_relres"] - rr)) <= 1e-11 * rr.max()


def test_residual_estimate_with_deflation(w1):
    """After b_4 = b_1 + b_2 is dropped, W has fewer columns (Sec. 3)."""
    wl, Ad, Aop = w1
    B, sigma = wl["B"], wl["sigma"]
    for k in (5, 9, 14):
        X, info = dsbcg(Aop, B, sigma, tol=0.0, freeze=False, stop_after_vectors=k, estimate=True)
        assert info["deflations"] == 1
        rr = true_relres(Aop, B, sigma, X)
        assert np.max(np.abs(info["est_relres"] - rr)) <= 1e-11 * rr.max()


def test_residual_orthogonal_to_lanczos_vectors(small):
    """Galerkin condition V^H (B - (sigma+A) X) = 0 at every vector count."""
    dims, Ad, B, sigma, Aop = small
    for k in (2, 5, 10):
        X, info = dsbcg(Aop, B, sigma, tol=0.0, freeze=False, stop_after_vectors=k, keep_basis=True)
        V = info["V"]
        for j, sg in enumerate(sigma):
            R = B - sg * X[j] - Aop(X[j])
            proj = V.conj() @ R.T
            assert np.max(np.abs(proj)) <= 1e-11 * np.max(np.abs(R)), (k, j)


def test_residual_estimate_m1_is_cg_residual(small):
    """m = s = 1: the estimate is ||r_k|| of textbook CG on (sigma + A) x = b."""
    dims, Ad, B, sigma, Aop = small
    b = B[0]
    sg = sigma[2]
    M = Ad + sg * np.eye(Ad.shape[0])
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    for k in range(1, 8):
        Mp = M @ p
        a = np.vdot(r, r).real / np.vdot(p, Mp).real
        x = x + a * p
        rn = r - a * Mp
        p = rn + (np.vdot(rn, rn).real / np.vdot(r, r).real) * p
        r = rn
        _, info = dsbcg(Aop, b[None], [sg], tol=0.0, freeze=False, stop_after_vectors=k, estimate=True)
        want = np.linalg.norm(r) / np.linalg.norm(b)
        assert abs(info["est_relres"][0, 0] - want) <= 1e-10 * want, k


def _cg_iterates(M, b, steps):
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    out = []
    for _ in range(steps):
        Mp = M @ p
        a = np.vdot(r, r).real / np.vdot(p, Mp).real
        x = x + a * p
        rn = r - a * Mp
        p = rn + (np.vdot(rn, rn).real / np.vdot(r, r).real) * p
        r = rn
        out.append(x.copy())
    return out


def test_m1_is_shifted_cg(small):
    """m = 1, s = 4: every shift follows its own textbook CG iterates (the
    shifted CG of Sec. 1), from one Lanczos run."""
    dims, Ad, B, sigma, Aop = small
    b = B[1]
    I = np.eye(Ad.shape[0])
    ref = [_cg_iterates(Ad + sg * I, b, 9) for sg in sigma]
    for k in (1, 4, 9):
        X, _ = dsbcg(Aop, b[None], sigma, tol=0.0, freeze=False, stop_after_vectors=k)
        for j in range(len(sigma)):
            x = ref[j][k - 1]
            assert np.linalg.norm(X[j, 0] - x) <= 1e-10 * np.linalg.norm(x), (k, j)


def test_s1_is_block_cg(small):
    """s = 1: the iterates of O'Leary's block CG at every block step (no
    dependent right-hand sides here, so no deflation)."""
    dims, Ad, B, sigma, Aop = small
    sg = sigma[1]
    M = Ad + sg * np.eye(Ad.shape[0])
    m = B.shape[0]
    Xb = np.zeros((Ad.shape[0], m), dtype=np.complex128)
    R = B.T.copy()
    P = R.copy()
    for k in range(1, 6):
        MP = M @ P
        alpha = np.linalg.solve(P.conj().T @ MP, R.conj().T @ R)
        Xb = Xb + P @ alpha
        Rn = R - MP @ alpha
        beta = np.linalg.solve(R.conj().T @ R, Rn.conj().T @ Rn)
        P = Rn + P @ beta
        R = Rn
        X, info = dsbcg(Aop, B, [sg], tol=0.0, freeze=False, stop_after_vectors=m * k)
        assert info["deflations"] == 0
        err = np.linalg.norm(X[0] - Xb.T, axis=1) / np.linalg.norm(Xb.T, axis=1)
        assert err.max() <= 1e-9, (k, err.max())


def test_rational_combination_is_r_of_A(small):
    """alpha_0 B + sum_j alpha_j X_j = Q r(Lambda) Q^H B (Sec. 1), with the
    iterates of one DSBlockCG run and r evaluated on A's eigenvalues."""
    dims, Ad, B, sigma, Aop = small
    X, info = dsbcg(Aop, B, sigma, tol=1e-13)
    assert info["converged"]
    alpha0, alpha = 0.3, np.array([0.7, -0.2, 1.5, 0.05])
    Y = rational_combination(B, X, alpha0, alpha)
    lam, Q = np.linalg.eigh(Ad)
    r = alpha0 + sum(a / (lam + sg) for a, sg in zip(alpha, sigma))
    Yd = (Q @ (r[:, None] * (Q.conj().T @ B.T))).T
    assert np.linalg.norm(Y - Yd) <= 1e-10 * np.linalg.norm(Yd)


def test_rational_combination_partial_fraction(small):
    """1/((x+a)(x+b)) = (1/(x+a) - 1/(x+b)) / (b-a): the combination equals a
    solve with the product (A+a)(A+b)."""
    dims, Ad, B, sigma, Aop = small
    a, b = 0.01, 0.5
    X, _ = dsbcg(Aop, B, [a, b], tol=1e-13)
    Y = rational_combination(B, X, 0.0, [1.0 / (b - a), -1.0 / (b - a)])
    I = np.eye(Ad.shape[0])
    Yd = np.linalg.solve((Ad + a * I) @ (Ad + b * I), B.T).T
    assert np.linalg.norm(Y - Yd) <= 1e-9 * np.linalg.norm(Yd)


def test_rational_inverse_square_root(small):
    """nu = -1/2: the substitution t = e^u in x^{-1/2} = (2/pi) int_0^inf
    dt / (t^2 + x) and the trapezoidal rule give shifts sigma_k = e^{2 u_k}
    and weights alpha_k = (2 h / pi) e^{u_k}.  A is hermitian, so
    ||r(A) b - A^{-1/2} b|| <= max over A's eigenvalues |r - lambda^{-1/2}|
    times ||b||."""
    dims, Ad, B, sigma, Aop = small
    lam, Q = np.linalg.eigh(Ad)
    assert lam.min() > 0
    h = 0.35
    u = np.arange(-40, 41) * h
    sig, alpha = np.exp(2 * u), (2 * h / np.pi) * np.exp(u)
    X, info = dsbcg(Aop, B, sig, tol=1e-13)
    assert info["converged"]
    Y = rational_combination(B, X, 0.0, alpha)
    r = sum(a / (lam + s_) for a, s_ in zip(alpha, sig))
    bound = np.max(np.abs(r - lam ** -0.5))
    assert bound < 1e-5                                # the rule is accurate here
    Yd = (Q @ ((lam ** -0.5)[:, None] * (Q.conj().T @ B.T))).T
    for i in range(B.shape[0]):
        err = np.linalg.norm(Y[i] - Yd[i])
        assert err <= bound * np.linalg.norm(B[i]) + 1e-9 * np.linalg.norm(Yd[i]), i


def test_frozen_systems_are_not_updated(small):
    """Freezing (Sec. 4): once (i, j) meets tol it is no longer updated, so its
    final iterate is the iterate after the vector count at which it froze."""
    dims, Ad, B, sigma, Aop = small
    m = B.shape[0]
    tol = 1e-8
    X, info = dsbcg(Aop, B, sigma, tol=tol, check_every=m)
    assert info["converged"]
    fa = info["frozen_at"]
    assert np.all(fa > 0)
    assert len(np.unique(fa)) > 1                      # systems freeze at different times
    assert fa[-1].max() <= fa[0].min()                 # the largest shift converges first
    for k in np.unique(fa):
        Xk, _ = dsbcg(Aop, B, sigma, tol=0.0, freeze=False, stop_after_vectors=int(k))
        for j, i in zip(*np.nonzero(fa == k)):
            assert np.array_equal(X[j, i], Xk[j, i]), (j, i, k)
    rr = true_relres(Aop, B, sigma, X)
    assert rr.max() <= tol


def test_frozen_at_survives_a_capped_solve(small):
    """With a vector cap the smallest shift does not converge; the final
    residual pass must keep the freeze points of the systems frozen earlier."""
    dims, Ad, B, sigma, Aop = small
    m = B.shape[0]
    tol = 1e-8
    _, full = dsbcg(Aop, B, sigma, tol=tol, check_every=m)
    cap = int(full["frozen_at"][0].min()) - m       # before the smallest shift meets tol
    X, info = dsbcg(Aop, B, sigma, tol=tol, check_every=m, max_vectors=cap)
    assert not info["converged"] and info["nvec"] == cap
    fa = info["frozen_at"]
    early = fa[-1] > 0
    assert early.all() and fa[-1].max() < cap        # the largest shift froze before the cap
    assert np.array_equal(fa[-1], full["frozen_at"][-1])
    assert np.all(fa[0] < 0)


def test_zero_right_hand_side_is_deflated(small):
    """b_2 = 0: the zero candidate is dropped when it comes up, right after
    v_1 is built from b_1 (Sec. 3 deflation); x_2j = 0 exactly, and the other
    systems are solved as without it."""
    dims, Ad, B, sigma, Aop = small
    Bz = B.copy()
    Bz[1] = 0.0
    X, info = dsbcg(Aop, Bz, sigma, tol=1e-12)
    assert info["converged"] and info["deflations"] >= 1 and info["deflated_at"][0] == 1
    assert np.all(X[:, 1] == 0)
    Xd = dense_solve(Ad, Bz[[0, 2]], sigma)
    err = np.linalg.norm(X[:, [0, 2]] - Xd, axis=2) / np.linalg.norm(Xd, axis=2)
    assert err.max() < 1e-10


def test_all_zero_B(small):
    """B = 0: no Lanczos vector is built and X = 0 is the exact solution."""
    dims, Ad, B, sigma, Aop = small
    X, info = dsbcg(Aop, np.zeros_like(B), sigma, tol=1e-12)
    assert info["nvec"] == 0 and info["converged"] and info["deflations"] == B.shape[0]
    assert np.all(X == 0)
