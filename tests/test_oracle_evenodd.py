"""Pins for the even-odd (Schur complement) Wilson operator of the oracle (CPU).

  * H connects only opposite parities: in parity order the diagonal blocks of
    the dense D are exactly the identity,
  * Dhat equals the dense Schur complement D_oo - D_oe D_ee^{-1} D_eo,
  * D x = b solved through the half system plus reconstruction equals the
    dense LU solve, and det D = det Dhat,
  * spectrum: H anticommutes with the parity sign, so its eigenvalues come in
    pairs +-h and Dhat has the eigenvalues 1 - kappa^2 h^2, each pair once
    (any gauge field),
  * gamma_5-hermiticity of Dhat; Ahat hermitian positive semidefinite,
  * the oracle's DSBlockCG on sigma + Ahat against dense LU.
"""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from oracle import evenodd as EO
from oracle import wilson as W
from oracle.dsbcg import dense_solve, dsbcg
from paper_1205_0359_gb300 import synth


@pytest.fixture(scope="module", params=[(2, 2, 2, 2), (2, 4, 2, 4)])
def lat(request):
    dims = request.param
    rng = np.random.Generator(np.random.PCG64(77))
    U = synth.su3_links(dims, 0.5, rng)
    kappa = 0.13
    Dd = W.dense_D(U, kappa, dims)
    e = EO.parity_sites(dims, EO.EVEN)
    o = EO.parity_sites(dims, EO.ODD)
    ie = (12 * e[:, None] + np.arange(12)).reshape(-1)
    io = (12 * o[:, None] + np.arange(12)).reshape(-1)
    return dims, U, kappa, Dd, ie, io


def test_parity_blocks_are_identity(lat):
    dims, U, kappa, Dd, ie, io = lat
    nh = ie.size
    assert np.max(np.abs(Dd[np.ix_(ie, ie)] - np.eye(nh))) == 0.0
    assert np.max(np.abs(Dd[np.ix_(io, io)] - np.eye(nh))) == 0.0
    assert np.max(np.abs(Dd[np.ix_(ie, io)])) > 0.01


def test_dense_schur_complement(lat):
    dims, U, kappa, Dd, ie, io = lat
    Dee, Deo = Dd[np.ix_(ie, ie)], Dd[np.ix_(ie, io)]
    Doe, Doo = Dd[np.ix_(io, ie)], Dd[np.ix_(io, io)]
    S = Doo - Doe @ np.linalg.solve(Dee, Deo)
    Dh = EO.dense_Dhat(U, kappa, dims)
    assert np.max(np.abs(Dh - S)) < 1e-13


def test_schur_solve_and_determinant(lat):
    dims, U, kappa, Dd, ie, io = lat
    Dh = EO.dense_Dhat(U, kappa, dims)
    rng = np.random.Generator(np.random.PCG64(5))
    b = synth.gaussian_rhs(Dd.shape[0], 1, rng)[0]
    x = EO.schur_solve_D(U, kappa, dims, b, lambda c: np.linalg.solve(Dh, c))
    xd = np.linalg.solve(Dd, b)
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)
    s1, l1 = np.linalg.slogdet(Dd)
    s2, l2 = np.linalg.slogdet(Dh)
    assert abs(l1 - l2) < 1e-10 and abs(s1 - s2) < 1e-10


def test_spectrum_from_hopping_pairs(lat):
    dims, U, kappa, Dd, ie, io = lat
    H = (np.eye(Dd.shape[0]) - Dd) / kappa
    h = np.linalg.eigvals(H)
    # +-h pairs: the spectrum of H is symmetric
    cost = np.abs(h[:, None] + h[None, :])
    r, c = linear_sum_assignment(cost)
    assert cost[r, c].max() < 1e-9
    want = 1.0 - kappa ** 2 * h ** 2                   # every value twice
    got = np.linalg.eigvals(EO.dense_Dhat(U, kappa, dims))
    got2 = np.concatenate([got, got])
    cost = np.abs(want[:, None] - got2[None, :])
    r, c = linear_sum_assignment(cost)
    assert cost[r, c].max() < 1e-9


def test_gamma5_hermiticity_and_Ahat(lat):
    dims, U, kappa, Dd, ie, io = lat
    Dh = EO.dense_Dhat(U, kappa, dims)
    nh = Dh.shape[0]
    g5 = np.kron(np.eye(nh // 12), np.kron(W.G5, np.eye(3)))
    assert np.max(np.abs(g5 @ Dh @ g5 - Dh.conj().T)) < 1e-13
    Ah = EO.dense_Ahat(U, kappa, dims)
    assert np.max(np.abs(Ah - Ah.conj().T)) < 1e-13
    assert np.linalg.eigvalsh(Ah).min() > -1e-12
    rng = np.random.Generator(np.random.PCG64(9))
    v = synth.gaussian_rhs(nh, 2, rng)
    assert np.max(np.abs(EO.Ahat_vec(U, kappa, dims, v) - v @ Ah.T)) < 1e-12


def test_odd_extent_rejected():
    with pytest.raises(ValueError):
        EO.parity_sites((2, 3, 2, 2), EO.ODD)


def test_pack_unpack_roundtrip():
    dims = (2, 4, 2, 2)
    rng = np.random.Generator(np.random.PCG64(3))
    v = synth.gaussian_rhs(12 * 32, 2, rng)
    back = EO.unpack(EO.pack(v, dims, EO.EVEN), dims, EO.EVEN) + \
        EO.unpack(EO.pack(v, dims, EO.ODD), dims, EO.ODD)
    assert np.array_equal(back, v)


def test_dsbcg_on_schur_operator():
    """The solver is operator-agnostic: sigma_j + Ahat solved with one run."""
    dims = (4, 2, 2, 4)
    rng = np.random.Generator(np.random.PCG64(11))
    U = synth.su3_links(dims, 0.4, rng)
    kappa = 0.12
    nh = 6 * synth.volume(dims)
    B = synth.gaussian_rhs(nh, 3, rng)
    sigma = synth.log_shifts(1e-3, 1.0, 3)
    X, info = dsbcg(lambda v: EO.Ahat_vec(U, kappa, dims, v), B, sigma, tol=1e-12)
    assert info["converged"]
    Xd = dense_solve(EO.dense_Ahat(U, kappa, dims), B, sigma)
    err = np.linalg.norm(X - Xd, axis=2) / np.linalg.norm(Xd, axis=2)
    assert err.max() < 1e-9
