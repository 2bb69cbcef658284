"""Pins for the oracle's gradients (CPU only): central finite differences.

Loss L = sum_j alpha_j sum_i Re(b_i^H x_ij) with x_ij = (sigma_j + A)^{-1} b_i,
the RHMC-style loss of the gradient workload.  Directional derivatives of L
along random directions in B, sigma and the (unconstrained, complex) links
are compared with the oracle's analytic gradients.  The loss is evaluated
with dense LU on 2^4 and with the oracle solver at tol 1e-13 on 4^4.
"""
import numpy as np
import pytest

from oracle import wilson as W
from oracle.dsbcg import dense_solve, dsbcg
from oracle.force import link_gradient, rhmc_gradients, rhmc_loss
from paper_1205_0359_gb300 import synth


def _loss_dense(U, kappa, dims, B, sigma, alpha):
    Ad = W.dense_A(U, kappa, dims)
    X = dense_solve(Ad, B, sigma)
    return rhmc_loss(B, X, alpha), X


def _cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _re_inner(g, d):
    return float(np.sum(np.real(np.conj(g) * d)))


def test_fd_gradients_2x2x2x2():
    dims = (2, 2, 2, 2)
    rng = np.random.Generator(np.random.PCG64(404))
    U = synth.su3_links(dims, 0.5, rng)
    kappa = 0.12
    n = 12 * synth.volume(dims)
    B = synth.gaussian_rhs(n, 2, rng)
    sigma = np.array([1e-2, 1e-1, 1.0])
    alpha = np.array([0.2, 0.3, 0.5])
    L0, X = _loss_dense(U, kappa, dims, B, sigma, alpha)
    gB, gs, gU = rhmc_gradients(U, kappa, dims, B, sigma, alpha, X)
    h = 1e-6
    for _ in range(6):
        dB = _cplx(rng, B.shape)
        fd = (_loss_dense(U, kappa, dims, B + h * dB, sigma, alpha)[0]
              - _loss_dense(U, kappa, dims, B - h * dB, sigma, alpha)[0]) / (2 * h)
        an = _re_inner(gB, dB)
        assert abs(fd - an) <= 1e-6 * abs(an)
    for j in range(3):
        e = np.zeros(3)
        e[j] = 1.0
        fd = (_loss_dense(U, kappa, dims, B, sigma + h * e, alpha)[0]
              - _loss_dense(U, kappa, dims, B, sigma - h * e, alpha)[0]) / (2 * h)
        assert abs(fd - gs[j]) <= 1e-6 * abs(gs[j])
    for _ in range(6):
        dU = _cplx(rng, U.shape)
        fd = (_loss_dense(U + h * dU, kappa, dims, B, sigma, alpha)[0]
              - _loss_dense(U - h * dU, kappa, dims, B, sigma, alpha)[0]) / (2 * h)
        an = _re_inner(gU, dU)
        assert abs(fd - an) <= 1e-6 * abs(an)
    # single link entries, including ones on the time boundary
    for (t, mu, a, b) in [(0, 3, 0, 1), (1, 3, 2, 2), (1, 0, 1, 0)]:
        dU = np.zeros_like(U)
        dU[t, 1, 0, 1, mu, a, b] = 1.0
        fd = (_loss_dense(U + h * dU, kappa, dims, B, sigma, alpha)[0]
              - _loss_dense(U - h * dU, kappa, dims, B, sigma, alpha)[0]) / (2 * h)
        an = _re_inner(gU, dU)
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-8)


def test_fd_protocol_2x2x2x2():
    """The finite-difference protocol for the gradient workload's shape (m = 2,
    s = 3, h = 1e-6, FP64): 20 random directions in each parameter group (B,
    sigma, U) and 60 random single coordinates (B entries, shifts, link
    entries; every link coordinate on the time boundary is in the mix), each
    directional derivative of the loss against the oracle's analytic
    gradient.  Dense LU solves on 2^4 make each loss evaluation cheap."""
    dims = (2, 2, 2, 2)
    rng = np.random.Generator(np.random.PCG64(407))
    U = synth.su3_links(dims, 0.4, rng)
    kappa = 0.125
    n = 12 * synth.volume(dims)
    B = synth.gaussian_rhs(n, 2, rng)
    sigma = np.array([1e-2, 1e-1, 1.0])
    alpha = np.array([0.2, 0.3, 0.5])
    L0, X = _loss_dense(U, kappa, dims, B, sigma, alpha)
    gB, gs, gU = rhmc_gradients(U, kappa, dims, B, sigma, alpha, X)
    h = 1e-6

    def L(Uv=U, Bv=B, sg=sigma):
        return _loss_dense(Uv, kappa, dims, Bv, sg, alpha)[0]

    def check(fd, an, what):
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-6), (what, fd, an)

    for k in range(20):
        dB = _cplx(rng, B.shape)
        check((L(Bv=B + h * dB) - L(Bv=B - h * dB)) / (2 * h), _re_inner(gB, dB), ("B dir", k))
        ds = rng.standard_normal(3)
        check((L(sg=sigma + h * ds) - L(sg=sigma - h * ds)) / (2 * h), float(gs @ ds), ("sigma dir", k))
        dU = _cplx(rng, U.shape)
        check((L(Uv=U + h * dU) - L(Uv=U - h * dU)) / (2 * h), _re_inner(gU, dU), ("U dir", k))
    coords = []
    for _ in range(20):
        coords.append(("B", (int(rng.integers(2)), int(rng.integers(n))), complex(*rng.standard_normal(2))))
    for j in range(3):
        coords.append(("sigma", (j,), 1.0))
    for _ in range(27):
        idx = tuple(int(rng.integers(k)) for k in U.shape)
        coords.append(("U", idx, complex(*rng.standard_normal(2))))
    # time-boundary links (t = 0 and t = Lt - 1, mu = t), real and imaginary parts
    for t in (0, dims[3] - 1):
        for ph in (1.0, 1.0j):
            coords.append(("U", (t, 1, 0, 1, 3, 1, 2), ph))
            coords.append(("U", (t, 0, 1, 0, 3, 0, 0), ph))
    assert len(coords) >= 50
    for grp, idx, ph in coords:
        if grp == "B":
            d = np.zeros_like(B)
            d[idx] = ph
            check((L(Bv=B + h * d) - L(Bv=B - h * d)) / (2 * h), _re_inner(gB, d), (grp, idx))
        elif grp == "sigma":
            d = np.zeros(3)
            d[idx] = ph
            check((L(sg=sigma + h * d) - L(sg=sigma - h * d)) / (2 * h), float(gs @ d), (grp, idx))
        else:
            d = np.zeros_like(U)
            d[idx] = ph
            check((L(Uv=U + h * d) - L(Uv=U - h * d)) / (2 * h), _re_inner(gU, d), (grp, idx))


@pytest.mark.parametrize("weights", [None, (0.3, 1.7)])
def test_fd_link_gradient_general_adjoint_2x2x2x2(weights):
    """General incoming gradient: L = sum_j w_j Re tr(C_j^H X_j) for fixed
    C_j; then Lambda_j = (sigma_j + A)^{-1} C_j and link_gradient with the
    per-shift weights w_j (default 1) gives dL/dU."""
    dims = (2, 2, 2, 2)
    rng = np.random.Generator(np.random.PCG64(405))
    U = synth.su3_links(dims, 0.5, rng)
    kappa = 0.12
    n = 12 * synth.volume(dims)
    B = synth.gaussian_rhs(n, 2, rng)
    C = _cplx(rng, (2, 2, n))
    sigma = np.array([0.05, 0.5])
    wt = np.ones(2) if weights is None else np.asarray(weights)

    def loss(Uv):
        X = dense_solve(W.dense_A(Uv, kappa, dims), B, sigma)
        return sum(wt[j] * _re_inner(C[j], X[j]) for j in range(2))

    Ad = W.dense_A(U, kappa, dims)
    X = dense_solve(Ad, B, sigma)
    Lam = np.array([np.linalg.solve(Ad + sigma[j] * np.eye(n), C[j].T).T for j in range(2)])
    # dL = -Re tr(Lam^H dA X) -> the sign is carried by link_gradient's convention
    gU = link_gradient(U, kappa, dims, X, Lam, weights)
    h = 1e-6
    for _ in range(4):
        dU = _cplx(rng, U.shape)
        fd = (loss(U + h * dU) - loss(U - h * dU)) / (2 * h)
        an = _re_inner(gU, dU)
        assert abs(fd - an) <= 1e-6 * abs(an)


@pytest.mark.slow
def test_fd_gradients_workload_4x4x4x4():
    wl = synth.make_workload("w4_grad_4x4x4x4")
    dims, U, kappa, B, sigma, alpha = (wl["dims"], wl["U"], wl["kappa"], wl["B"],
                                       wl["sigma"], wl["weights"])

    def solve(Uv, Bv, sg):
        Aop = lambda v: W.A_vec(Uv, kappa, dims, v)
        X, info = dsbcg(Aop, Bv, sg, tol=1e-13, freeze=False)
        assert info["converged"]
        return X

    X = solve(U, B, sigma)
    gB, gs, gU = rhmc_gradients(U, kappa, dims, B, sigma, alpha, X)
    rng = np.random.Generator(np.random.PCG64(406))
    h = 1e-6
    # three random directions per group, every shift, and link coordinates on
    # the time boundary
    for _ in range(3):
        dU = _cplx(rng, U.shape)
        fd = (rhmc_loss(B, solve(U + h * dU, B, sigma), alpha)
              - rhmc_loss(B, solve(U - h * dU, B, sigma), alpha)) / (2 * h)
        an = _re_inner(gU, dU)
        assert abs(fd - an) <= 1e-5 * abs(an)
        dB = _cplx(rng, B.shape)
        fd = (rhmc_loss(B + h * dB, solve(U, B + h * dB, sigma), alpha)
              - rhmc_loss(B - h * dB, solve(U, B - h * dB, sigma), alpha)) / (2 * h)
        an = _re_inner(gB, dB)
        assert abs(fd - an) <= 1e-5 * abs(an)
    for j in range(3):
        e = np.zeros(3)
        e[j] = 1.0
        fd = (rhmc_loss(B, solve(U, B, sigma + h * e), alpha)
              - rhmc_loss(B, solve(U, B, sigma - h * e), alpha)) / (2 * h)
        assert abs(fd - gs[j]) <= 1e-5 * abs(gs[j])
    # a single link entry moves the loss little (derivative ~1e-2), so the
    # 1e-13 solves' noise over 2h = 2e-6 would exceed 1e-5 of it: these
    # coordinates take h = 1e-4 (central-difference truncation ~1e-8 relative)
    hc = 1e-4
    for idx in [(0, 2, 1, 3, 3, 0, 2), (3, 0, 0, 0, 3, 1, 1)]:
        d = np.zeros_like(U)
        d[idx] = 1.0 + 0.5j
        fd = (rhmc_loss(B, solve(U + hc * d, B, sigma), alpha)
              - rhmc_loss(B, solve(U - hc * d, B, sigma), alpha)) / (2 * hc)
        an = _re_inner(gU, d)
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-8)
