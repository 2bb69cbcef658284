"""Pins for the oracle's Wilson operator (CPU only).

Each test checks the oracle against something other than itself: Clifford
algebra, SU(3) group properties, the free-field (unit gauge) Fourier closed
form of D and of the spectrum of A = D^H D, gamma5-hermiticity, hermiticity of
A, gauge covariance, and a hand-written single-site hop computed with plain
Python loops.
"""
import itertools

import numpy as np
import pytest

from oracle import wilson as W
from paper_1205_0359_gb300 import synth


def test_gamma_algebra():
    g = W.GAMMA
    for mu, nu in itertools.product(range(4), range(4)):
        ac = g[mu] @ g[nu] + g[nu] @ g[mu]
        assert np.allclose(ac, 2.0 * np.eye(4) * (mu == nu), atol=1e-15)
    for mu in range(5):
        assert np.allclose(g[mu], g[mu].conj().T)
    assert np.allclose(g[4], np.diag([-1, -1, 1, 1]))
    for mu in range(4):
        assert np.allclose(g[4] @ g[mu], -g[mu] @ g[4])


def test_su3_links_are_special_unitary():
    rng = np.random.Generator(np.random.PCG64(7))
    U = synth.su3_links((2, 3, 2, 4), 0.6, rng)
    uu = np.einsum("...ab,...cb->...ac", U, np.conj(U))
    assert np.max(np.abs(uu - np.eye(3))) < 1e-14
    assert np.max(np.abs(np.linalg.det(U) - 1.0)) < 1e-14
    # not trivially the identity
    assert np.min(np.abs(U - np.eye(3)).reshape(-1, 9).max(axis=1)) > 1e-3


def _free_links(dims):
    Lx, Ly, Lz, Lt = dims
    return np.broadcast_to(np.eye(3, dtype=np.complex128), (Lt, Lz, Ly, Lx, 4, 3, 3)).copy()


def _momenta(dims):
    Lx, Ly, Lz, Lt = dims
    for nx, ny, nz, nt in itertools.product(range(Lx), range(Ly), range(Lz), range(Lt)):
        yield np.array([2 * np.pi * nx / Lx, 2 * np.pi * ny / Ly, 2 * np.pi * nz / Lz,
                        (2 * nt + 1) * np.pi / Lt])


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_free_field_spectrum_closed_form(dims):
    kappa = 0.13
    U = _free_links(dims)
    Ad = W.dense_A(U, kappa, dims)
    ev = np.sort(np.linalg.eigvalsh(Ad))
    closed = []
    for p in _momenta(dims):
        lam = (1 - 2 * kappa * np.sum(np.cos(p))) ** 2 + 4 * kappa ** 2 * np.sum(np.sin(p) ** 2)
        closed += [lam] * 12
    assert np.allclose(ev, np.sort(closed), atol=1e-13)


def test_free_field_plane_wave_4x4x4x4():
    """D e^{ip.x} chi = [(1 - 2k sum cos p) + 2ik sum gamma_mu sin p_mu] e^{ip.x} chi."""
    dims = (4, 4, 4, 4)
    kappa = 0.12
    U = _free_links(dims)
    rng = np.random.default_rng(3)
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(range(Lt), range(Lz), range(Ly), range(Lx), indexing="ij")
    for p in [np.array([2 * np.pi / 4, 0, 2 * np.pi * 3 / 4, 3 * np.pi / 4]),
              np.array([0, 2 * np.pi / 4, 2 * np.pi / 4, np.pi / 4])]:
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        f = phase[..., None, None] * chi
        Dp = (1 - 2 * kappa * np.sum(np.cos(p))) * np.eye(4) + 2j * kappa * sum(
            W.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
        expect = phase[..., None, None] * (Dp @ chi)
        got = W.apply_D(U, kappa, f)
        assert np.max(np.abs(got - expect)) < 1e-13


@pytest.fixture(scope="module")
def rough():
    dims = (4, 2, 4, 4)
    rng = np.random.Generator(np.random.PCG64(11))
    U = synth.su3_links(dims, 0.8, rng)
    n = 12 * synth.volume(dims)
    u = synth.gaussian_rhs(n, 1, rng)[0]
    v = synth.gaussian_rhs(n, 1, rng)[0]
    return dims, U, u, v


def test_gamma5_hermiticity_and_A_hermitian(rough):
    dims, U, u, v = rough
    k = 0.13
    lhs = np.vdot(u, W.D_vec(U, k, dims, v))
    rhs = np.vdot(W.Ddag_vec(U, k, dims, u), v)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    a1 = np.vdot(u, W.A_vec(U, k, dims, v))
    a2 = np.conj(np.vdot(v, W.A_vec(U, k, dims, u)))
    assert abs(a1 - a2) <= 1e-13 * abs(a1)
    # positive semidefinite quadratic form
    assert np.vdot(u, W.A_vec(U, k, dims, u)).real > 0


def test_dense_gamma5_hermiticity_2x2x2x2():
    dims = (2, 2, 2, 2)
    rng = np.random.Generator(np.random.PCG64(5))
    U = synth.su3_links(dims, 0.7, rng)
    Dm = W.dense_D(U, 0.12, dims)
    nsite = synth.volume(dims)
    g5 = np.kron(np.eye(nsite), np.kron(W.G5, np.eye(3)))
    assert np.max(np.abs(Dm.conj().T - g5 @ Dm @ g5)) < 1e-14


def test_gauge_covariance(rough):
    dims, U, u, _ = rough
    k = 0.11
    rng = np.random.Generator(np.random.PCG64(99))
    Lx, Ly, Lz, Lt = dims
    g = synth.su3_links(dims, 1.0, rng)[..., 0, :, :]       # one SU(3) matrix per site
    Ug = np.empty_like(U)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=3 - mu)               # g(x + mu), site axes (t,z,y,x)
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    f = W.to_field(u, dims)
    fg = np.einsum("...ab,...sb->...sa", g, f)
    lhs = W.apply_D(Ug, k, fg)
    rhs = np.einsum("...ab,...sb->...sa", g, W.apply_D(U, k, f))
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_single_site_hops_by_hand():
    """A point source at site y: D psi is non-zero only at y and its 8 neighbours,
    with the values written out term by term."""
    dims = (3, 4, 2, 4)
    Lx, Ly, Lz, Lt = dims
    rng = np.random.Generator(np.random.PCG64(1234))
    U = synth.su3_links(dims, 0.9, rng)
    k = 0.1
    y = (1, 2, 1, 3)              # x, y, z, t  (t = Lt - 1: forward t hop wraps)
    chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    f = np.zeros((Lt, Lz, Ly, Lx, 4, 3), dtype=np.complex128)
    f[y[3], y[2], y[1], y[0]] = chi
    out = W.apply_D(U, k, f)
    g = W.GAMMA
    expect = {}

    def add(site, val):
        key = tuple(site)
        expect[key] = expect.get(key, 0) + val

    add(y, chi)
    L = [Lx, Ly, Lz, Lt]
    for mu in range(4):
        # site x = y - mu sees psi(x + mu) = chi through U_mu(x)
        x = list(y)
        x[mu] -= 1
        sign = 1.0
        if x[mu] < 0:
            x[mu] += L[mu]
            sign = -1.0 if mu == 3 else 1.0
        Ux = U[x[3], x[2], x[1], x[0], mu]
        add(x, -k * sign * (np.eye(4) - g[mu]) @ (chi @ Ux.T))
        # site x = y + mu sees psi(x - mu) = chi through U_mu(x - mu)^H = U_mu(y)^H
        x = list(y)
        x[mu] += 1
        sign = 1.0
        if x[mu] >= L[mu]:
            x[mu] -= L[mu]
            sign = -1.0 if mu == 3 else 1.0
        Uy = U[y[3], y[2], y[1], y[0], mu]
        add(x, -k * sign * (np.eye(4) + g[mu]) @ (chi @ np.conj(Uy)))
    ref = np.zeros_like(f)
    for (xx, yy, zz, tt), val in expect.items():
        ref[tt, zz, yy, xx] += val
    assert np.max(np.abs(out - ref)) < 1e-14
