"""Even-odd (Schur complement) reduction of the Wilson operator, plain numpy.

Test infrastructure only (see oracle/__init__.py).

Not part of the paper's method: the paper applies its solver to the full
Wilson matrix and exploits no structure of it (Sec. 4).  This module defines
the preconditioned variant that a later solver path is checked against.

Write D = 1 - kappa H with H the nearest-neighbour hopping term of
oracle.wilson (gamma projections, links, time-boundary sign).  Colour the
sites by the parity of x + y + z + t.  When every extent is even, H only
connects sites of opposite parity, so in (even, odd) block order

    D = [[ 1,            -kappa H_eo ],
         [ -kappa H_oe,   1          ]]

and the Schur complement on the odd sites is

    Dhat = 1 - kappa^2 H_oe H_eo.

A solution of D x = b follows from the half-size system
    Dhat x_o = b_o + kappa H_oe b_e,      x_e = b_e + kappa H_eo x_o,
and det D = det Dhat.  Dhat^H = gamma_5 Dhat gamma_5 (from the same property
of D), so Ahat = Dhat^H Dhat is hermitian positive semidefinite and
sigma I + Ahat is hpd for sigma > 0: DSBlockCG applies to it unchanged.

Half-lattice vectors list the sites of one parity in increasing canonical
site order (site = x + Lx (y + Ly (z + Lz t))), 12 components per site
(spin * 3 + colour), n_half = 12 V / 2.
"""
from __future__ import annotations

import numpy as np

from . import wilson as W

EVEN, ODD = 0, 1


def parity_sites(dims, parity):
    """Canonical indices of the sites whose x + y + z + t has this parity."""
    Lx, Ly, Lz, Lt = dims
    if any(L % 2 for L in dims):
        raise ValueError("even-odd reduction needs every lattice extent even")
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                             indexing="ij")
    par = ((x + y + z + t) % 2).reshape(-1)
    return np.nonzero(par == parity)[0]


def pack(v, dims, parity):
    """Full vector(s) (..., 12 V) -> half vector(s) (..., 6 V) of one parity."""
    sites = parity_sites(dims, parity)
    f = v.reshape(v.shape[:-1] + (-1, 12))
    return f[..., sites, :].reshape(v.shape[:-1] + (-1,))


def unpack(h, dims, parity):
    """Half vector(s) of one parity -> full vector(s), zero on the other parity."""
    sites = parity_sites(dims, parity)
    V = int(np.prod(dims))
    out = np.zeros(h.shape[:-1] + (V, 12), dtype=np.complex128)
    out[..., sites, :] = h.reshape(h.shape[:-1] + (-1, 12))
    return out.reshape(h.shape[:-1] + (-1,))


def hop_vec(U, kappa, dims, v):
    """H v = (v - D v) / kappa on full vectors."""
    return (v - W.D_vec(U, kappa, dims, v)) / kappa


def Dhat_vec(U, kappa, dims, h):
    """Dhat h = h - kappa^2 H_oe H_eo h on odd half vectors."""
    he = pack(hop_vec(U, kappa, dims, unpack(h, dims, ODD)), dims, EVEN)      # H_eo h
    ho = pack(hop_vec(U, kappa, dims, unpack(he, dims, EVEN)), dims, ODD)     # H_oe H_eo h
    return h - kappa * kappa * ho


def _g5_half(h):
    f = h.reshape(h.shape[:-1] + (-1, 4, 3))
    return np.einsum("st,...tb->...sb", W.G5, f).reshape(h.shape)


def Dhat_dag_vec(U, kappa, dims, h):
    """Dhat^H h = gamma_5 Dhat gamma_5 h."""
    return _g5_half(Dhat_vec(U, kappa, dims, _g5_half(h)))


def Ahat_vec(U, kappa, dims, h):
    """Ahat h = Dhat^H Dhat h."""
    return Dhat_dag_vec(U, kappa, dims, Dhat_vec(U, kappa, dims, h))


def schur_solve_D(U, kappa, dims, b, solve_Dhat):
    """x with D x = b through the odd-site Schur system.

    solve_Dhat maps a right-hand side c (odd half vector) to Dhat^{-1} c.
    """
    be, bo = pack(b, dims, EVEN), pack(b, dims, ODD)
    c = bo + kappa * pack(hop_vec(U, kappa, dims, unpack(be, dims, EVEN)), dims, ODD)
    xo = solve_Dhat(c)
    xe = be + kappa * pack(hop_vec(U, kappa, dims, unpack(xo, dims, ODD)), dims, EVEN)
    return unpack(xe, dims, EVEN) + unpack(xo, dims, ODD)


def dense_Dhat(U, kappa, dims):
    """Dense n_half x n_half matrix of Dhat (tiny lattices only)."""
    nh = 6 * int(np.prod(dims))
    eye = np.eye(nh, dtype=np.complex128)
    return Dhat_vec(U, kappa, dims, eye).T.copy()


def dense_Ahat(U, kappa, dims):
    Dh = dense_Dhat(U, kappa, dims)
    return Dh.conj().T @ Dh
