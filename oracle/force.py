"""Gradients of shifted solves w.r.t. B, the shifts and the gauge links.

Test infrastructure only (see oracle/__init__.py).

Not in the paper: the paper motivates multiple shifts by the RHMC rational
approximation (Sec. 1), whose molecular-dynamics force needs derivatives of
the shifted solutions.  With M_j = sigma_j I + A (hermitian) and
X_j = M_j^{-1} B, a real loss L with incoming gradients G_j = dL/dX_j has
adjoint solutions Lambda_j = M_j^{-1} G_j and

    dL/dB       = sum_j Lambda_j
    dL/dsigma_j = -Re tr(Lambda_j^H X_j)
    dL/dU_mu(y) = kappa * sum_j w_j sum_i [F(D x_ij, lambda_ij) + F(D lambda_ij, x_ij)]_mu(y)

where, for spin-colour fields a and b,

    F(a, b)_mu(y) = sum_spin [(1 - gamma_mu) a(y)] (x) conj(b(y+mu))
                  + sum_spin [(1 + gamma_mu) b(y)] (x) conj(a(y+mu)),

with (x) the colour outer product and the time-boundary sign on the hop.
Complex gradients follow PyTorch's convention dL/dRe z + i dL/dIm z.  For the
loss L = sum_j alpha_j sum_i Re(b_i^H x_ij), G_j = alpha_j B, so
Lambda_j = alpha_j X_j and no extra solve is needed.
"""
from __future__ import annotations

import numpy as np

from .wilson import EYE4, GAMMA, apply_D, shift_forward, to_field


def rhmc_loss(B, X, alpha):
    """L = sum_j alpha_j sum_i Re(b_i^H x_ij); B (m, n), X (s, m, n)."""
    return float(sum(a * np.sum(np.real(np.conj(B) * X[j])) for j, a in enumerate(alpha)))


def F_outer(a, b):
    """F(a, b) summed over leading batch axes; a, b (K, Lt, Lz, Ly, Lx, 4, 3).

    Returns complex128 (Lt, Lz, Ly, Lx, 4, 3, 3) [mu, row, col].
    """
    out = np.zeros(a.shape[1:5] + (4, 3, 3), dtype=np.complex128)
    for mu in range(4):
        pm = EYE4 - GAMMA[mu]
        pp = EYE4 + GAMMA[mu]
        b_fwd = shift_forward(b, mu)
        a_fwd = shift_forward(a, mu)
        t1 = np.einsum("st,kTZYXtA,kTZYXsB->TZYXAB", pm, a, np.conj(b_fwd))
        t2 = np.einsum("st,kTZYXtA,kTZYXsB->TZYXAB", pp, b, np.conj(a_fwd))
        out[..., mu, :, :] = t1 + t2
    return out


def link_gradient(U, kappa, dims, X, Lam, weights=None):
    """dL/dU for solutions X and adjoint solutions Lam, both (s, m, n).

    weights w_j multiply shift j's contribution (default 1).
    """
    s, m, n = X.shape
    if weights is None:
        weights = np.ones(s)
    Xf = to_field(X.reshape(s * m, n), dims)
    Lf = to_field(Lam.reshape(s * m, n), dims)
    w = np.repeat(np.asarray(weights, dtype=np.float64), m)
    Wf = w[:, None, None, None, None, None, None]
    eta_x = apply_D(U, kappa, Xf)
    eta_l = apply_D(U, kappa, Lf)
    return kappa * (F_outer(Wf * eta_x, Lf) + F_outer(Wf * eta_l, Xf))


def rhmc_gradients(U, kappa, dims, B, sigma, alpha, X):
    """Gradients of rhmc_loss at the exact solutions X (s, m, n).

    Returns (grad_B (m, n), grad_sigma (s,), grad_U (Lt,Lz,Ly,Lx,4,3,3)).
    """
    alpha = np.asarray(alpha, dtype=np.float64)
    # direct term alpha_j b_i^H x_ij plus the solve term through x_ij = M_j^{-1} b_i
    grad_B = 2.0 * np.einsum("j,jmn->mn", alpha, X)
    grad_sigma = -alpha * np.sum(np.abs(X) ** 2, axis=(1, 2))
    Lam = alpha[:, None, None] * X
    grad_U = link_gradient(U, kappa, dims, X, Lam)
    return grad_B, grad_sigma, grad_U
