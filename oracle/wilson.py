"""Wilson-Dirac operator on a 4D lattice, plain numpy, complex128.

Test infrastructure only (see oracle/__init__.py).

The paper names "the Wilson fermion matrix" as the operator (Sec. 1) and
stores it as a generic sparse matrix (Sec. 4) without fixing a convention.
Convention used here:

  (D psi)(x) = psi(x) - kappa * sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
                                       + (1 + gamma_mu) U_mu(x-mu)^H psi(x-mu) ]

periodic in x, y, z; a hop across the t boundary carries a factor -1
(antiperiodic in time).  Chiral gamma basis:
  gamma_k = [[0, i sigma_k], [-i sigma_k, 0]]  (k = 1, 2, 3),
  gamma_4 = [[0, I], [I, 0]],
  gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(-1, -1, 1, 1).
D^H = gamma_5 D gamma_5 and A = D^H D is hermitian positive semidefinite, so
sigma_j I + A is hpd for every sigma_j > 0 (Sec. 1, Eq. 1.1).

Fields are arrays of shape (..., Lt, Lz, Ly, Lx, 4, 3) [spin, colour]; links
(Lt, Lz, Ly, Lx, 4, 3, 3) [mu, row, col].  Direction mu = 0, 1, 2, 3 is
x, y, z, t, i.e. lattice axes -1, -2, -3, -4 of the site block.
"""
from __future__ import annotations

import numpy as np

SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)


def gamma_matrices():
    """[gamma_1, gamma_2, gamma_3, gamma_4, gamma_5] in the chiral basis."""
    g = []
    for k in range(3):
        g.append(np.block([[_Z2, 1j * SIGMA[k]], [-1j * SIGMA[k], _Z2]]))
    g.append(np.block([[_Z2, _I2], [_I2, _Z2]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g + [g5]


GAMMA = gamma_matrices()
G5 = GAMMA[4]
EYE4 = np.eye(4, dtype=np.complex128)


def field_shape(dims):
    Lx, Ly, Lz, Lt = dims
    return (Lt, Lz, Ly, Lx, 4, 3)


def to_field(v: np.ndarray, dims) -> np.ndarray:
    """Vector(s) in canonical order (site*12 + spin*3 + colour) -> field array."""
    return v.reshape(v.shape[:-1] + field_shape(dims))


def to_vector(f: np.ndarray) -> np.ndarray:
    return f.reshape(f.shape[:-6] + (-1,))


def _axis(mu: int) -> int:
    # site block axes of a field (..., Lt, Lz, Ly, Lx, 4, 3): x=-3, y=-4, z=-5, t=-6
    return -3 - mu


def shift_forward(f: np.ndarray, mu: int) -> np.ndarray:
    """g(x) = f(x + mu) with the time boundary sign."""
    ax = _axis(mu)
    g = np.roll(f, -1, axis=ax)
    if mu == 3:
        idx = [slice(None)] * g.ndim
        idx[ax] = -1                      # sites with t = Lt-1 read t = 0
        g[tuple(idx)] *= -1.0
    return g


def shift_backward(f: np.ndarray, mu: int) -> np.ndarray:
    """g(x) = f(x - mu) with the time boundary sign."""
    ax = _axis(mu)
    g = np.roll(f, 1, axis=ax)
    if mu == 3:
        idx = [slice(None)] * g.ndim
        idx[ax] = 0                       # sites with t = 0 read t = Lt-1
        g[tuple(idx)] *= -1.0
    return g


def _link_backward(U: np.ndarray, mu: int) -> np.ndarray:
    """U_mu(x - mu)^H as a (Lt, Lz, Ly, Lx, 3, 3) array (no boundary sign)."""
    u = U[..., mu, :, :]
    u = np.roll(u, 1, axis=-3 - mu)       # axes of (Lt,Lz,Ly,Lx,3,3): x=-3 ... t=-6
    return np.conj(np.swapaxes(u, -1, -2))


def apply_D(U: np.ndarray, kappa: float, f: np.ndarray) -> np.ndarray:
    """D f for field(s) f of shape (..., Lt, Lz, Ly, Lx, 4, 3)."""
    out = f.copy()
    for mu in range(4):
        fwd = shift_forward(f, mu)
        bwd = shift_backward(f, mu)
        Uf = U[..., mu, :, :]
        Ub = _link_backward(U, mu)
        t_f = np.einsum("...ab,...sb->...sa", Uf, fwd)
        t_b = np.einsum("...ab,...sb->...sa", Ub, bwd)
        t_f = np.einsum("st,...tb->...sb", EYE4 - GAMMA[mu], t_f)
        t_b = np.einsum("st,...tb->...sb", EYE4 + GAMMA[mu], t_b)
        out -= kappa * (t_f + t_b)
    return out


def apply_g5(f: np.ndarray) -> np.ndarray:
    return np.einsum("st,...tb->...sb", G5, f)


def apply_Ddag(U, kappa, f):
    """D^H f = gamma_5 D gamma_5 f."""
    return apply_g5(apply_D(U, kappa, apply_g5(f)))


def apply_A(U, kappa, f):
    """A f = D^H D f."""
    return apply_Ddag(U, kappa, apply_D(U, kappa, f))


# ---- vector-level wrappers (canonical ordering) -------------------------------

def D_vec(U, kappa, dims, v):
    return to_vector(apply_D(U, kappa, to_field(v, dims)))


def Ddag_vec(U, kappa, dims, v):
    return to_vector(apply_Ddag(U, kappa, to_field(v, dims)))


def A_vec(U, kappa, dims, v):
    return to_vector(apply_A(U, kappa, to_field(v, dims)))


def dense_D(U, kappa, dims) -> np.ndarray:
    """Dense n x n matrix of D (tiny lattices only), built column by column."""
    n = 12 * int(np.prod(dims))
    eye = np.eye(n, dtype=np.complex128)
    cols = D_vec(U, kappa, dims, eye)     # row i = D e_i
    return cols.T.copy()


def dense_A(U, kappa, dims) -> np.ndarray:
    Dm = dense_D(U, kappa, dims)
    return Dm.conj().T @ Dm
