"""Seeded synthetic inputs: SU(3) gauge links, right-hand sides and shifts.

This module is the only code shared between the CUDA path's tests/bench and the
FP64 oracle.  It draws random inputs and nothing else: no Dirac operator, no
solver arithmetic.  Everything is generated on the host in float64/complex128
from numpy's PCG64 with a fixed seed per workload.

Canonical external layouts (the C ABI uses the same ones):
  * lattice site index  site = x + Lx*(y + Ly*(z + Lz*t))
  * gauge field         complex128 array [Lt][Lz][Ly][Lx][mu=x,y,z,t][row][col]
  * spinor vector       complex128, index site*12 + spin*3 + colour  (n = 12*V)
  * right-hand sides    complex128 [m][n];  solutions complex128 [s][m][n]

The paper's gauge configuration (quenched, beta = 6.0, Sec. 4) is not
available; smooth random SU(3) links U = exp(i*eps*H), with H a Gaussian
traceless hermitian 3x3 matrix per link, stand in for it.  The shifts are
log-spaced so that the shifted systems span the conditioning range the paper
describes for its experiments (Sec. 4).
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "volume", "su3_links", "gaussian_rhs", "z2_rhs", "log_shifts",
    "Workload", "WORKLOADS", "make_workload", "sha256_of",
]


def volume(dims) -> int:
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    return Lx * Ly * Lz * Lt


def _unitarise_su3(u: np.ndarray) -> np.ndarray:
    """Project nearly-unitary 3x3 matrices (last two axes) onto SU(3).

    Row 1 is normalised, row 2 is Gram-Schmidt orthogonalised against it and
    normalised, row 3 is the complex conjugate of the cross product of rows 1
    and 2, which makes the determinant exactly one.
    """
    r1 = u[..., 0, :]
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = u[..., 1, :]
    r2 = r2 - np.sum(np.conj(r1) * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.linalg.norm(r2, axis=-1, keepdims=True)
    r3 = np.conj(np.cross(r1, r2))
    return np.stack([r1, r2, r3], axis=-2)


def su3_links(dims, eps: float, rng: np.random.Generator) -> np.ndarray:
    """Random SU(3) links U = exp(i*eps*H) for every site and direction.

    H = (G + G^H)/2 - tr(.)/3 with G_ab = (g + i g')/sqrt(2), g, g' ~ N(0, 1).
    The exponential is taken through the eigendecomposition of H, then the
    result is re-projected onto SU(3) to remove rounding drift.
    Returns complex128 [Lt][Lz][Ly][Lx][4][3][3].
    """
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    shape = (Lt, Lz, Ly, Lx, 4, 3, 3)
    g = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
    h = 0.5 * (g + np.conj(np.swapaxes(g, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[..., None, None] * np.eye(3)
    lam, q = np.linalg.eigh(h)
    ph = np.exp(1j * eps * lam)
    u = np.einsum("...ab,...b,...cb->...ac", q, ph, np.conj(q))
    return _unitarise_su3(u)


def gaussian_rhs(n: int, m: int, rng: np.random.Generator) -> np.ndarray:
    """m complex Gaussian vectors of length n, entries (g + i g')/sqrt(2). [m][n]"""
    return (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(2.0)


def z2_rhs(n: int, m: int, rng: np.random.Generator) -> np.ndarray:
    """m Z2-noise vectors, entries (+-1 +- i)/sqrt(2). [m][n]"""
    re = rng.integers(0, 2, size=(m, n)) * 2 - 1
    im = rng.integers(0, 2, size=(m, n)) * 2 - 1
    return (re + 1j * im) / np.sqrt(2.0)


def log_shifts(lo: float, hi: float, s: int) -> np.ndarray:
    """s real shifts log-spaced over [lo, hi] (partial-fraction-like spacing)."""
    if s == 1:
        return np.array([float(lo)])
    return 10.0 ** np.linspace(np.log10(lo), np.log10(hi), s)


@dataclass
class Workload:
    name: str
    dims: tuple
    kappa: float
    eps: float
    m: int
    s: int
    rhs: str                 # "gaussian" | "z2"
    shifts: tuple            # explicit shift list
    tol: float
    seed: int
    dependent: str = ""      # "" | "exact" (b_m = b_1 + b_2) | "near" (b_m = b_1 + 1e-9 noise)
    weights: tuple = ()      # rational-approximation weights alpha_j (gradient workload)
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return 12 * volume(self.dims)


# The five workloads: sizes, link smoothness, kappa, RHS kind, shifts and
# tolerances.  Seeds are fixed per workload.
WORKLOADS = {
    "w1_4x4x4x4": Workload(
        "w1_4x4x4x4", (4, 4, 4, 4), 0.12, 0.3, 4, 4, "gaussian",
        (1e-3, 1e-2, 1e-1, 1.0), 1e-10, seed=12050359_1, dependent="exact",
        note="plain FP64; b_4 = b_1 + b_2 exactly so deflation must trigger"),
    "w2_16x16x16x32": Workload(
        "w2_16x16x16x32", (16, 16, 16, 32), 0.125, 0.5, 12, 12, "z2",
        tuple(log_shifts(1e-4, 10.0, 12)), 1e-8, seed=12050359_2,
        note="Z2 noise RHS; FP32 with FP64 reliable updates vs plain FP64"),
    "w3_24x24x24x48": Workload(
        "w3_24x24x24x48", (24, 24, 24, 48), 0.13, 0.6, 8, 8, "gaussian",
        tuple(log_shifts(1e-4, 1.0, 8)), 1e-8, seed=12050359_3,
        note="storage precision ladder fp64/fp32/bf16/fp16"),
    "w4_grad_4x4x4x4": Workload(
        "w4_grad_4x4x4x4", (4, 4, 4, 4), 0.12, 0.3, 2, 3, "gaussian",
        (1e-2, 1e-1, 1.0), 1e-13, seed=12050359_4, weights=(0.2, 0.3, 0.5),
        note="finite-difference gradient check"),
    "w4_force_16x16x16x32": Workload(
        "w4_force_16x16x16x32", (16, 16, 16, 32), 0.125, 0.5, 8, 8, "gaussian",
        tuple(log_shifts(1e-4, 1.0, 8)), 1e-8, seed=12050359_44,
        weights=tuple(np.linspace(0.05, 0.4, 8)),
        note="force kernel throughput in FP32"),
    "cmp_16x16x16x16": Workload(
        "cmp_16x16x16x16", (16, 16, 16, 16), 0.125, 0.5, 4, 7, "gaussian",
        tuple(log_shifts(1e-6, 1e-1, 7)), 1e-8, seed=12050359_6,
        note="the paper's algorithm comparison (Sec. 4, Table 1): 16^4, 4 RHS, 7 shifts over 1e-6..1e-1"),
    "cmp_critical_16x16x16x16": Workload(
        "cmp_critical_16x16x16x16", (16, 16, 16, 16), 0.15, 0.5, 4, 7, "gaussian",
        tuple(log_shifts(1e-6, 1e-1, 7)), 1e-8, seed=12050359_7,
        note="the comparison of Sec. 4 on a lattice near its critical kappa (smooth links, kappa 0.15), "
             "where DSBlockCG needs fewer A applications than shifted CG"),
    "w5_32x32x32x64": Workload(
        "w5_32x32x32x64", (32, 32, 32, 64), 0.13, 0.6, 16, 8, "gaussian",
        tuple(log_shifts(1e-5, 1.0, 8)), 1e-8, seed=12050359_5, dependent="near",
        note="b_16 = b_1 + 1e-9 noise; mixed precision, ~70 GB"),
}


def make_workload(name_or_wl, dims=None, m=None, s=None, seed=None):
    """Generate (U, B, sigma) for a workload, optionally resized.

    Returns a dict with keys: dims, kappa, U (complex128 [Lt][Lz][Ly][Lx][4][3][3]),
    B (complex128 [m][n]), sigma (float64 [s]), tol, weights, name.
    Resizing keeps the recipe (link smoothness, kappa, RHS kind, dependency)
    and re-spaces the shifts over the same range.
    """
    wl = WORKLOADS[name_or_wl] if isinstance(name_or_wl, str) else name_or_wl
    dims = tuple(dims) if dims is not None else wl.dims
    m = int(m) if m is not None else wl.m
    s = int(s) if s is not None else wl.s
    seed = int(seed) if seed is not None else wl.seed
    rng = np.random.Generator(np.random.PCG64(seed))
    U = su3_links(dims, wl.eps, rng)
    n = 12 * volume(dims)
    if wl.rhs == "z2":
        B = z2_rhs(n, m, rng)
    else:
        B = gaussian_rhs(n, m, rng)
    if wl.dependent == "exact" and m >= 3:
        B[m - 1] = B[0] + B[1]
    elif wl.dependent == "near" and m >= 2:
        B[m - 1] = B[0] + 1e-9 * gaussian_rhs(n, 1, rng)[0]
    if s == len(wl.shifts):
        sigma = np.array(wl.shifts, dtype=np.float64)
    else:
        sigma = log_shifts(min(wl.shifts), max(wl.shifts), s)
    weights = np.array(wl.weights if len(wl.weights) == s else np.linspace(0.1, 0.5, s))
    return dict(name=wl.name, dims=dims, kappa=wl.kappa, U=U, B=B, sigma=sigma,
                tol=wl.tol, weights=weights)


def sha256_of(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()
