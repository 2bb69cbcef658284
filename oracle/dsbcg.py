"""DSBlockCG oracle: deflated shifted block CG in plain numpy, complex128.

Test infrastructure only (see oracle/__init__.py).

Problem (Sec. 1, Eqs. 1.1/1.2): (sigma_j I + A) x_ij = b_i, i = 1..m,
j = 1..s, with sigma_j I + A hermitian positive definite.

Method (Sec. 3).  A hermitian band Lanczos process with deflation -- the
hermitian restriction of the multiple-starting-vector Lanczos method of
Aliaga, Boley, Freund and Hernandez, cited in Sec. 1 -- builds orthonormal
vectors v_1, v_2, ... spanning the deflated block Krylov subspace and the
banded hermitian T = V^H A V (Eq. 3.1).  The iterate of shift sigma is the
Galerkin solution X = V (sigma I + T)^{-1} V^H B (Eq. 3.2, with the shift
handled as in the last paragraph of Sec. 3).  It is updated one Lanczos
vector at a time from a root-free Cholesky factorisation
sigma I + T = L D L^H, extended by one row per vector:

    u^(k) = (V^H B)_k - sum_i l_ki u^(i)          (row vector, length m)
    p^(k) = v_k - sum_i conj(l_ki) p^(i)          (n-vector)
    X    += p^(k) u^(k) / d_k                       (Sec. 3, update formula)

The sums run over the band of row k only (short recurrences of length <= m).
The same Lanczos vectors and T serve every shift; only L, D, p, u are per
shift (Sec. 3, last paragraph).

The process runs vector by vector ("band" form).  The CUDA path runs the
same process block by block; in exact arithmetic both span the same deflated
block Krylov subspace, so their iterates agree at block boundaries and their
converged solutions agree with the unique solution of Eq. 1.1.

Readings where the paper is silent (it defers details to a later paper):
  * deflation test: a candidate is dropped when its norm after
    orthogonalisation is <= dtol times its norm when it was created;
  * T's entries above the diagonal are taken from hermitian symmetry;
  * convergence is judged on the explicit residual ||b_i - (sigma_j+A) x_ij||
    relative to ||b_i||, recomputed every `check_every` vectors; converged
    systems stop being updated (Sec. 4, discussion of Fig. 1).
"""
from __future__ import annotations

import numpy as np


class NotHPD(ArithmeticError):
    pass


def dsbcg(apply_A, B, sigma, tol, dtol=1e-12, max_vectors=None, freeze=True,
          check_every=None, keep_basis=False, stop_after_vectors=None,
          estimate=False):
    """Solve (sigma_j I + A) X_j = B for all shifts with one band Lanczos run.

    apply_A : callable mapping an (n,) or (k, n) complex array to A times it
    B       : (m, n) complex128, rows are right-hand sides b_i
    sigma   : (s,) real shifts, sigma_j I + A hpd
    tol     : stop when every ||b_i - (sigma_j+A) x_ij|| <= tol ||b_i||
    stop_after_vectors : stop after exactly this many Lanczos vectors (no
              convergence test, no final residual pass); used to compare
              against Eq. 3.2 at fixed k and to time a bounded sample.
    estimate : also return info["est_relres"], shape (s, m): the residual
              norms of the Galerkin iterates after the last vector, computed
              without a product with A (Sec. 3, R = W C; see residual_estimate
              below).  Meaningful with freeze=False: a frozen system's
              iterate is no longer the Galerkin iterate.

    Returns (X, info) with X of shape (s, m, n).  info["frozen_at"][j, i] is
    the number of Lanczos vectors after which system (i, j) met tol and was
    frozen (-1: never frozen).
    """
    B = np.asarray(B, dtype=np.complex128)
    if B.ndim == 1:
        B = B[None, :]
    m, n = B.shape
    sigma = np.atleast_1d(np.asarray(sigma, dtype=np.float64))
    s = sigma.size
    bnorm = np.linalg.norm(B, axis=1)
    if check_every is None:
        check_every = max(1, m)
    if max_vectors is None:
        max_vectors = 20 * n

    # Pending candidate vectors, first in first out.  Each remembers where it
    # came from: ("b", c) for the starting vector b_c, ("Av", j) for A v_j,
    # and its norm when created (the deflation reference).
    pending = [dict(vec=B[c].copy(), origin=("b", c), ref=bnorm[c]) for c in range(m)]

    V = []            # Lanczos vectors
    T = {}            # T[(k, i)], i <= k: lower triangle of the hermitian band T
    rho = {}          # rho[(k, c)] = v_k^H b_c  (B = V rho)

    Lrow = [dict() for _ in range(s)]     # Lrow[j][k] = {i: l_ki}
    dval = [dict() for _ in range(s)]     # dval[j][k] = d_k
    urow = [dict() for _ in range(s)]     # urow[j][k] = u^(k), shape (m,)
    pvec = [dict() for _ in range(s)]     # pvec[j][k] = p^(k), shape (n,)
    X = np.zeros((s, m, n), dtype=np.complex128)
    active = np.ones((s, m), dtype=bool)
    relres = np.full((s, m), np.inf)
    frozen_at = np.full((s, m), -1)      # vector count at which (j, i) was frozen
    deflations = 0
    deflated_at = []

    def record(k, origin, value):
        kind, idx = origin
        if kind == "b":
            rho[(k, idx)] = value
        else:
            T[(k, idx)] = value          # coefficient of v_k in A v_idx, idx < k

    def check():
        # explicit residuals of the still-active systems
        for j in range(s):
            cols = np.nonzero(active[j])[0] if freeze else np.arange(m)
            if cols.size == 0:
                continue
            Xa = X[j, cols]
            R = B[cols] - sigma[j] * Xa - apply_A(Xa)
            rr = np.linalg.norm(R, axis=1) / np.where(bnorm[cols] > 0, bnorm[cols], 1.0)
            relres[j, cols] = rr
            if freeze:
                done = cols[rr <= tol]
                active[j, done] = False
                first = done[frozen_at[j, done] < 0]
                frozen_at[j, first] = len(V)

    converged = False
    while pending and len(V) < max_vectors:
        cand = pending.pop(0)
        tau = np.linalg.norm(cand["vec"])
        if tau <= dtol * cand["ref"]:
            # deflation: the candidate is (numerically) in the span of the
            # vectors already built; drop it.
            deflations += 1
            deflated_at.append(len(V))
            continue
        k = len(V)
        v = cand["vec"] / tau
        V.append(v)
        record(k, cand["origin"], tau)
        for other in pending:
            c = np.vdot(v, other["vec"])
            other["vec"] = other["vec"] - c * v
            record(k, other["origin"], c)

        # next candidate: A v_k minus its components along earlier vectors
        # (from the hermitian symmetry of T) and along v_k itself.
        w = apply_A(v)
        ref = np.linalg.norm(w)
        band = sorted(i for (r, i) in T if r == k and i < k)
        for i in band:
            w = w - V[i] * np.conj(T[(k, i)])
        tkk = np.vdot(v, w).real
        T[(k, k)] = tkk
        w = w - tkk * v
        pending.append(dict(vec=w, origin=("Av", k), ref=ref))

        # row k of T is now complete; extend each shift's L D L^H by one row.
        rho_k = np.array([rho.get((k, c), 0.0) for c in range(m)], dtype=np.complex128)
        i0 = band[0] if band else k
        for j in range(s):
            Lk = {}
            for i in range(i0, k):
                acc = T.get((k, i), 0.0)
                Li = Lrow[j].get(i, {})
                for q, lkq in Lk.items():
                    if q < i:
                        acc = acc - lkq * dval[j][q] * np.conj(Li.get(q, 0.0))
                Lk[i] = acc / dval[j][i]
            dk = tkk + sigma[j] - sum(abs(l) ** 2 * dval[j][q] for q, l in Lk.items())
            dk = float(np.real(dk))
            if not dk > 0.0:
                raise NotHPD(f"pivot d_{k} = {dk} <= 0 for shift {sigma[j]}")
            uk = rho_k.copy()
            pk = v.copy()
            for i, lki in Lk.items():
                uk = uk - lki * urow[j][i]
                pk = pk - np.conj(lki) * pvec[j][i]
            Lrow[j][k] = Lk
            dval[j][k] = dk
            urow[j][k] = uk
            pvec[j][k] = pk
            coef = uk / dk
            if freeze:
                coef = np.where(active[j], coef, 0.0)
            X[j] += coef[:, None] * pk[None, :]
            # entries older than the band start are never read again
            for old in [q for q in pvec[j] if q < i0 - 1]:
                del pvec[j][old], urow[j][old]
        if stop_after_vectors is not None:
            if len(V) >= stop_after_vectors:
                break
            continue
        if len(V) % check_every == 0:
            check()
            if np.all(relres <= tol):
                converged = True
                break

    est = None
    if estimate:
        est = residual_estimate(pending, Lrow, dval, urow, len(V), s, m, bnorm)
    if not converged and stop_after_vectors is None:
        # final explicit residuals of every system (frozen ones included)
        was_active = active.copy()
        active[:] = True
        check()
        converged = bool(np.all(relres <= tol))
        active[:] = was_active
    info = dict(nvec=len(V), deflations=deflations, deflated_at=deflated_at,
                relres=relres, converged=converged, invariant=not pending,
                frozen_at=frozen_at)
    if est is not None:
        info["est_relres"] = est
    if keep_basis:
        k = len(V)
        Tm = np.zeros((k, k), dtype=np.complex128)
        for (r, i), val in T.items():
            if r < k and i < k:
                Tm[r, i] = val
                Tm[i, r] = np.conj(val)
        Rm = np.zeros((k, m), dtype=np.complex128)
        for (r, c), val in rho.items():
            if r < k:
                Rm[r, c] = val
        info.update(V=np.array(V), T=Tm, rho=Rm)
    return X, info


def residual_estimate(pending, Lrow, dval, urow, k, s, m, bnorm):
    """Residual norms of the Galerkin iterates from the recurrences (Sec. 3).

    The paper states that R = B - (sigma + A) X is orthogonal to the Lanczos
    vectors built so far and equals W C with W the next (at most m)
    orthonormal Lanczos vectors, so that ||r_i|| is the norm of column i of
    C, obtained from T and its root-free Cholesky factors alone.  In the
    vector-wise process this reads as follows.  With k vectors built, each
    pending candidate w is orthogonal to v_1..v_k and
      * if it came from b_c:   b_c   = V rho[:, c] + w,
      * if it came from A v_q: A v_q = V T[:, q]   + w,
    so with y = (sigma + T_k)^{-1} rho_k,
        r_c = sum_{w from b_c} w  -  sum_{w from A v_q} w * y[q, c].
    The rows y[q] needed are the last ones; they follow from the stored
    band of the factorisation by back substitution, L^H y = D^{-1} u
    (u = L^{-1} rho are the u^(i) of the update formula).  W is an
    orthonormal basis of the pending candidates (QR), and C = R_factor times
    the coefficient matrix above.  Deflated candidates were dropped as
    (numerically) zero, so R = W C holds to the deflation tolerance.

    Returns est[j, c] = ||C_j[:, c]|| / ||b_c||, shape (s, m).
    """
    est = np.zeros((s, m))
    if not pending:
        return est                      # invariant subspace: exact solution
    Wp = np.array([c["vec"] for c in pending]).T          # n x m_c
    _, Rf = np.linalg.qr(Wp)
    av = [c["origin"][1] for c in pending if c["origin"][0] == "Av"]
    lo = min(av) if av else k
    bsafe = np.where(bnorm > 0, bnorm, 1.0)
    for j in range(s):
        y = {}
        for i in range(k - 1, lo - 1, -1):
            yi = urow[j][i] / dval[j][i]
            for l in range(i + 1, k):
                lli = Lrow[j][l].get(i)
                if lli is not None:
                    yi = yi - np.conj(lli) * y[l]
            y[i] = yi
        coef = np.zeros((len(pending), m), dtype=np.complex128)
        for r, c in enumerate(pending):
            kind, idx = c["origin"]
            if kind == "b":
                coef[r, idx] = 1.0
            else:
                coef[r] = -y[idx]
        C = Rf @ coef
        est[j] = np.linalg.norm(C, axis=0) / bsafe
    return est


def rational_combination(B, X, alpha0, alpha):
    """Y = alpha_0 B + sum_j alpha_j X_j, shape (m, n).

    With X_j = (sigma_j I + A)^{-1} B this is r(A) B for the partial fraction
    r(x) = alpha_0 + sum_j alpha_j / (x + sigma_j): the form in which a
    rational approximation of A^nu turns into the shifted systems of Eq. 1.1
    (Sec. 1, the RHMC application).
    """
    B = np.asarray(B, dtype=np.complex128)
    Y = alpha0 * B
    for j, a in enumerate(np.atleast_1d(alpha)):
        Y = Y + a * X[j]
    return Y


def galerkin_iterate(A_dense, B, sigma, nblocks):
    """Definition of the block Galerkin iterate (Eqs. 2.2 and 3.2).

    Builds an orthonormal basis of K_k(A, B) = colspan[B, AB, ..., A^{k-1}B]
    (Eq. 2.1) block by block with full orthogonalisation against every
    earlier block (done twice) and an SVD of each new block, discarding
    directions below 1e-10 of the block's largest singular value (deflation),
    and returns X = V (V^H (sigma I + A) V)^{-1} V^H B for each shift,
    shape (s, m, n).  No short recurrence and no Cholesky update is used.
    """
    B = np.asarray(B, dtype=np.complex128)          # (m, n)

    def orth(W):
        Uu, sv, _ = np.linalg.svd(W, full_matrices=False)
        if sv.size == 0 or sv[0] == 0.0:
            return W[:, :0]
        return Uu[:, : int(np.sum(sv > 1e-10 * sv[0]))]

    Q = orth(B.T)
    basis = [Q]
    for _ in range(1, nblocks):
        if Q.shape[1] == 0:
            break
        W = A_dense @ Q
        scale = np.linalg.norm(W)
        for _rep in range(2):
            for P in basis:
                W = W - P @ (P.conj().T @ W)
        Uu, sv, _ = np.linalg.svd(W, full_matrices=False)
        Q = Uu[:, : int(np.sum(sv > 1e-10 * scale))]
        basis.append(Q)
    Vb = np.concatenate(basis, axis=1)
    r = Vb.shape[1]
    out = []
    for sg in np.atleast_1d(sigma):
        H = Vb.conj().T @ (A_dense @ Vb) + sg * np.eye(r)
        Y = np.linalg.solve(H, Vb.conj().T @ B.T)
        out.append((Vb @ Y).T)
    return np.array(out)


def dense_solve(A_dense, B, sigma):
    """Exact solutions x_ij = (sigma_j I + A)^{-1} b_i by LU (numpy/LAPACK)."""
    n = A_dense.shape[0]
    out = []
    for sg in np.atleast_1d(sigma):
        out.append(np.linalg.solve(A_dense + sg * np.eye(n), np.asarray(B).T).T)
    return np.array(out)


def true_relres(apply_A, B, sigma, X):
    """||b_i - (sigma_j + A) x_ij|| / ||b_i|| for every (j, i); shape (s, m)."""
    B = np.asarray(B)
    bn = np.linalg.norm(B, axis=1)
    out = np.zeros((len(sigma), B.shape[0]))
    for j, sg in enumerate(sigma):
        R = B - sg * X[j] - apply_A(X[j])
        out[j] = np.linalg.norm(R, axis=1) / bn
    return out
