"""True residuals of GPU solutions recomputed with the oracle's own FP64
Wilson operator, for every (rhs, shift) pair of a large workload.

The oracle's solver cannot run at 16^3 x 32 and above, but its operator
can: ||b_i - (sigma_j + A) x_ij|| / ||b_i|| with A = D^H D applied by
oracle.wilson (plain numpy), one vector per call.  numpy releases the GIL in
the array loops, so the vectors of one shift are spread over a thread pool
on the host cores.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from oracle import wilson as W


def _workers():
    return max(1, min(16, os.cpu_count() or 1))


def relres_all(wl, X, shifts=None, rows=None):
    """rel[j, i] for the shifts j in `shifts` (default all) and right-hand
    sides i in `rows` (default all); entries not computed are NaN.

    X: (s, m, n) complex128 (torch tensor on any device, or numpy)."""
    B, sigma = wl["B"], np.asarray(wl["sigma"])
    U, kappa, dims = wl["U"], wl["kappa"], wl["dims"]
    s, m = len(sigma), B.shape[0]
    shifts = range(s) if shifts is None else shifts
    rows = range(m) if rows is None else rows
    bn = np.linalg.norm(B, axis=1)
    rel = np.full((s, m), np.nan)

    def one(args):
        j, i, x = args
        r = B[i] - sigma[j] * x - W.A_vec(U, kappa, dims, x)
        return j, i, float(np.linalg.norm(r) / bn[i])

    with ThreadPoolExecutor(_workers()) as ex:
        for j in shifts:
            Xj = X[j]
            Xj = Xj.cpu().numpy() if hasattr(Xj, "cpu") else np.asarray(Xj)
            for jj, i, v in ex.map(one, [(j, i, Xj[i]) for i in rows]):
                rel[jj, i] = v
            del Xj
    return rel
