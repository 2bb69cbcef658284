"""FP64 CPU oracle for the deflated shifted block CG method (DSBlockCG).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library and
its Python binding) imports, links or runs this package.  It is called only
from tests/, from the smoke check in __graft_entry__ and from the CPU-baseline
leg of bench.py.

It shares no code with the CUDA path: its own gamma matrices, its own Wilson
operator written with dense 4x4 spin matrices and numpy.roll, its own
vector-by-vector band Lanczos solver.  The only shared module is the seeded
input generator (paper_1205_0359_gb300.synth), which holds no method
arithmetic.

Modules
  wilson  -- Wilson-Dirac operator D, D^dagger = g5 D g5, A = D^dagger D (Sec. 1)
  dsbcg   -- DSBlockCG: hermitian band Lanczos with deflation + per-shift
             root-free Cholesky updates of the iterates (Sec. 3, Eqs. 3.1-3.2)
  force   -- gradients of the RHMC-style loss w.r.t. B, sigma_j and the links
  evenodd -- even-odd Schur complement Dhat = 1 - kappa^2 H_oe H_eo of D and
             Ahat = Dhat^H Dhat on the odd sites (a preconditioned variant,
             not the paper's operator)

Parity status: every function here is pinned by tests in tests/test_oracle_*.py
(dense LU, free-field closed form, gamma5-hermiticity, Galerkin definition,
textbook, shifted and block CG, deflation, residual estimate, finite
differences, dense Schur complement and the paired spectrum of the hopping
term).
"""
