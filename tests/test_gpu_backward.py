"""dsbcg_backward and the autograd Functions against the FP64 oracle.

With M_j = sigma_j I + A hermitian, the adjoint solutions are
Lambda_j = M_j^{-1} G_j and the gradients of a real loss through
X_j = M_j^{-1} B are dL/dB = sum_j Lambda_j, dL/dsigma_j =
-Re tr(Lambda_j^H X_j) and dL/dU = the force on (X, Lambda).  Expected values
come from dense LU solves of M_j (4^4 lattice) and the oracle's link
gradient (itself pinned by central finite differences in
tests/test_oracle_force.py).  The autograd gradients are also checked by
central finite differences of the GPU solves themselves (step 1e-6, FP64).
"""
import numpy as np
import pytest
import torch

from oracle import wilson as W
from oracle.dsbcg import dense_solve, rational_combination
from oracle.force import link_gradient
from paper_1205_0359_gb300 import dsbcg, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


@pytest.fixture(scope="module")
def w4():
    wl = synth.make_workload("w4_grad_4x4x4x4")
    Ad = W.dense_A(wl["U"], wl["kappa"], wl["dims"])
    X = dense_solve(Ad, wl["B"], wl["sigma"])
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(DEV), wl["kappa"])
    yield wl, Ad, X, ctx
    ctx.close()


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _cpu(t):
    return t.cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)


@pytest.mark.parametrize("storage,bound,ubound", [("fp64", 1e-9, 1e-9), ("fp32", 1e-9, 1e-5)])
def test_backward_per_shift_gradients(w4, storage, bound, ubound):
    """G_j differs per shift: all s adjoint systems in one call."""
    wl, Ad, X, ctx = w4
    s, m, n = X.shape
    rng = np.random.Generator(np.random.PCG64(21))
    G = synth.gaussian_rhs(n, s * m, rng).reshape(s, m, n)
    Lam_d = np.stack([dense_solve(Ad, G[j], [wl["sigma"][j]])[0] for j in range(s)])
    Lam = torch.empty((s, m, n), dtype=torch.complex128, device=DEV)
    gB, gs, gU, st = ctx.backward(torch.from_numpy(G).to(DEV), wl["sigma"], 1e-12,
                                  X=torch.from_numpy(X).to(DEV), storage=storage, Lambda=Lam)
    assert st["code"] == 0 and st["true_relres"].max() <= 1e-12
    assert _rel(_cpu(Lam), Lam_d) <= bound
    assert _rel(_cpu(gB), Lam_d.sum(axis=0)) <= bound
    want_s = -np.real(np.sum(np.conj(Lam_d) * X, axis=(1, 2)))
    assert _rel(gs, want_s) <= bound
    assert _rel(_cpu(gU), link_gradient(wl["U"], wl["kappa"], wl["dims"], X, Lam_d)) <= ubound


def test_backward_shared_gradient_one_joint_solve(w4):
    """G_j = w_j G with a direct term: dL/dB = a0 G + sum_j w_j M_j^{-1} G,
    from one joint DSBlockCG solve of G; host buffers in and out."""
    wl, Ad, X, ctx = w4
    s, m, n = X.shape
    rng = np.random.Generator(np.random.PCG64(22))
    G = synth.gaussian_rhs(n, m, rng)
    w = np.array([0.5, -1.25, 2.0])
    a0 = 0.75
    Lam_d = w[:, None, None] * dense_solve(Ad, G, wl["sigma"])
    gB, gs, gU, st = ctx.backward(G, wl["sigma"], 1e-12, X=X, g_weights=w, g_direct=a0, storage="fp64")
    assert isinstance(gB, np.ndarray) and st["code"] == 0
    assert _rel(gB, a0 * G + Lam_d.sum(axis=0)) <= 1e-9
    assert _rel(gs, -np.real(np.sum(np.conj(Lam_d) * X, axis=(1, 2)))) <= 1e-9
    assert _rel(gU, link_gradient(wl["U"], wl["kappa"], wl["dims"], X, Lam_d)) <= 1e-9


def test_backward_recomputes_solutions(w4):
    """X = None: the solutions are recomputed from B inside the call; the
    gradients equal those computed from stored solutions."""
    wl, Ad, X, ctx = w4
    s, m, n = X.shape
    rng = np.random.Generator(np.random.PCG64(23))
    G = torch.from_numpy(synth.gaussian_rhs(n, s * m, rng).reshape(s, m, n)).to(DEV)
    Xt = torch.from_numpy(X).to(DEV)
    B = torch.from_numpy(wl["B"]).to(DEV)
    a = ctx.backward(G, wl["sigma"], 1e-12, X=Xt, storage="fp64")
    b = ctx.backward(G, wl["sigma"], 1e-12, B=B, storage="fp64")
    assert b[3]["code"] == 0 and b[3]["block_steps"] > a[3]["block_steps"]
    for u, v in ((a[0], b[0]), (a[1], b[1]), (a[2], b[2])):
        assert _rel(_cpu(v), _cpu(u)) <= 1e-9


def test_backward_argument_errors(w4):
    wl, Ad, X, ctx = w4
    s, m, n = X.shape
    G = np.zeros((m, n), dtype=np.complex128)
    with pytest.raises(dsbcg.DSBCGError) as e:          # a direct term needs shared G
        ctx.backward(np.zeros((s, m, n), dtype=np.complex128), wl["sigma"], 1e-10, X=X, g_direct=1.0)
    assert e.value.code == -1
    with pytest.raises(dsbcg.DSBCGError) as e:          # non-finite weight
        ctx.backward(G, wl["sigma"], 1e-10, X=X, g_weights=[1.0, np.nan, 1.0])
    assert e.value.code == -1


def _fd_check(loss_of, params, grads, rng, ndir, coords, h=1e-6, rtol=1e-5):
    """Central differences of loss_of along random directions of each
    parameter and along single coordinates, against <grad, direction>
    (real part of the complex pairing for complex parameters)."""
    with torch.no_grad():
        for name, p in params.items():
            g = grads[name]
            dirs = []
            for _ in range(ndir):
                if p.is_complex():
                    d = torch.from_numpy(rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape))
                else:
                    d = torch.from_numpy(rng.standard_normal(p.shape))
                dirs.append(d.to(device=p.device, dtype=p.dtype))
            for _ in range(coords.get(name, 0)):
                d = torch.zeros_like(p)
                idx = tuple(int(rng.integers(0, k)) for k in p.shape)
                d[idx] = (1.0 + 1.0j) if p.is_complex() else 1.0
                dirs.append(d)
            for d in dirs:
                plus = {k: (v + h * d if k == name else v) for k, v in params.items()}
                minus = {k: (v - h * d if k == name else v) for k, v in params.items()}
                fd = (loss_of(**plus) - loss_of(**minus)).item() / (2 * h)
                an = torch.sum(torch.real(torch.conj(g) * d)).item()
                assert abs(fd - an) <= rtol * max(abs(an), 1e-3 * abs(fd) + 1e-12), (name, fd, an)


def test_autograd_solve_oracle_and_fd(w4):
    """DSBCGSolve: gradients of L = sum_j alpha_j sum_i Re(b_i^H x_ij) w.r.t.
    B, sigma and U against the oracle, and central finite differences along
    random directions of every group and every shift."""
    from oracle.force import rhmc_gradients, rhmc_loss
    wl, Ad, X, ctx = w4
    alpha = torch.tensor(wl["weights"], dtype=torch.float64)
    args = dict(dims=wl["dims"], kappa=wl["kappa"], tol=1e-12, storage="fp64")

    def loss_of(B, sigma, U):
        Xt = dsbcg.DSBCGSolve.apply(B, sigma, U, args)
        return sum(alpha[j] * torch.real(torch.sum(torch.conj(B) * Xt[j])) for j in range(len(alpha)))

    P = dict(B=torch.from_numpy(wl["B"]).to(DEV).requires_grad_(True),
             sigma=torch.tensor(wl["sigma"], dtype=torch.float64).requires_grad_(True),
             U=torch.from_numpy(wl["U"]).to(DEV).requires_grad_(True))
    L = loss_of(**P)
    L.backward()
    gB, gs, gU = rhmc_gradients(wl["U"], wl["kappa"], wl["dims"], wl["B"], wl["sigma"], wl["weights"], X)
    assert abs(L.item() - rhmc_loss(wl["B"], X, wl["weights"])) < 1e-9 * abs(L.item())
    assert _rel(_cpu(P["B"].grad), gB) < 1e-8
    assert _rel(P["sigma"].grad.numpy(), gs) < 1e-8
    assert _rel(_cpu(P["U"].grad), gU) < 1e-8
    grads = {k: v.grad for k, v in P.items()}
    rng = np.random.Generator(np.random.PCG64(12))
    _fd_check(loss_of, {k: v.detach() for k, v in P.items()}, grads, rng, ndir=3,
              coords=dict(B=2, U=4))
    # every shift coordinate
    with torch.no_grad():
        for j in range(len(wl["sigma"])):
            e = torch.zeros(len(wl["sigma"]), dtype=torch.float64)
            e[j] = 1.0
            h = 1e-6
            fd = (loss_of(P["B"], P["sigma"] + h * e, P["U"]) - loss_of(P["B"], P["sigma"] - h * e, P["U"])).item()
            fd /= 2 * h
            assert abs(fd - P["sigma"].grad[j].item()) <= 1e-5 * abs(P["sigma"].grad[j].item())


def test_autograd_rational_oracle_and_fd(w4):
    """DSBCGRational: Y = a0 B + sum_j alpha_j X_j with L = Re sum conj(C) Y;
    the backward is one joint adjoint solve of C.  Against the oracle's
    gradients and finite differences; recompute mode gives the same
    gradients."""
    wl, Ad, X, ctx = w4
    s, m, n = X.shape
    rng = np.random.Generator(np.random.PCG64(31))
    C = torch.from_numpy(synth.gaussian_rhs(n, m, rng)).to(DEV)
    a0, alpha = 0.4, [0.2, 0.3, 0.5]
    Lam_d = np.asarray(alpha)[:, None, None] * dense_solve(Ad, C.cpu().numpy(), wl["sigma"])
    want_B = a0 * C.cpu().numpy() + Lam_d.sum(axis=0)
    want_s = -np.real(np.sum(np.conj(Lam_d) * X, axis=(1, 2)))
    want_U = link_gradient(wl["U"], wl["kappa"], wl["dims"], X, Lam_d)
    Yd = rational_combination(wl["B"], X, a0, alpha)
    for recompute in (False, True):
        args = dict(dims=wl["dims"], kappa=wl["kappa"], tol=1e-12, storage="fp64", alpha0=a0, alpha=alpha,
                    recompute=recompute)

        def loss_of(B, sigma, U):
            Y = dsbcg.DSBCGRational.apply(B, sigma, U, args)
            return torch.real(torch.sum(torch.conj(C) * Y))

        P = dict(B=torch.from_numpy(wl["B"]).to(DEV).requires_grad_(True),
                 sigma=torch.tensor(wl["sigma"], dtype=torch.float64).requires_grad_(True),
                 U=torch.from_numpy(wl["U"]).to(DEV).requires_grad_(True))
        Y = dsbcg.DSBCGRational.apply(P["B"], P["sigma"], P["U"], args)
        assert _rel(_cpu(Y.detach()), Yd) < 1e-9
        L = torch.real(torch.sum(torch.conj(C) * Y))
        L.backward()
        assert _rel(_cpu(P["B"].grad), want_B) < 1e-8
        assert _rel(P["sigma"].grad.numpy(), want_s) < 1e-8
        assert _rel(_cpu(P["U"].grad), want_U) < 1e-8
        if not recompute:
            _fd_check(loss_of, {k: v.detach() for k, v in P.items()}, {k: v.grad for k, v in P.items()},
                      np.random.Generator(np.random.PCG64(32)), ndir=2, coords=dict(U=2))


def test_autograd_context_reuse_and_retained_graph(w4):
    """A caller-owned Context serves several forwards (links packed once) and
    stays open; a retained graph runs backward twice with equal results."""
    wl, Ad, X, ctx = w4
    U = torch.from_numpy(wl["U"]).to(DEV)
    args = dict(dims=wl["dims"], kappa=wl["kappa"], tol=1e-12, storage="fp64", context=ctx)
    B = torch.from_numpy(wl["B"]).to(DEV).requires_grad_(True)
    sig = torch.tensor(wl["sigma"], dtype=torch.float64)
    for _ in range(2):
        Xt = dsbcg.DSBCGSolve.apply(B, sig, U, args)
        L = torch.real(torch.sum(torch.conj(B.detach()) * Xt[0]))
        L.backward(retain_graph=True)
        g1 = B.grad.clone()
        B.grad = None
        L.backward()
        assert torch.allclose(B.grad, g1, rtol=0, atol=0)
        B.grad = None
    assert ctx._ctx                                   # still open
    Xc, _ = ctx.solve(torch.from_numpy(wl["B"]).to(DEV), wl["sigma"], 1e-10, storage="fp64")
    assert _rel(_cpu(Xc), X) < 1e-7
