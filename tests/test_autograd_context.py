"""Lifetime of the library context inside the autograd Functions (CPU only:
the library is replaced by a fake Context that counts opens and closes).

* a forward whose inputs need no gradient closes its own context at once;
* a forward that records a graph keeps the context until the graph is
  freed, and a retained graph can run backward twice;
* a caller-owned context (args["context"]) is never closed by the Function.
"""
import gc

import numpy as np
import pytest
import torch

from paper_1205_0359_gb300 import dsbcg


class FakeContext:
    opened = 0
    closed = 0

    def __init__(self, dims=None, U=None, kappa=None, **kw):
        FakeContext.opened += 1
        self._ctx = True
        self.n = 12

    def close(self):
        if self._ctx:
            FakeContext.closed += 1
            self._ctx = False

    def solve(self, B, sigma, tol, storage="fp32", **kw):
        assert self._ctx, "solve on a closed context"
        sig = torch.as_tensor(np.asarray(sigma))
        return torch.stack([B / (1.0 + s) for s in sig]), {}

    def solve_rational(self, B, sigma, alpha0, alpha, tol, storage="fp32", X=None, **kw):
        assert self._ctx
        Xs, _ = self.solve(B, sigma, tol)
        if X is not None:
            X.copy_(Xs)
        return alpha0 * B + sum(a * Xs[j] for j, a in enumerate(alpha)), {}

    def backward(self, G, sigma, tol, X=None, B=None, g_weights=None, g_direct=0.0, want=(), **kw):
        assert self._ctx, "backward on a closed context"
        sig = np.asarray(sigma)
        if g_weights is None:
            gB = sum(G[j] / (1.0 + s) for j, s in enumerate(sig))
        else:
            gB = g_direct * G + sum(w * G / (1.0 + s) for w, s in zip(g_weights, sig))
        return (gB if "B" in want else None, np.zeros(sig.size) if "sigma" in want else None, None, {})


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(dsbcg, "Context", FakeContext)
    FakeContext.opened = FakeContext.closed = 0
    yield FakeContext


ARGS = dict(dims=(1, 1, 1, 1), kappa=0.1, tol=1e-8)


def _inputs(grad_b):
    B = torch.randn(2, 12, dtype=torch.complex128, requires_grad=grad_b)
    sig = torch.tensor([0.1, 1.0], dtype=torch.float64)
    U = torch.zeros(1, 1, 1, 1, 4, 3, 3, dtype=torch.complex128)
    return B, sig, U


@pytest.mark.parametrize("fn", [dsbcg.DSBCGSolve, dsbcg.DSBCGRational])
def test_no_grad_forward_closes_context(fake, fn):
    B, sig, U = _inputs(False)
    args = dict(ARGS, alpha0=0.5, alpha=[1.0, 2.0])
    fn.apply(B, sig, U, args)
    assert fake.opened == 1 and fake.closed == 1
    with torch.no_grad():
        B.requires_grad_(True)
        fn.apply(B, sig, U, args)
    assert fake.opened == 2 and fake.closed == 2


@pytest.mark.parametrize("fn", [dsbcg.DSBCGSolve, dsbcg.DSBCGRational])
def test_graph_keeps_context_and_retained_backward(fake, fn):
    B, sig, U = _inputs(True)
    args = dict(ARGS, alpha0=0.5, alpha=[1.0, 2.0])
    out = fn.apply(B, sig, U, args)
    L = torch.real(out.sum())
    assert fake.opened == 1 and fake.closed == 0
    L.backward(retain_graph=True)
    g1 = B.grad.clone()
    B.grad = None
    L.backward()                                      # second backward on the retained graph
    assert torch.equal(B.grad, g1)
    assert fake.closed == 0
    del out, L
    gc.collect()
    assert fake.closed == 1                           # freed with the graph


def test_forward_without_backward_is_freed_with_graph(fake):
    B, sig, U = _inputs(True)
    out = dsbcg.DSBCGSolve.apply(B, sig, U, dict(ARGS))
    assert fake.closed == 0
    del out
    gc.collect()
    assert fake.opened == 1 and fake.closed == 1


def test_caller_owned_context_is_never_closed(fake):
    c = FakeContext()
    B, sig, U = _inputs(True)
    for _ in range(3):
        out = dsbcg.DSBCGSolve.apply(B, sig, U, dict(ARGS, context=c))
        torch.real(out.sum()).backward()
        del out
    with torch.no_grad():
        dsbcg.DSBCGSolve.apply(B, sig, U, dict(ARGS, context=c))
    gc.collect()
    assert fake.opened == 1 and fake.closed == 0 and c._ctx
