"""Python binding of libdsbcg.so (C ABI in include/dsbcg.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the compiled library is missing, every call raises.

Entry points (same names as the C ABI):
  Context(dims, U, kappa)                  dsbcg_create / dsbcg_destroy
  Context.solve(B, sigma, tol, ...)        dsbcg_solve
  Context.solve_rational(B, sigma, ...)    dsbcg_solve_rational
  Context.backward(G, sigma, ...)          dsbcg_backward
  Context.apply(op, fields, ...)           dsbcg_apply
  Context.force(X, Lam, w, ...)            dsbcg_force
  DSBCGSolve, DSBCGRational                torch.autograd.Functions around
                                           solve / solve_rational and backward
"""
from __future__ import annotations

import ctypes
import os
import re
import weakref

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdsbcg.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "dsbcg.h")

PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3, "df32": 4}
OPS = {"D": 0, "Ddag": 1, "A": 2}
STATUS = {0: "OK", 1: "NOT_CONVERGED", -1: "ERR_ARG", -2: "ERR_NOT_HPD", -3: "ERR_CUDA",
          -4: "ERR_OOM", -5: "ERR_NONFINITE", -6: "ERR_UNSUPPORTED"}
KCLASS = ["dslash", "gram", "update", "shift", "small", "residual", "other", "unused"]


class DSBCGError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"dsbcg status {code} ({STATUS.get(code, '?')}): {msg}")


class Params(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("dtol", ctypes.c_double),
                ("max_block_steps", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("restart_drop", ctypes.c_double), ("poll_every", ctypes.c_int),
                ("freeze_converged", ctypes.c_int), ("refine", ctypes.c_int),
                ("fp64_residuals", ctypes.c_int), ("x0", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("block_steps", ctypes.c_int), ("mvms", ctypes.c_longlong),
                ("deflations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("final_rank", ctypes.c_int), ("seconds", ctypes.c_double),
                ("true_relres", ctypes.POINTER(ctypes.c_double)),
                ("conv_step", ctypes.POINTER(ctypes.c_int)),
                ("kernel_ms", ctypes.c_double * 8), ("kernel_launches", ctypes.c_longlong * 8),
                ("kernel_bytes", ctypes.c_double * 8), ("kernel_flops", ctypes.c_double * 8)]


_lib_handle = None


def lib():
    """Load libdsbcg.so; raise if it has not been built."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1205_0359_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.dsbcg_params_default.argtypes = [ctypes.POINTER(Params)]
    L.dsbcg_params_default.restype = None
    L.dsbcg_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), vp, dp, ip, vp]
    L.dsbcg_create.restype = ip
    L.dsbcg_update_gauge.argtypes = [vp, vp]
    L.dsbcg_update_gauge.restype = ip
    L.dsbcg_solve.argtypes = [vp, ip, vp, ip, ctypes.POINTER(ctypes.c_double), dp,
                              ctypes.POINTER(Params), vp, ctypes.POINTER(Stats)]
    L.dsbcg_solve.restype = ip
    L.dsbcg_apply.argtypes = [vp, ip, ip, ip, vp, vp]
    L.dsbcg_apply.restype = ip
    L.dsbcg_apply_static.argtypes = [vp, ip, ip, ip, vp, vp]
    L.dsbcg_apply_static.restype = ip
    L.dsbcg_force.argtypes = [vp, ip, ip, vp, vp, ctypes.POINTER(ctypes.c_double), ip, vp]
    L.dsbcg_force.restype = ip
    dpp = ctypes.POINTER(ctypes.c_double)
    L.dsbcg_solve_rational.argtypes = [vp, ip, vp, ip, dpp, dp, dpp, dp, ctypes.POINTER(Params), vp, vp,
                                       ctypes.POINTER(Stats)]
    L.dsbcg_solve_rational.restype = ip
    L.dsbcg_backward.argtypes = [vp, ip, vp, ip, dpp, vp, vp, dpp, dp, dp, ctypes.POINTER(Params), vp, dpp, vp,
                                 vp, ctypes.POINTER(Stats)]
    L.dsbcg_backward.restype = ip
    L.dsbcg_debug_first_wait.argtypes = [vp, ip]
    L.dsbcg_debug_first_wait.restype = ip
    L.dsbcg_debug_shift_chunk.argtypes = [vp, ip]
    L.dsbcg_debug_shift_chunk.restype = ip
    L.dsbcg_set_operator.argtypes = [vp, ip]
    L.dsbcg_set_operator.restype = ip
    L.dsbcg_set_profiling.argtypes = [vp, ip]
    L.dsbcg_set_profiling.restype = ip
    L.dsbcg_destroy.argtypes = [vp]
    L.dsbcg_destroy.restype = None
    L.dsbcg_error_string.argtypes = [ip]
    L.dsbcg_error_string.restype = ctypes.c_char_p
    L.dsbcg_version.argtypes = []
    L.dsbcg_version.restype = ctypes.c_char_p
    _lib_handle = L
    return L


def header_symbols(path: str = HEADER):
    """Function names declared in include/dsbcg.h."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dsbcg_[a-z_0-9]+)\s*\(", txt)))


def _check(code, what=""):
    if code not in (0, 1):
        raise DSBCGError(code, what + ": " + lib().dsbcg_error_string(code).decode())
    return code


def _ptr(t):
    """Device or host address of a contiguous complex128 tensor or numpy array."""
    if isinstance(t, torch.Tensor):
        assert t.is_contiguous(), "tensor must be contiguous"
        return ctypes.c_void_p(t.data_ptr())
    assert isinstance(t, np.ndarray) and t.flags.c_contiguous
    return ctypes.c_void_p(t.ctypes.data)


def _stream_handle(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream) if torch.cuda.is_available() else None
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """One lattice, gauge field and kappa (dsbcg_create).

    U: complex128 [Lt][Lz][Ly][Lx][4][3][3] (torch on CUDA or CPU, or numpy).
    """

    def __init__(self, dims, U, kappa, t_antiperiodic=True, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.kappa = float(kappa)
        self.V = int(np.prod(self.dims))
        self.n = 12 * self.V
        self._ctx = ctypes.c_void_p()
        self.stream = stream
        d = (ctypes.c_int * 4)(*self.dims)
        U = _as_c128(U)
        _check(lib().dsbcg_create(ctypes.byref(self._ctx), d, _ptr(U), self.kappa,
                                  int(bool(t_antiperiodic)), _stream_handle(stream)), "dsbcg_create")

    def close(self):
        if self._ctx:
            lib().dsbcg_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_operator(self, op):
        """dsbcg_set_operator: "normal" (A = D^H D, fields of n = 12 V) or
        "schur" (the even-odd operator Ahat on odd-site half fields, n = 6 V)."""
        code = {"normal": 0, "schur": 1}[op]
        _check(lib().dsbcg_set_operator(self._ctx, code), "dsbcg_set_operator")
        self.n = (12 if code == 0 else 6) * self.V
        self.operator = op

    def update_gauge(self, U):
        _check(lib().dsbcg_update_gauge(self._ctx, _ptr(_as_c128(U))), "dsbcg_update_gauge")

    def debug_first_wait(self, polls):
        """dsbcg_debug_first_wait (test hook): polls >= 0 makes the block
        Gram kernel's first wait give up after that many tests; -1 restores
        the normal limit."""
        _check(lib().dsbcg_debug_first_wait(self._ctx, int(polls)), "dsbcg_debug_first_wait")

    def debug_shift_chunk(self, steps):
        """dsbcg_debug_shift_chunk (test hook): caps the shift-update chunk
        at `steps` block steps (1..16); 0 restores the automatic length."""
        _check(lib().dsbcg_debug_shift_chunk(self._ctx, int(steps)), "dsbcg_debug_shift_chunk")

    def set_profiling(self, on=True):
        _check(lib().dsbcg_set_profiling(self._ctx, int(bool(on))), "dsbcg_set_profiling")

    def read_profile(self):
        """dsbcg_read_profile: {class: ms} and {class: launches} since the
        last read (or solve); resets them."""
        ms = (ctypes.c_double * 8)()
        nl = (ctypes.c_longlong * 8)()
        _check(lib().dsbcg_read_profile(self._ctx, ms, nl), "dsbcg_read_profile")
        return ({KCLASS[q]: ms[q] for q in range(7)}, {KCLASS[q]: nl[q] for q in range(7)})

    def solve(self, B, sigma, tol, storage="fp32", out=None, dtol=0.0, max_block_steps=None,
              max_restarts=None, restart_drop=None, poll_every=None, freeze=True, refine=True,
              fp64_residuals=True, x0=None, raise_on_error=True):
        """X (s, m, n) complex128 for (sigma_j + A) X_j = B; B (m, n) complex128.

        B and out may live on the GPU or on the host; the result has B's device.
        x0: optional initial guess (s, m, n) to resume from (dsbcg_params.x0).
        Returns (X, stats dict)."""
        B = _as_c128(B)
        m = B.shape[0]
        sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(-1))
        s = sig.size
        if out is None:
            if isinstance(B, torch.Tensor):
                out = torch.empty((s, m, self.n), dtype=torch.complex128, device=B.device)
            else:
                out = np.empty((s, m, self.n), dtype=np.complex128)
        p = make_params(storage, dtol, max_block_steps, max_restarts, restart_drop, poll_every, freeze,
                        refine, fp64_residuals)
        if x0 is not None:
            # initial guess (s, m, n): the solve resumes from it, in place in `out`
            if isinstance(out, torch.Tensor):
                if x0 is not out:
                    out.copy_(torch.as_tensor(x0).reshape(out.shape))
            else:
                out[...] = np.asarray(x0).reshape(out.shape)
            p.x0 = 1
        st, rel, conv = _new_stats(s, m)
        code = lib().dsbcg_solve(self._ctx, m, _ptr(B), s, _dptr(sig), float(tol),
                                 ctypes.byref(p), _ptr(out), ctypes.byref(st))
        if raise_on_error:
            _check(code, "dsbcg_solve")
        return out, _stats_dict(code, st, rel, conv)

    def solve_rational(self, B, sigma, alpha0, alpha, tol, storage="fp32", Y=None, X=None, raise_on_error=True,
                       **kw):
        """dsbcg_solve_rational: Y = alpha0 B + sum_j alpha_j (sigma_j + A)^{-1} B, shape (m, n).

        X: None (per-shift solutions not written) or an (s, m, n) output
        buffer.  Other keywords as solve().  Returns (Y, stats)."""
        B = _as_c128(B)
        m = B.shape[0]
        sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(-1))
        al = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).reshape(-1))
        assert al.size == sig.size, "one alpha_j per shift"
        s = sig.size
        if Y is None:
            Y = torch.empty_like(B) if isinstance(B, torch.Tensor) else np.empty_like(B)
        p = make_params(storage, **kw)
        st, rel, conv = _new_stats(s, m)
        code = lib().dsbcg_solve_rational(self._ctx, m, _ptr(B), s, _dptr(sig), float(alpha0), _dptr(al),
                                          float(tol), ctypes.byref(p), _ptr(Y),
                                          _ptr(X) if X is not None else None, ctypes.byref(st))
        if raise_on_error:
            _check(code, "dsbcg_solve_rational")
        return Y, _stats_dict(code, st, rel, conv)

    def backward(self, G, sigma, tol, X=None, B=None, g_weights=None, g_direct=0.0, storage="fp32",
                 want=("B", "sigma", "U"), Lambda=None, raise_on_error=True, **kw):
        """dsbcg_backward: gradients through X_j = (sigma_j + A)^{-1} B.

        G: (s, m, n) per-shift incoming gradients, or (m, n) with g_weights
        (G_j = g_weights[j] G: one joint solve; g_direct adds g_direct * G to
        dL/dB).  X: (s, m, n) solutions, or
        None to recompute them from B.  want: subset of {"B", "sigma", "U"}.
        Lambda: optional (s, m, n) output for the adjoint solutions.
        Returns (gB or None, gsigma (s,) numpy or None, gU or None, stats)."""
        G = _as_c128(G)
        sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(-1))
        s = sig.size
        m = G.shape[-2]
        if g_weights is None:
            assert G.ndim == 3 and G.shape[0] == s, "per-shift gradients G have shape (s, m, n)"
            wp = None
        else:
            assert G.ndim == 2, "shared gradient G has shape (m, n)"
            wv = np.ascontiguousarray(np.asarray(g_weights, dtype=np.float64).reshape(-1))
            assert wv.size == s
            wp = _dptr(wv)
        if X is not None:
            X = _as_c128(X)
        if B is not None:
            B = _as_c128(B)
        assert X is not None or B is not None, "backward needs X or B (to recompute X)"
        like = G
        mk = (lambda shape: torch.empty(shape, dtype=torch.complex128, device=like.device)) \
            if isinstance(like, torch.Tensor) else (lambda shape: np.empty(shape, dtype=np.complex128))
        gB = mk((m, self.n)) if "B" in want else None
        gsig = np.zeros(s, dtype=np.float64) if "sigma" in want else None
        gU = mk(self.dims[::-1] + (4, 3, 3)) if "U" in want else None
        p = make_params(storage, **kw)
        st, rel, conv = _new_stats(s, m)
        code = lib().dsbcg_backward(self._ctx, m, _ptr(B) if B is not None else None, s, _dptr(sig),
                                    _ptr(X) if X is not None else None, _ptr(G), wp, float(g_direct), float(tol),
                                    ctypes.byref(p),
                                    _ptr(gB) if gB is not None else None,
                                    _dptr(gsig) if gsig is not None else None,
                                    _ptr(gU) if gU is not None else None,
                                    _ptr(Lambda) if Lambda is not None else None, ctypes.byref(st))
        if raise_on_error:
            _check(code, "dsbcg_backward")
        return gB, gsig, gU, _stats_dict(code, st, rel, conv)

    def apply(self, op, fields, storage="fp64", out=None):
        """op(fields) for op in {"D", "Ddag", "A"}; fields (m, n) complex128."""
        fields = _as_c128(fields)
        if out is None:
            out = torch.empty_like(fields) if isinstance(fields, torch.Tensor) else np.empty_like(fields)
        m = fields.shape[0]
        _check(lib().dsbcg_apply(self._ctx, OPS[op], PREC[storage], m, _ptr(fields), _ptr(out)),
               "dsbcg_apply")
        return out

    def apply_static(self, op, fields, storage="fp64", out=None):
        """dsbcg_apply_static: op(fields) with no device allocation in the
        library; fields and out must be CUDA tensors (m, n) complex128."""
        fields = _as_c128(fields)
        if out is None:
            out = torch.empty_like(fields)
        _check(lib().dsbcg_apply_static(self._ctx, OPS[op], PREC[storage], fields.shape[0],
                                        _ptr(fields), _ptr(out)), "dsbcg_apply_static")
        return out

    def force(self, X, Lam, weights=None, storage="fp64", out=None):
        """Gauge-link gradient for solutions X and adjoint solutions Lam (s, m, n)."""
        X = _as_c128(X)
        Lam = _as_c128(Lam)
        s, m, _ = X.shape
        if out is None:
            shape = self.dims[::-1] + (4, 3, 3)
            if isinstance(X, torch.Tensor):
                out = torch.empty(shape, dtype=torch.complex128, device=X.device)
            else:
                out = np.empty(shape, dtype=np.complex128)
        w = None
        if weights is not None:
            w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
            wp = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        else:
            wp = None
        _check(lib().dsbcg_force(self._ctx, m, s, _ptr(X), _ptr(Lam), wp, PREC[storage], _ptr(out)),
               "dsbcg_force")
        return out


def make_params(storage="fp32", dtol=0.0, max_block_steps=None, max_restarts=None, restart_drop=None,
                poll_every=None, freeze=True, refine=True, fp64_residuals=True):
    """dsbcg_params from the library defaults and keyword overrides."""
    p = Params()
    lib().dsbcg_params_default(ctypes.byref(p))
    p.storage = PREC[storage] if isinstance(storage, str) else int(storage)
    p.dtol = float(dtol)
    if max_block_steps is not None:
        p.max_block_steps = int(max_block_steps)
    if max_restarts is not None:
        p.max_restarts = int(max_restarts)
    if restart_drop is not None:
        p.restart_drop = float(restart_drop)
    if poll_every is not None:
        p.poll_every = int(poll_every)
    p.freeze_converged = int(bool(freeze))
    p.refine = int(bool(refine))
    p.fp64_residuals = int(bool(fp64_residuals))
    return p


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _new_stats(s, m):
    rel = np.zeros((s, m), dtype=np.float64)
    conv = np.zeros((s, m), dtype=np.int32)
    st = Stats()
    st.true_relres = rel.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st.conv_step = conv.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    return st, rel, conv


def _stats_dict(code, st, rel, conv):
    return dict(status=STATUS.get(code, code), code=code, block_steps=st.block_steps,
                mvms=st.mvms, deflations=st.deflations, restarts=st.restarts,
                final_rank=st.final_rank, seconds=st.seconds, true_relres=rel, conv_step=conv,
                kernel_ms={KCLASS[q]: st.kernel_ms[q] for q in range(7)},
                kernel_launches={KCLASS[q]: st.kernel_launches[q] for q in range(7)},
                kernel_bytes={KCLASS[q]: st.kernel_bytes[q] for q in range(7)},
                kernel_flops={KCLASS[q]: st.kernel_flops[q] for q in range(7)})


def _as_c128(t):
    if isinstance(t, torch.Tensor):
        if t.dtype != torch.complex128:
            t = t.to(torch.complex128)
        return t.contiguous()
    return np.ascontiguousarray(np.asarray(t, dtype=np.complex128))


def _context_for(ctx, U, args):
    """The Context of one autograd node: the caller's (args["context"], never
    closed here) or a new one for U, closed when the node's graph is freed
    (weakref.finalize on the node), or right after forward when no input
    needs a gradient.  A retained graph (retain_graph=True) keeps it open, so
    backward can run more than once."""
    c = args.get("context")
    if c is not None:
        return c
    c = Context(args["dims"], U.detach(), args["kappa"])
    if not any(ctx.needs_input_grad):
        return _ClosingContext(c)
    try:
        weakref.finalize(ctx, c.close)
    except TypeError:            # node without weakref support: Context.__del__ closes it
        pass
    return c


class _ClosingContext:
    """Wraps a Context that is closed as soon as the forward has used it."""

    def __init__(self, c):
        self.c = c

    def __getattr__(self, name):
        return getattr(self.c, name)

    def done(self):
        self.c.close()


def _finish_forward(c):
    if isinstance(c, _ClosingContext):
        c.done()
        return None
    return c


class DSBCGSolve(torch.autograd.Function):
    """X = DSBCGSolve.apply(B, sigma, U, args) with X_j = (sigma_j + A(U))^{-1} B.

    B: (m, n) complex128 CUDA tensor; sigma: (s,) float64 tensor; U: gauge
    field complex128 (Lt, Lz, Ly, Lx, 4, 3, 3).  args: dict(dims, kappa, tol,
    storage="fp32", adj_tol=tol, context=None, recompute=False).
    * context: a caller-owned Context for U, reused across calls (no repacking
      of the links); otherwise one is created per forward (see _context_for).
    * recompute: keep only B for the backward and let dsbcg_backward solve for
      X again (memory instead of storage).
    The backward is one dsbcg_backward call: the adjoint systems
    (sigma_j + A) Lambda_j = dL/dX_j of all shifts in one library call, and
    dL/dB, dL/dsigma and dL/dU formed by the library's kernels.
    """

    @staticmethod
    def forward(ctx, B, sigma, U, args):
        c = _context_for(ctx, U, args)
        X, _ = c.solve(B.detach(), sigma.detach().cpu().numpy(), args["tol"], storage=args.get("storage", "fp32"))
        ctx.c = _finish_forward(c)
        ctx.args = args
        ctx.recompute = bool(args.get("recompute", False))
        ctx.save_for_backward(B if ctx.recompute else X, sigma)
        return X

    @staticmethod
    def backward(ctx, gX):
        saved, sigma = ctx.saved_tensors
        c, args = ctx.c, ctx.args
        want = tuple(k for k, need in zip(("B", "sigma", "U"), ctx.needs_input_grad[:3]) if need)
        kw = dict(X=saved) if not ctx.recompute else dict(B=saved.detach())
        gB, gsig, gU, _ = c.backward(gX.contiguous(), sigma.detach().cpu().numpy(),
                                     args.get("adj_tol", args["tol"]), storage=args.get("storage", "fp32"),
                                     want=want, **kw)
        gs = torch.from_numpy(gsig).to(device=sigma.device, dtype=sigma.dtype) if gsig is not None else None
        return gB, gs, gU, None


class DSBCGRational(torch.autograd.Function):
    """Y = DSBCGRational.apply(B, sigma, U, args) with
    Y = alpha0 B + sum_j alpha_j (sigma_j + A(U))^{-1} B (dsbcg_solve_rational),
    the rational-approximation use of the shifted solves (Sec. 1).

    args: as DSBCGSolve plus alpha0 (float) and alpha (s floats).  The
    incoming gradient dL/dY gives dL/dX_j = alpha_j dL/dY, so the backward's
    adjoint is ONE joint DSBlockCG solve of dL/dY for all shifts
    (dsbcg_backward with g_weights = alpha, g_direct = alpha0)."""

    @staticmethod
    def forward(ctx, B, sigma, U, args):
        c = _context_for(ctx, U, args)
        sig = sigma.detach().cpu().numpy()
        ctx.recompute = bool(args.get("recompute", False))
        X = None
        if not ctx.recompute:
            X = torch.empty((sig.size,) + tuple(B.shape), dtype=torch.complex128, device=B.device)
        Y, _ = c.solve_rational(B.detach(), sig, float(args["alpha0"]), args["alpha"], args["tol"],
                                storage=args.get("storage", "fp32"), X=X)
        ctx.c = _finish_forward(c)
        ctx.args = args
        ctx.save_for_backward(B if ctx.recompute else X, sigma)
        return Y

    @staticmethod
    def backward(ctx, gY):
        saved, sigma = ctx.saved_tensors
        c, args = ctx.c, ctx.args
        want = tuple(k for k, need in zip(("B", "sigma", "U"), ctx.needs_input_grad[:3]) if need)
        kw = dict(X=saved) if not ctx.recompute else dict(B=saved.detach())
        gB, gsig, gU, _ = c.backward(gY.contiguous(), sigma.detach().cpu().numpy(),
                                     args.get("adj_tol", args["tol"]), g_weights=args["alpha"],
                                     g_direct=float(args["alpha0"]), storage=args.get("storage", "fp32"),
                                     want=want, **kw)
        gs = torch.from_numpy(gsig).to(device=sigma.device, dtype=sigma.dtype) if gsig is not None else None
        return gB, gs, gU, None
