"""dsbcg_apply_static: the operator application with no device allocation.

Some callers cannot call cudaMalloc when they apply the operator (a memory
pool that already owns the whole GPU, or a latency-critical loop that cannot
afford cudaMalloc's implicit synchronisation).  dsbcg_apply_static keeps its
working fields in the library's static device array instead.  Its results
must equal those of dsbcg_apply, call after call, although every call reuses
the same array.  The calls go through the C ABI.  This file is collected last
so that a run stopping at the first failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1205_0359_gb300 import dsbcg, synth

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-13, "fp32": 2e-6}


@pytest.fixture(scope="module")
def ctx():
    dims = (4, 4, 4, 6)
    rng = np.random.Generator(np.random.PCG64(2024))
    U = synth.su3_links(dims, 0.6, rng)
    c = dsbcg.Context(dims, torch.from_numpy(U).cuda(), 0.13)
    yield c, dims, rng
    c.close()


def _call(c, op, storage, F):
    out = torch.empty_like(F)
    code = dsbcg.lib().dsbcg_apply_static(c._ctx, dsbcg.OPS[op], dsbcg.PREC[storage], F.shape[0],
                                          ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(out.data_ptr()))
    return code, out


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_matches_dsbcg_apply_two_calls_in_a_row(ctx, storage):
    c, dims, rng = ctx
    n = 12 * synth.volume(dims)
    c.apply("D", torch.zeros((1, n), dtype=torch.complex128, device="cuda"), storage=storage)  # packs links
    for call, m in enumerate((5, 3)):
        F = torch.from_numpy(synth.gaussian_rhs(n, m, rng)).cuda()
        for op in ("D", "Ddag", "A"):
            code, got = _call(c, op, storage, F)
            assert code == 0, (call, op, code)
            want = c.apply(op, F, storage=storage)
            err = (torch.linalg.norm(got - want, dim=1) / torch.linalg.norm(want, dim=1)).max().item()
            assert err <= TOL[storage], (call, op, err)


def test_rejects_sizes_beyond_the_static_array(ctx):
    c, dims, rng = ctx
    n = 12 * synth.volume(dims)
    ld = (n + 127) // 128 * 128
    m_big = (32 << 20) // (3 * 16 * ld) + 1
    F = torch.zeros((m_big, n), dtype=torch.complex128, device="cuda")
    code, _ = _call(c, "A", "fp64", F)
    assert code == -1
    code, out = _call(c, "A", "fp64", F[:2].contiguous())
    assert code == 0
