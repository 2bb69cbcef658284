"""The failure path of the kernels' bounded shared-memory waits, taken
without any GPU fault.

dsbcg_debug_first_wait(ctx, 0) makes the first wait of every consumer warp
of the staged block Gram kernel give up at once.  The kernel then drains
its own bulk copies (the producer's waits keep their normal limit and stop
waiting for buffers the consumers abandoned), records the timeout in the
solve's control block and returns.  The solve reports DSBCG_ERR_CUDA, the
CUDA context stays usable, the context can be destroyed, and a new context
solves correctly.
"""
import numpy as np
import pytest
import torch

from paper_1205_0359_gb300 import dsbcg, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
def test_gram_wait_timeout_reports_error(storage):
    wl = synth.make_workload("w1_4x4x4x4")
    U = torch.from_numpy(wl["U"]).to(DEV)
    B = torch.from_numpy(wl["B"]).to(DEV)
    ctx = dsbcg.Context(wl["dims"], U, wl["kappa"])
    ctx.debug_first_wait(0)
    with pytest.raises(dsbcg.DSBCGError) as e:
        ctx.solve(B, wl["sigma"], 1e-10, storage=storage)
    assert e.value.code == -3                         # DSBCG_ERR_CUDA
    torch.cuda.synchronize()                          # no sticky CUDA error
    ctx.close()
    ctx = dsbcg.Context(wl["dims"], U, wl["kappa"])
    try:
        X, st = ctx.solve(B, wl["sigma"], 1e-10, storage=storage)
        assert st["code"] == 0 and st["true_relres"].max() <= 1e-10
        assert bool(torch.isfinite(X).all())
    finally:
        ctx.close()


def test_hook_off_restores_normal_waits():
    wl = synth.make_workload("w1_4x4x4x4")
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(DEV), wl["kappa"])
    try:
        ctx.debug_first_wait(0)
        ctx.debug_first_wait(-1)
        X, st = ctx.solve(torch.from_numpy(wl["B"]).to(DEV), wl["sigma"], 1e-10, storage="fp64")
        assert st["code"] == 0
        assert np.isfinite(st["true_relres"]).all()
    finally:
        ctx.close()
