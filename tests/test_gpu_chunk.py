"""The chunked shift update against the per-step one.

The per-shift recurrences X_j += P_j Ut_j, P_j <- V_{k+1} - P_j Lh_j (Sec. 3)
run in the library over chunks of up to 16 block steps, with P_j and X_j
held on chip and the chunk's basis blocks in a ring.  Per element the
operations and their order are those of one launch per step, so every
chunk length gives bitwise the same solutions, residuals and step counts.
dsbcg_debug_shift_chunk caps the chunk length: 1 (one launch per step), 3
(chunks that do not divide the 16-step batches) and 16 are compared on the
4^4 workload, whose fourth right-hand side is b_1 + b_2, so the block width
drops from 4 to 3 at the first step and the chunks cross a deflation.  The
joint solve, the early hand-off of frozen shifts and the restarts all run
through the same kernel.
"""
import numpy as np
import pytest
import torch

from paper_1205_0359_gb300 import dsbcg, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


@pytest.mark.parametrize("storage", ["fp32", "bf16", "fp64"])
def test_chunk_lengths_give_bitwise_equal_solutions(storage):
    wl = synth.make_workload("w1_4x4x4x4")
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(DEV), wl["kappa"])
    B = torch.from_numpy(wl["B"]).to(DEV)
    runs = {}
    try:
        for steps in (1, 3, 16, 0):
            ctx.debug_shift_chunk(steps)
            runs[steps] = ctx.solve(B, wl["sigma"], 1e-10, storage=storage)
    finally:
        ctx.close()
    X1, st1 = runs[1]
    assert st1["code"] == 0 and st1["true_relres"].max() <= 1e-10
    assert st1["deflations"] >= 1
    for steps in (3, 16, 0):
        X, st = runs[steps]
        assert torch.equal(X, X1), steps
        assert np.array_equal(st["true_relres"], st1["true_relres"]), steps
        assert st["block_steps"] == st1["block_steps"] and st["restarts"] == st1["restarts"], steps


def test_chunk_hook_rejects_lengths_out_of_range():
    wl = synth.make_workload("w1_4x4x4x4")
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(DEV), wl["kappa"])
    try:
        for bad in (-1, 17):
            with pytest.raises(dsbcg.DSBCGError) as e:
                ctx.debug_shift_chunk(bad)
            assert e.value.code == -1
    finally:
        ctx.close()
