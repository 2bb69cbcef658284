"""GPU parity of the multi-RHS Wilson stencil (D, D^H, A) against the oracle.

Calls go through the C ABI (dsbcg_apply).  Lattices include an asymmetric
one with a ragged last CTA tile (2x4x6x5 = 240 sites, 7.5 tiles of 32) and
the L = 2 case where the forward and backward neighbours coincide.
"""
import numpy as np
import pytest
import torch

from oracle import wilson as W
from paper_1205_0359_gb300 import dsbcg, synth

pytestmark = pytest.mark.gpu

# df32: double-float pairs (48-bit significands), a few 2^-48 per operation
TOL = {"fp64": 1e-13, "df32": 5e-13, "fp32": 2e-6, "fp16": 4e-3, "bf16": 3e-2}


def _setup(dims, m, seed, eps=0.7, kappa=0.13):
    rng = np.random.Generator(np.random.PCG64(seed))
    U = synth.su3_links(dims, eps, rng)
    n = 12 * synth.volume(dims)
    F = synth.gaussian_rhs(n, m, rng)
    return U, F, kappa


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 5), (2, 2, 2, 2), (8, 4, 4, 6)])
@pytest.mark.parametrize("storage", ["fp64", "df32", "fp32", "fp16", "bf16"])
def test_operators_match_oracle(dims, storage):
    m = 5
    U, F, kappa = _setup(dims, m, 17)
    dev = torch.device("cuda")
    ctx = dsbcg.Context(dims, torch.from_numpy(U).to(dev), kappa)
    Ft = torch.from_numpy(F).to(dev)
    for op, ref in [("D", W.D_vec), ("Ddag", W.Ddag_vec), ("A", W.A_vec)]:
        got = ctx.apply(op, Ft, storage=storage).cpu().numpy()
        want = ref(U, kappa, dims, F)
        err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
        assert err.max() < TOL[storage], (op, storage, err.max())
    ctx.close()


def test_multi_rhs_equals_single_rhs_bitwise():
    dims = (4, 4, 4, 8)
    U, F, kappa = _setup(dims, 12, 5)
    dev = torch.device("cuda")
    ctx = dsbcg.Context(dims, torch.from_numpy(U).to(dev), kappa)
    Ft = torch.from_numpy(F).to(dev)
    for storage in ("fp64", "df32", "fp32"):
        many = ctx.apply("A", Ft, storage=storage)
        for i in (0, 7, 11):
            one = ctx.apply("A", Ft[i:i + 1].contiguous(), storage=storage)
            assert torch.equal(one[0], many[i])
    ctx.close()


def test_host_buffers_and_periodic_time():
    dims = (4, 2, 2, 4)
    U, F, kappa = _setup(dims, 2, 9)
    ctx = dsbcg.Context(dims, U, kappa, t_antiperiodic=False)   # numpy host inputs
    got = ctx.apply("D", F)
    # periodic time: the oracle's hop written out with no boundary sign
    Ff = W.to_field(F, dims)
    out = Ff.copy()
    for mu in range(4):
        ax = -3 - mu
        fwd = np.roll(Ff, -1, axis=ax)
        bwd = np.roll(Ff, 1, axis=ax)
        Uf = U[..., mu, :, :]
        Ub = np.conj(np.swapaxes(np.roll(Uf, 1, axis=-3 - mu), -1, -2))
        tf = np.einsum("...ab,...sb->...sa", Uf, fwd)
        tb = np.einsum("...ab,...sb->...sa", Ub, bwd)
        out -= kappa * (np.einsum("st,...tb->...sb", W.EYE4 - W.GAMMA[mu], tf)
                        + np.einsum("st,...tb->...sb", W.EYE4 + W.GAMMA[mu], tb))
    want = W.to_vector(out)
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))
    ctx.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_links_off_su3_use_full_storage(storage):
    """FP32 and 16-bit storages keep only rows 0 and 1 of each link when the
    gauge field is in SU(3) (row 2 = conj(row 0 x row 1) is rebuilt); a field
    off SU(3) by 1e-3 must fall back to all 9 entries and still match the
    oracle to the storage tolerance.  The same field projected back onto
    SU(3) then takes the 12-real path (also matched), and an update of the
    gauge field switches between the two."""
    dims = (4, 4, 4, 6)
    U, F, kappa = _setup(dims, 6, 23)
    rng = np.random.Generator(np.random.PCG64(24))
    Ubad = U + 1e-3 * (rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape))
    dev = torch.device("cuda")
    Ft = torch.from_numpy(F).to(dev)
    ctx = dsbcg.Context(dims, torch.from_numpy(Ubad).to(dev), kappa)
    try:
        for Ucur in (Ubad, U, Ubad):
            ctx.update_gauge(torch.from_numpy(Ucur).to(dev))
            for op, ref in [("D", W.D_vec), ("A", W.A_vec)]:
                got = ctx.apply(op, Ft, storage=storage).cpu().numpy()
                want = ref(Ucur, kappa, dims, F)
                err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
                assert err.max() < TOL[storage], (op, storage, err.max())
    finally:
        ctx.close()


@pytest.mark.parametrize("operator,per_apply", [("normal", 1), ("schur", 2)])
def test_stencil_bench_tool(capsys, operator, per_apply):
    """python -m paper_1205_0359_gb300.stencil_bench: one JSON line with the
    stencil's time and rate; D is one launch (two half-lattice passes for
    the Schur operator)."""
    import json
    from paper_1205_0359_gb300 import stencil_bench
    stencil_bench.main(["--lattice", "4,4,4,8", "--fields", "3", "--storage", "fp32", "--reps", "2",
                        "--operator", operator])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["stencil_launches_per_apply"] == per_apply
    assert line["ms_per_launch"] > 0 and line["GBps"] > 0 and 0 < line["frac_of_hbm"] < 2
