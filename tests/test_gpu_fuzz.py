"""Randomised configurations (seeded, so every run checks the same cases)
against the FP64 oracle: subgrid shapes, storage types, list kinds and
lengths (empty, ragged, single), tunings, summing arms and the compensated
form, forward and adjoint (GPU only).  Within one configuration every
summing arm must give the footprint-cache path's bits."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2102_12739_gb300 as dg  # noqa: E402
from paper_2102_12739_gb300 import synth  # noqa: E402
from tests.test_gpu_parity import G_UV, G_W, TOL, dev, rel_l2, small_workload, upload  # noqa: E402

pytestmark = pytest.mark.gpu

N_CASES = 64


def config(seed):
    rng = np.random.default_rng(1000 + seed)
    nz = int(rng.choice([4, 4, 5, 8]))
    shape = (int(rng.integers(16, 81)), int(rng.integers(16, 81)), nz)
    S = int(rng.integers(1, 7))
    counts = [int(rng.choice([0, 1, 31, 32, 33, int(rng.integers(2, 3000))])) for _ in range(S)]
    if sum(counts) == 0:
        counts[0] = 77
    return dict(shape=shape, counts=counts, kind=str(rng.choice(["line", "scatter", "mixed"])),
                dtype=str(rng.choice(["c64", "f16", "bf16"])), comp=bool(rng.integers(2)),
                chunk=int(rng.choice([32, 64, 96, 256, 1024])), warps=int(rng.choice([1, 2, 4, 8])),
                invalid=int(rng.integers(0, 3)), seed=seed)


@pytest.mark.parametrize("seed", range(N_CASES))
def test_random_configuration(seed):
    d = dev()
    c = config(seed)
    shape, counts = c["shape"], c["counts"]
    ny, nx, nz = shape
    w = small_workload(counts, kind=c["kind"], shape=shape, seed=200 + seed)
    rng = np.random.default_rng(2000 + seed)
    if nz > 4:                                     # use the whole w axis
        w.uvw[:, 2] = rng.uniform(1.0, nz - 3 - 1e-3, w.n_vis)
    for i in rng.choice(w.n_vis, min(c["invalid"], w.n_vis), replace=False):
        w.uvw[i] = [np.nan, 5.0, 1.5] if i % 2 else [nx + 10.0, 5.0, 1.5]
    sub_np = synth.subgrid_stack(len(counts), shape=shape, seed=seed)
    sub, uvw, offs = upload(w, sub_np)
    codes, scale = (sub, None) if c["dtype"] == "c64" else dg.pack_subgrids(sub, c["dtype"])
    ref, bad = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), w.uvw, w.vis_offsets)

    outs = {}
    with dg.DegridPlan(shape=shape, dtype=c["dtype"], device=d, compensated=c["comp"]) as p:
        p.set_tuning(c["chunk"], c["warps"], 0)
        outs["cache"] = p.degrid(codes, uvw, offs, scale=scale).cpu().numpy()
        assert p.status() == bad
        p.set_direct_runs(int(rng.integers(1, 33)))
        outs["direct"] = p.degrid(codes, uvw, offs, scale=scale).cpu().numpy()
        assert p.status() == bad
        p.set_direct_runs(dg._native.DG_DIRECT_RUNS_NEVER)
        if nz == 4:
            p.set_gather(True)
            outs["gather"] = p.degrid(codes, uvw, offs, scale=scale).cpu().numpy()
            assert p.status() == bad
    base = outs["cache"]
    for arm, o in outs.items():
        np.testing.assert_array_equal(o.view(np.uint32), base.view(np.uint32), err_msg=arm)
    assert rel_l2(base, ref) <= TOL[c["dtype"]], c

    # the adjoint of the same configuration (complex64 output), both kernels
    y = synth.adjoint_vis(w.n_vis, seed=3000 + seed)
    gref, _ = oracle.grid(G_UV, G_W, shape, len(counts), w.uvw, w.vis_offsets, y)
    yd = torch.from_numpy(y).to(d)
    for gather in ((False, True) if nz == 4 else (False,)):
        with dg.DegridPlan(shape=shape, device=d, gather=gather) as p:
            p.set_tuning(c["chunk"], c["warps"], 0)
            g = p.grid(yd, uvw, offs, len(counts)).cpu().numpy()
            assert p.status() == bad
        assert rel_l2(g, gref) <= TOL["c64"], (c, gather)
