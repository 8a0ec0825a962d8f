"""Maximum sizes (GPU only): one call over more than 2^31 visibilities, and a
stack of more than 2^31 subgrid elements, through every summing arm, both
gridding kernels and 16-bit storage.  The inputs are generated on the device
(synth); the visibilities and subgrids each check needs are copied back and
handed to the FP64 oracle, value by value.  Skipped on devices without the
memory (about 100 GB and 50 GB free)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2102_12739_gb300 as dg  # noqa: E402
from paper_2102_12739_gb300 import synth  # noqa: E402
from tests.test_gpu_parity import G_UV, G_W, TOL, dev, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu

GIB = 1 << 30


def need_free(nbytes):
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info(dev())
    if free < nbytes:
        pytest.skip(f"needs {nbytes / GIB:.0f} GiB free on the device ({free / GIB:.0f} GiB free)")


def bits_equal(a, b):
    return torch.equal(torch.view_as_real(a).view(torch.int32), torch.view_as_real(b).view(torch.int32))


def test_more_than_2_31_visibilities_in_one_call():
    d = dev()
    # two dense lines of 2^30 visibilities and a scattered list that starts
    # below visibility 2^31 and ends above it: 2^31 + 2^26 + 6 in all
    counts = [1 << 30, (1 << 30) - 7, (1 << 26) + 13]
    n = sum(counts)
    assert n > (1 << 31)
    need_free(n * (24 + 8 + 8) + 8 * GIB)
    offs_np = synth.offsets_from_counts(counts)
    rng = np.random.default_rng(71)
    uvw = torch.empty((n, 3), dtype=torch.float64, device=d)
    synth.random_line_on_device(uvw, 0, counts[0], rng)
    synth.random_line_on_device(uvw, int(offs_np[1]), counts[1], rng)
    synth.fill_scattered_on_device(uvw, int(offs_np[2]), counts[2], seed=72)
    sub = synth.subgrid_stack_on_device(3, d, seed=73)
    offs = torch.from_numpy(offs_np).to(d)

    # checked visibilities: both ends, the subgrid boundaries, the 32-bit
    # boundary, and a random sample
    edges = [np.arange(0, 64), np.arange(n - 64, n), np.arange((1 << 31) - 96, (1 << 31) + 96)]
    edges += [np.arange(o - 40, o + 40) for o in offs_np[1:-1]]
    idx = np.unique(np.concatenate(edges + [rng.integers(0, n, 4000)]))
    idx_d = torch.from_numpy(idx).to(d)
    rows = uvw.index_select(0, idx_d).cpu().numpy()
    s_of = np.searchsorted(offs_np, idx, side="right") - 1
    sample_offs = synth.offsets_from_counts(np.bincount(s_of, minlength=3))
    sub_np = sub.cpu().numpy()
    ref, bad = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), rows, sample_offs)
    assert bad == 0

    with dg.DegridPlan(device=d) as p:
        out = p.degrid(sub, uvw, offs)
        assert p.status() == 0
        got = out.index_select(0, idx_d).cpu().numpy()
        assert rel_l2(got, ref) <= TOL["c64"]
        for arm in ("direct", "gather"):
            if arm == "direct":
                p.set_direct_runs(1)
            else:
                p.set_direct_runs(dg._native.DG_DIRECT_RUNS_NEVER)
                p.set_gather(True)
            other = p.degrid(sub, uvw, offs)
            assert p.status() == 0
            assert bits_equal(other, out), arm
            del other
    del out

    # 16-bit storage
    codes, scale = dg.pack_subgrids(sub, "bf16")
    with dg.DegridPlan(dtype="bf16", device=d) as p:
        out = p.degrid(codes, uvw, offs, scale=scale)
        assert p.status() == 0
        got = out.index_select(0, idx_d).cpu().numpy()
    assert rel_l2(got, ref) <= TOL["bf16"]
    del out

    # gridding: values only at the checked visibilities (zero elsewhere, which
    # adds exact zeros), so the whole output is the oracle's gridding of them
    yv = synth.adjoint_vis(len(idx), seed=74)
    y = torch.zeros(n, dtype=torch.complex64, device=d)
    y[idx_d] = torch.from_numpy(yv).to(d)
    gref, _ = oracle.grid(G_UV, G_W, synth.SUBGRID_SHAPE, 3, rows, sample_offs, yv)
    with dg.DegridPlan(device=d) as p:
        g = p.grid(y, uvw, offs, 3).cpu().numpy()
        assert p.status() == 0
    assert rel_l2(g, gref) <= TOL["c64"]


def test_stack_of_more_than_2_31_elements():
    d = dev()
    S = 2049                                        # 2049 x 2^20 elements > 2^31
    plane = int(np.prod(synth.SUBGRID_SHAPE))
    assert S * plane > (1 << 31)
    need_free(S * plane * (8 + 4 + 8) + 6 * GIB)
    sub = synth.subgrid_stack_on_device(S, d, seed=81)
    rng = np.random.default_rng(82)
    lists = {0: ("scatter", 700), 1023: ("line", 300), 2047: ("line", 1500), 2048: ("scatter", 2500)}
    keep = sorted(lists)
    parts = [synth.scattered_list(c, rng) if kind == "scatter" else synth.random_line(c, rng)
             for kind, c in (lists[s] for s in keep)]
    uvw_np = np.ascontiguousarray(np.concatenate(parts))
    counts = [lists[s][1] if s in lists else 0 for s in range(S)]
    uvw = torch.from_numpy(uvw_np).to(d)
    offs = torch.from_numpy(synth.offsets_from_counts(counts)).to(d)
    ref_offs = synth.offsets_from_counts([lists[s][1] for s in keep])
    sub_np = torch.stack([sub[s] for s in keep]).cpu().numpy()
    ref, bad = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), uvw_np, ref_offs)
    assert bad == 0

    for dtype in ("c64", "bf16"):
        codes, scale = (sub, None) if dtype == "c64" else dg.pack_subgrids(sub, dtype)
        outs = {}
        with dg.DegridPlan(dtype=dtype, device=d) as p:
            outs["cache"] = p.degrid(codes, uvw, offs, scale=scale)
            p.set_direct_runs(1)
            outs["direct"] = p.degrid(codes, uvw, offs, scale=scale)
            p.set_direct_runs(dg._native.DG_DIRECT_RUNS_NEVER)
            p.set_gather(True)
            outs["gather"] = p.degrid(codes, uvw, offs, scale=scale)
            assert p.status() == 0
        for arm, o in outs.items():
            assert bits_equal(o, outs["cache"]), (dtype, arm)
        assert rel_l2(outs["cache"].cpu().numpy(), ref) <= TOL[dtype], dtype
        del codes, scale, outs

    y = synth.adjoint_vis(len(uvw_np), seed=83)
    yd = torch.from_numpy(y).to(d)
    gref, _ = oracle.grid(G_UV, G_W, synth.SUBGRID_SHAPE, len(keep), uvw_np, ref_offs, y)
    for gather in (False, True):
        with dg.DegridPlan(device=d, gather=gather) as p:
            g = p.grid(yd, uvw, offs, S)
            assert p.status() == 0
        got = torch.stack([g[s] for s in keep]).cpu().numpy()
        assert rel_l2(got, gref) <= TOL["c64"], gather
        # every other subgrid of the 17 GB output is zero (cleared by the call)
        touched = torch.count_nonzero(torch.view_as_real(g).reshape(S, -1), dim=1).cpu().numpy()
        assert set(np.flatnonzero(touched)) == set(keep), gather
        del g
