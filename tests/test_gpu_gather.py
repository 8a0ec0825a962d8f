"""The gather kernel (every footprint streamed through shared memory) against
the FP64 oracle and, bit for bit, against the footprint-cache kernel: both do
the same arithmetic in the same order (GPU only)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2102_12739_gb300 as dg  # noqa: E402
from paper_2102_12739_gb300 import synth  # noqa: E402
from tests.test_gpu_parity import (G_UV, G_W, TOL, dev, oracle_all, rel_l2,  # noqa: E402
                                   small_workload, upload)

pytestmark = pytest.mark.gpu


def bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


def degrid_both(dtype, comp, sub, uvw, offs, chunk=256):
    """(footprint-cache result, gather result, their status counts)."""
    codes, scale = (sub, None) if dtype == "c64" else dg.pack_subgrids(sub, dtype)
    outs, stats = [], []
    for gather in (False, True):
        with dg.DegridPlan(dtype=dtype, device=sub.device, compensated=comp, gather=gather) as p:
            p.set_tuning(chunk, 8, 0)
            assert p.gather == gather
            outs.append(p.degrid(codes, uvw, offs, scale=scale).cpu().numpy())
            stats.append(p.status())
    return outs[0], outs[1], stats


@pytest.mark.parametrize("comp", [False, True])
@pytest.mark.parametrize("dtype", ["c64", "f16", "bf16"])
@pytest.mark.parametrize("kind", ["scatter", "mixed", "line"])
def test_gather_matches_oracle_and_the_cached_path_bitwise(kind, dtype, comp):
    d = dev()
    # ragged lists: an empty one, 513 = 16 x 32 + 1, 3 (< one stage of 4)
    w = small_workload([700, 0, 513, 64, 3], kind=kind, seed=41)
    w.uvw[9] = [np.nan, 10.0, 1.5]
    w.uvw[-1] = [600.0, 10.0, 1.5]                 # outside the subgrid
    sub_np = synth.subgrid_stack(5)
    sub, uvw, offs = upload(w, sub_np)
    cached, gathered, stats = degrid_both(dtype, comp, sub, uvw, offs)
    assert stats == [2, 2]
    np.testing.assert_array_equal(bits(cached), bits(gathered))
    assert gathered[9] == 0 and gathered[-1] == 0
    ref, bad = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), w.uvw, w.vis_offsets)
    assert bad == 2
    assert rel_l2(gathered, ref) <= TOL[dtype]


def test_gather_chunk_sizes_give_the_same_bits():
    d = dev()
    w = small_workload([1000, 37, 0, 2049], kind="scatter", seed=43)
    sub_np = synth.subgrid_stack(4)
    sub, uvw, offs = upload(w, sub_np)
    outs = []
    with dg.DegridPlan(device=d, gather=True) as p:
        for chunk in (32, 64, 256, 1024):
            p.set_tuning(chunk, 8, 0)
            outs.append(p.degrid(sub, uvw, offs).cpu().numpy())
        assert p.status() == 0
    for o in outs[1:]:
        np.testing.assert_array_equal(bits(outs[0]), bits(o))


def test_gather_full_size_scattered_workload_every_visibility():
    # 16 subgrids x 250,000 scattered visibilities, the launch configuration
    # the benchmark times for this workload; every visibility against the
    # oracle and bitwise against the footprint-cache kernel
    d = dev()
    w = synth.workload("scatter16_250k")
    sub_np = w.subgrids()
    sub, uvw, offs = upload(w, sub_np)
    ref = oracle_all(w, lambda s: sub_np[s])
    for dtype in ("c64", "bf16"):
        cached, gathered, stats = degrid_both(dtype, False, sub, uvw, offs, chunk=256)
        assert stats == [0, 0]
        np.testing.assert_array_equal(bits(cached), bits(gathered))
        assert rel_l2(gathered, ref) <= TOL[dtype]


def test_gather_host_entry_point_and_graph_capture():
    d = dev()
    w = small_workload([300, 0, 150, 77], kind="scatter", seed=47)
    sub_np = synth.subgrid_stack(4)
    sub, uvw, offs = upload(w, sub_np)
    with dg.DegridPlan(device=d, gather=True) as p:
        ref = p.degrid(sub, uvw, offs).cpu().numpy()
        host = p.degrid_host(sub_np, w.uvw, w.vis_offsets).numpy()
        np.testing.assert_array_equal(bits(host), bits(ref))
        out = torch.empty(w.n_vis, dtype=torch.complex64, device=d)
        s = torch.cuda.Stream(d)
        with torch.cuda.stream(s):
            p.degrid(sub, uvw, offs, out=out)       # sizes the scratch before capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            p.degrid(sub, uvw, offs, out=out)
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(bits(out.cpu().numpy()), bits(ref))
        assert p.status() == 0


def test_gather_is_refused_where_it_cannot_run():
    d = dev()
    with dg.DegridPlan(device=d, g_uv2=synth.default_table_2d()) as p2:
        with pytest.raises(dg.DegridError):
            p2.set_gather(True)
        assert not p2.gather
    with dg.DegridPlan(shape=(64, 64, 8), device=d) as p8:
        with pytest.raises(dg.DegridError):
            p8.set_gather(True)
        p8.set_gather(False)
    with dg.DegridPlan(device=d) as p:
        assert dg.load().degrid_plan_set_gather(p.handle, 2) == dg._native.DG_ERR_ARG
        v = ctypes.c_int(-1)
        assert dg.load().degrid_plan_get_gather(p.handle, ctypes.byref(v)) == 0 and v.value == 0


@pytest.mark.parametrize("kind", ["scatter", "mixed", "line"])
def test_scatter_gridding_matches_oracle(kind):
    # the adjoint with the plan's gather setting: one tensor reduce-add per
    # visibility; ragged lists, an empty subgrid, invalid points, accumulate
    d = dev()
    w = small_workload([1500, 0, 513, 64, 3], kind=kind, seed=61)
    w.uvw[9] = [np.nan, 10.0, 1.5]
    w.uvw[-1] = [600.0, 10.0, 1.5]
    y = synth.adjoint_vis(w.n_vis)
    uvw = torch.from_numpy(w.uvw).to(d)
    offs = torch.from_numpy(w.vis_offsets).to(d)
    yd = torch.from_numpy(y).to(d)
    ref, bad = oracle.grid(G_UV, G_W, synth.SUBGRID_SHAPE, 5, w.uvw, w.vis_offsets, y)
    assert bad == 2
    with dg.DegridPlan(device=d, gather=True) as p:
        got = p.grid(yd, uvw, offs, 5).cpu().numpy()
        assert p.status() == 2
        assert rel_l2(got, ref) <= TOL["c64"]
        assert np.all(got[1] == 0)
        base = torch.ones((5,) + synth.SUBGRID_SHAPE, dtype=torch.complex64, device=d)
        acc = p.grid(yd, uvw, offs, 5, out=base, accumulate=True).cpu().numpy()
        assert p.status() == 2
        assert rel_l2(acc - 1, ref) <= TOL["c64"]
    with dg.DegridPlan(device=d) as p0:             # the run-accumulating kernel agrees
        other = p0.grid(yd, uvw, offs, 5).cpu().numpy()
    assert rel_l2(got, other) <= 1e-6


def test_scatter_gridding_full_size_and_dot_product():
    # 16 subgrids x 250,000 scattered visibilities: the whole gridded stack
    # against the oracle, and <D s, y> = <s, G y> with both directions on the
    # gather kernels
    d = dev()
    w = synth.workload("scatter16_250k")
    sub_np = w.subgrids()
    sub, uvw, offs = upload(w, sub_np)
    y = synth.adjoint_vis(w.n_vis)
    yd = torch.from_numpy(y).to(d)
    with dg.DegridPlan(device=d, gather=True) as p:
        g = p.grid(yd, uvw, offs, w.n_subgrids)
        dvis = p.degrid(sub, uvw, offs)
        assert p.status() == 0
        lhs = torch.vdot(dvis.to(torch.complex128), yd.to(torch.complex128)).item()
        rhs = torch.vdot(sub.to(torch.complex128).flatten(), g.to(torch.complex128).flatten()).item()
        gnp = g.cpu().numpy()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    ref, _ = oracle.grid(G_UV, G_W, synth.SUBGRID_SHAPE, w.n_subgrids, w.uvw, w.vis_offsets, y)
    assert rel_l2(gnp, ref) <= TOL["c64"]
