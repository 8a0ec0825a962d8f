"""CUDA path vs the FP64 oracle, through the C ABI (GPU only).

Bar (from the method's statement of the target):
  * indices and GCF rows bit-exact;
  * complex64 subgrids: relative L2 error <= 2e-6 over all visibilities;
  * FP16 / BF16 subgrids: <= 1e-3 / <= 8e-3 against the oracle on the
    original complex64 subgrids (quantisation included).
Small cases are compared element by element; the full-size workloads run in
the launch configuration the benchmark times and are checked against the
oracle on every visibility (the oracle covers 16M visibilities in well under
a minute on the host cores).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2102_12739_gb300 as dg  # noqa: E402
from paper_2102_12739_gb300 import synth  # noqa: E402
from tests.test_oracle import load_coord_cases  # noqa: E402

pytestmark = pytest.mark.gpu

G_UV, G_W = synth.default_tables()
SHAPE = synth.SUBGRID_SHAPE
TOL = {"c64": 2e-6, "f16": 1e-3, "bf16": 8e-3}


def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch.device("cuda", 0)


@pytest.fixture(scope="module")
def plan():
    p = dg.DegridPlan(device=dev())
    yield p
    p.close()


def rel_l2(got, ref):
    ref = np.asarray(ref)
    den = np.linalg.norm(ref)
    return np.linalg.norm(np.asarray(got) - ref) / (den if den > 0 else 1.0)


def upload(w: synth.Workload, sub=None):
    d = dev()
    sub = w.subgrids() if sub is None else sub
    return (torch.from_numpy(np.ascontiguousarray(sub)).to(d),
            torch.from_numpy(w.uvw).to(d), torch.from_numpy(w.vis_offsets).to(d))


def small_workload(counts, kind="line", shape=SHAPE, seed=0):
    """Lines ("line"), scattered points ("scatter") or segments/arcs ("mixed")."""
    parts = []
    for s, c in enumerate(counts):
        rng = np.random.default_rng([100 + seed, s])
        if kind == "line":
            parts.append(synth.random_line(c, rng, shape))
        elif kind == "mixed":
            parts.append(synth.piecewise_list(c, rng, shape))
        else:
            ny, nx, _ = shape
            u = rng.uniform(*synth.uv_box(nx), c)
            v = rng.uniform(*synth.uv_box(ny), c)
            w = rng.uniform(synth.W_LO, synth.W_HI, c)
            parts.append(np.stack([u, v, w], axis=1))
    uvw = np.ascontiguousarray(np.concatenate(parts)) if parts else np.zeros((0, 3))
    return synth.Workload("small", len(counts), tuple(shape), uvw, synth.offsets_from_counts(counts))


def oracle_degrid_sample(w: synth.Workload, subgrids_of, idx):
    """Oracle values of visibilities `idx` (sorted global indices)."""
    idx = np.sort(np.asarray(idx))
    s_of = np.searchsorted(w.vis_offsets, idx, side="right") - 1
    subs = np.unique(s_of)
    sub = np.stack([subgrids_of(s).astype(np.complex128) for s in subs])
    counts = [(s_of == s).sum() for s in subs]
    ref, bad = oracle.degrid(G_UV, G_W, sub, w.uvw[idx], synth.offsets_from_counts(counts))
    return idx, ref


# ---------------------------------------------------------------------------
# coordinates: bit-exact
# ---------------------------------------------------------------------------

def test_coords_hand_cases(plan):
    uvw, expect = load_coord_cases()
    got = plan.coords(torch.from_numpy(uvw).to(dev())).cpu().numpy()
    np.testing.assert_array_equal(got, expect)
    assert plan.status() == int((expect[:, 0] < 0).sum())


def test_coords_random_and_ties_bit_exact(plan):
    rng = np.random.default_rng(5)
    n = 400_000
    u = rng.uniform(-20, 540, n)
    # exact ties k + 1/2 at the oversampled resolution, and their neighbours
    k = rng.integers(0, 512 * 16384, n // 4)
    u[: n // 4] = (k + 0.5) / 16384.0
    u[n // 4: n // 2] = np.nextafter((k + 0.5) / 16384.0, np.inf)
    v = rng.uniform(-20, 540, n)
    v[: n // 4] = (rng.integers(0, 512 * 16384, n // 4) + 0.5) / 16384.0
    w = rng.uniform(0.9, 2.1, n)
    w[: n // 4] = (rng.integers(100, 270, n // 4) + 0.5) / 128.0
    special = [np.nan, np.inf, -np.inf, 0.0, -0.0, 5e-324, 1e300, -1e300, 2.0 ** 48, 2.0 ** 49]
    u[-len(special):] = special
    uvw = np.stack([u, v, w], axis=1)
    want, bad = oracle.coords(uvw, SHAPE)
    got = plan.coords(torch.from_numpy(uvw).to(dev())).cpu().numpy()
    np.testing.assert_array_equal(got, want)
    assert plan.status() == bad


def test_coords_extreme_values_on_every_axis(plan):
    # the snap scales q by 2^k through q's exponent field: values whose
    # exponent the add carries past the largest (into the sign bit), values
    # at and just below 2^31 after scaling, the edges of the valid start
    # range and the smallest denormals, each on u, v and w in turn
    ny, nx, nz = SHAPE
    ext = [1.7976931348623157e308, -1.7976931348623157e308, 2.0 ** 1010, 1.5 * 2.0 ** 1009, 2.0 ** 1015,
           2.0 ** 1016, 1.9 * 2.0 ** 1016, 2.0 ** 1017, 2.0 ** 1020, -2.0 ** 1017, 2.0 ** 17, 2.0 ** 17 - 2.0 ** -15,
           2.0 ** 24, 2.0 ** 24 - 2.0 ** -8, 2.0 ** -1074, -2.0 ** -1074, 2.0 ** -1022, 1e-310]
    for n_ax, W, O in ((nx, 8, 16384), (ny, 8, 16384), (nz, 4, 128)):
        top = n_ax - W // 2                         # start = n - W just below q = top - 1/2 / O
        low = W // 2 - 1                            # start = 0 from q = low - 1/2 / O on
        ext += [top, top - 0.5 / O, np.nextafter(top - 0.5 / O, -np.inf), top + 0.5 / O,
                low - 0.5 / O, np.nextafter(low - 0.5 / O, np.inf), np.nextafter(low - 0.5 / O, -np.inf),
                low + 0.0, (2.0 ** 31 - 1) / O, 2.0 ** 31 / O, (2.0 ** 31 + 1) / O]
    ext = np.asarray(ext, dtype=np.float64)
    base = np.array([200.25, 300.75, 2.0])
    rows = []
    for axis in range(3):
        r = np.tile(base, (len(ext), 1))
        r[:, axis] = ext
        rows.append(r)
    uvw = np.ascontiguousarray(np.concatenate(rows, axis=0))
    want, bad = oracle.coords(uvw, SHAPE)
    got = plan.coords(torch.from_numpy(uvw).to(dev())).cpu().numpy()
    np.testing.assert_array_equal(got, want)
    assert plan.status() == bad
    assert 0 < bad < len(uvw)


def test_coords_of_full_lines_workload(plan):
    w = synth.workload("lines64_250k")
    got = plan.coords(torch.from_numpy(w.uvw).to(dev())).cpu().numpy()
    want, bad = oracle.coords(w.uvw, SHAPE)
    assert bad == 0
    np.testing.assert_array_equal(got, want)
    assert plan.status() == 0


# ---------------------------------------------------------------------------
# degridding values
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["line", "scatter", "mixed"])
def test_degrid_small_elementwise(plan, kind):
    # several chunks, a ragged tail, an empty subgrid, invalid visibilities
    w = small_workload([1000, 0, 777, 33], kind=kind)
    w.uvw[5] = [np.nan, 10.0, 1.5]
    w.uvw[1200] = [600.0, 10.0, 1.5]
    w.uvw[1776] = [20.0, 20.0, 0.2]
    sub_np = synth.subgrid_stack(4)
    sub, uvw, offs = upload(w, sub_np)
    got = plan.degrid(sub, uvw, offs).cpu().numpy()
    n_bad = plan.status()
    ref, bad = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), w.uvw, w.vis_offsets)
    assert n_bad == bad == 3
    assert got[5] == 0 and got[1200] == 0 and got[1776] == 0
    assert rel_l2(got, ref) <= TOL["c64"]


def test_degrid_line1_20k_full(plan):
    w = synth.workload("line1_20k")
    sub_np = synth.subgrid_stack(1)
    sub, uvw, offs = upload(w, sub_np)
    got = plan.degrid(sub, uvw, offs).cpu().numpy()
    ref, bad = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), w.uvw, w.vis_offsets)
    assert bad == 0 and plan.status() == 0
    assert rel_l2(got, ref) <= TOL["c64"]
    # every visibility individually close, relative to the footprint scale
    assert np.max(np.abs(got - ref)) <= 1e-5


def oracle_all(w: synth.Workload, subgrids_of, group=8):
    """Oracle values of every visibility of `w`, complex128 [N], computed a
    group of subgrids at a time (subgrids_of(s) gives subgrid s, any complex
    type, promoted exactly)."""
    out = np.empty(w.n_vis, dtype=np.complex128)
    for s0 in range(0, w.n_subgrids, group):
        s1 = min(s0 + group, w.n_subgrids)
        lo, hi = int(w.vis_offsets[s0]), int(w.vis_offsets[s1])
        if hi == lo:
            continue
        sub = np.stack([subgrids_of(s).astype(np.complex128) for s in range(s0, s1)])
        ref, bad = oracle.degrid(G_UV, G_W, sub, w.uvw[lo:hi], w.vis_offsets[s0:s1 + 1] - lo)
        assert bad == 0
        out[lo:hi] = ref
    return out


def test_degrid_lines64_full_size_every_visibility(plan):
    # the throughput workload in the benchmark's default launch configuration:
    # all 16M visibilities against the FP64 oracle
    w = synth.workload("lines64_250k")
    sub, uvw, offs = upload(w)
    got = plan.degrid(sub, uvw, offs).cpu().numpy()
    assert plan.status() == 0
    assert np.all(np.isfinite(got))
    ref = oracle_all(w, w.subgrid)
    assert rel_l2(got, ref) <= TOL["c64"]
    # and per subgrid, so that no list hides behind the others
    for s in range(w.n_subgrids):
        lo, hi = w.vis_offsets[s], w.vis_offsets[s + 1]
        assert rel_l2(got[lo:hi], ref[lo:hi]) <= TOL["c64"], s
    # every configuration the autotuner may pick for the benchmark gives
    # these bits, over all 16M visibilities
    from paper_2102_12739_gb300 import tune
    bits = torch.view_as_real(torch.from_numpy(got)).view(torch.int32).to(dev())
    with dg.DegridPlan(device=dev()) as p:
        for cand in tune.DEFAULT_CANDIDATES:
            tune._apply(p, dict(zip(tune._KEYS, cand)))
            o = p.degrid(sub, uvw, offs)
            assert p.status() == 0
            assert torch.equal(torch.view_as_real(o).view(torch.int32).flatten(), bits.flatten()), cand


def test_degrid_batched512_every_visibility(plan):
    # 512 subgrids with counts over three decades: all 72.8M visibilities
    # against the FP64 oracle
    w = synth.workload("batched512")
    d = dev()
    sub = torch.empty((w.n_subgrids,) + SHAPE, dtype=torch.complex64, device=d)
    for s in range(w.n_subgrids):
        sub[s].copy_(torch.from_numpy(w.subgrid(s)))
    uvw = torch.from_numpy(w.uvw).to(d)
    offs = torch.from_numpy(w.vis_offsets).to(d)
    got = plan.degrid(sub, uvw, offs).cpu().numpy()
    assert plan.status() == 0
    ref = oracle_all(w, w.subgrid, group=32)
    assert rel_l2(got, ref) <= TOL["c64"]
    per = [rel_l2(got[w.vis_offsets[s]:w.vis_offsets[s + 1]], ref[w.vis_offsets[s]:w.vis_offsets[s + 1]])
           for s in range(w.n_subgrids)]
    assert max(per) <= TOL["c64"], int(np.argmax(per))


def test_reduced_precision_full_size_every_visibility():
    # config 3: the 16M-visibility workload stored as FP16 and BF16 (one
    # scale per subgrid), plain and compensated reduction; every visibility
    # against the oracle on the original complex64 subgrids (quantisation
    # included, the stated bounds) and on the stored values (kernel error)
    d = dev()
    w = synth.workload("lines64_250k")
    sub_np = w.subgrids()
    sub = torch.from_numpy(sub_np).to(d)
    uvw = torch.from_numpy(w.uvw).to(d)
    offs = torch.from_numpy(w.vis_offsets).to(d)
    ref = oracle_all(w, lambda s: sub_np[s])
    for dt in ("f16", "bf16"):
        codes, scale = dg.pack_subgrids(sub, dt)
        want_codes, want_scale = oracle.quantize(sub_np, dt)
        np.testing.assert_array_equal(scale.cpu().numpy(), want_scale)
        np.testing.assert_array_equal(codes.view(torch.int16).cpu().numpy().view(np.uint16), want_codes)
        ref_q = oracle_all(w, lambda s: oracle.dequantize(want_codes[s:s + 1], want_scale[s:s + 1], dt)[0])
        for comp in (False, True):
            with dg.DegridPlan(dtype=dt, device=d, compensated=comp) as p:
                got = p.degrid(codes, uvw, offs, scale=scale).cpu().numpy()
                assert p.status() == 0
            assert rel_l2(got, ref) <= TOL[dt], (dt, comp, rel_l2(got, ref))
            assert rel_l2(got, ref_q) <= TOL["c64"], (dt, comp, rel_l2(got, ref_q))
        del codes, scale


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_reduced_precision_storage(dtype):
    d = dev()
    w = small_workload([3000, 1, 2500], kind="mixed", seed=3)
    sub_np = synth.subgrid_stack(3)
    sub_np[1] *= 1e-3                       # subgrids with different scales
    sub_c64 = torch.from_numpy(sub_np).to(d)
    codes, scale = dg.pack_subgrids(sub_c64, dtype)
    want_codes, want_scale = oracle.quantize(sub_np, dtype)
    np.testing.assert_array_equal(scale.cpu().numpy(), want_scale)
    got_codes = codes.view(torch.int16).cpu().numpy().view(np.uint16)
    np.testing.assert_array_equal(got_codes, want_codes)
    with dg.DegridPlan(dtype=dtype, device=d) as p:
        uvw = torch.from_numpy(w.uvw).to(d)
        offs = torch.from_numpy(w.vis_offsets).to(d)
        got = p.degrid(codes, uvw, offs, scale=scale).cpu().numpy()
    ref, _ = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), w.uvw, w.vis_offsets)
    assert rel_l2(got, ref) <= TOL[dtype]
    # against the oracle on the stored (dequantised) values: kernel error only
    deq = oracle.dequantize(want_codes, want_scale, dtype)
    ref_q, _ = oracle.degrid(G_UV, G_W, deq, w.uvw, w.vis_offsets)
    assert rel_l2(got, ref_q) <= 2e-6


@pytest.mark.parametrize("kind", ["scatter", "mixed", "line"])
def test_direct_arm_is_bitwise_the_cached_path(kind):
    # the direct (per-visibility) arm and the footprint-cache arm do the same
    # arithmetic in the same order: every threshold gives the same bits
    d = dev()
    w = small_workload([700, 0, 513, 64], kind=kind, seed=31)
    w.uvw[9] = [np.nan, 10.0, 1.5]
    sub_np = synth.subgrid_stack(4)
    sub, uvw, offs = upload(w, sub_np)
    outs = {}
    with dg.DegridPlan(device=d) as p:
        assert p.direct_runs == dg._native.DG_DIRECT_RUNS_DEFAULT
        for runs in (1, 2, 9, 33):
            p.set_direct_runs(runs)
            outs[runs] = p.degrid(sub, uvw, offs).cpu().numpy()
            assert p.status() == 1
        with pytest.raises(dg.DegridError):
            p.set_direct_runs(0)
    for runs in (2, 9, 33):
        np.testing.assert_array_equal(outs[1].view(np.uint32), outs[runs].view(np.uint32))
    ref, bad = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), w.uvw, w.vis_offsets)
    assert bad == 1 and outs[1][9] == 0
    assert rel_l2(outs[1], ref) <= TOL["c64"]


def test_host_memory_entry_point_matches_device_path():
    # several subgrid groups (64 MB of subgrids each: 8 subgrids of 8 MB), an
    # empty group in the middle, empty subgrids, invalid points; pinned and
    # pageable host buffers; bitwise the device path's result
    d = dev()
    counts = [300, 0, 150, 1, 0, 77, 500, 20, 0, 0, 0, 0, 0, 0, 0, 0, 64, 9, 200]
    w = small_workload(counts, kind="mixed", seed=61)
    w.uvw[2] = [np.nan, 10.0, 1.5]
    sub_np = synth.subgrid_stack(len(counts))
    sub, uvw, offs = upload(w, sub_np)
    with dg.DegridPlan(device=d) as p:
        ref = p.degrid(sub, uvw, offs).cpu().numpy()
        assert p.status() == 1
        h_sub = torch.from_numpy(sub_np).pin_memory()
        got = p.degrid_host(h_sub, torch.from_numpy(w.uvw).pin_memory(),
                            torch.from_numpy(w.vis_offsets).pin_memory()).numpy()
        assert p.status() == 1
        np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))
        again = p.degrid_host(sub_np, w.uvw, w.vis_offsets).numpy()     # pageable numpy
        np.testing.assert_array_equal(again.view(np.uint32), ref.view(np.uint32))
        assert p.status() == 1
        # pinned inputs with pageable output, and in-place access disabled:
        # both take the copy pipeline
        h_uvw = torch.from_numpy(w.uvw).pin_memory()
        mixed = p.degrid_host(h_sub, h_uvw, w.vis_offsets,
                              out=torch.empty(w.n_vis, dtype=torch.complex64)).numpy()
        np.testing.assert_array_equal(mixed.view(np.uint32), ref.view(np.uint32))
        assert p.host_direct
        p.set_host_direct(False)
        copied = p.degrid_host(h_sub, h_uvw, w.vis_offsets).numpy()
        np.testing.assert_array_equal(copied.view(np.uint32), ref.view(np.uint32))
        p.set_host_direct(True)
        assert p.status() == 2
        bad = w.vis_offsets.copy()
        bad[3] = bad[2] - 1                                              # decreasing
        with pytest.raises(dg.DegridError):
            p.degrid_host(sub_np, w.uvw, bad)
    with dg.DegridPlan(dtype="f16", device=d) as p16:
        codes, scale = dg.pack_subgrids(sub, "f16")
        ref16 = p16.degrid(codes, uvw, offs, scale=scale).cpu().numpy()
        got16 = p16.degrid_host(codes.cpu(), w.uvw, w.vis_offsets, scale=scale.cpu()).numpy()
        np.testing.assert_array_equal(got16.view(np.uint32), ref16.view(np.uint32))
        # in place, with pinned codes and coordinates; pageable then pinned scales
        for sc in (scale.cpu(), scale.cpu().pin_memory()):
            got16p = p16.degrid_host(codes.cpu().pin_memory(), h_uvw, w.vis_offsets, scale=sc).numpy()
            np.testing.assert_array_equal(got16p.view(np.uint32), ref16.view(np.uint32))


@pytest.mark.parametrize("dtype", ["c64", "f16", "bf16"])
def test_compensated_reduction(dtype):
    # the compensated form: same bar as the plain one, deterministic, and no
    # less accurate than the plain sum against the FP64 oracle
    d = dev()
    w = small_workload([2500, 0, 1900, 40], kind="mixed", seed=11)
    w.uvw[7] = [np.inf, 10.0, 1.5]
    w.uvw[3000] = [20.0, -4.0, 1.5]
    sub_np = synth.subgrid_stack(4)
    sub_c64 = torch.from_numpy(sub_np).to(d)
    if dtype == "c64":
        sub, scale, ref_sub = sub_c64, None, sub_np.astype(np.complex128)
    else:
        sub, scale = dg.pack_subgrids(sub_c64, dtype)
        codes, sc = oracle.quantize(sub_np, dtype)
        ref_sub = oracle.dequantize(codes, sc, dtype)
    uvw = torch.from_numpy(w.uvw).to(d)
    offs = torch.from_numpy(w.vis_offsets).to(d)
    with dg.DegridPlan(dtype=dtype, device=d) as plain, \
            dg.DegridPlan(dtype=dtype, device=d, compensated=True) as comp:
        assert comp.compensated and not plain.compensated
        got_p = plain.degrid(sub, uvw, offs, scale=scale).cpu().numpy()
        got_c = comp.degrid(sub, uvw, offs, scale=scale).cpu().numpy()
        assert comp.status() == 2           # the count is cleared when read
        again = comp.degrid(sub, uvw, offs, scale=scale).cpu().numpy()
        assert comp.status() == 2
    np.testing.assert_array_equal(got_c.view(np.uint32), again.view(np.uint32))
    assert got_c[7] == 0 and got_c[3000] == 0
    ref, bad = oracle.degrid(G_UV, G_W, ref_sub, w.uvw, w.vis_offsets)
    assert bad == 2
    # kernel error only (the oracle runs on the values the kernel reads)
    e_c, e_p = rel_l2(got_c, ref), rel_l2(got_p, ref)
    assert e_c <= 2e-6
    assert e_c <= 1.1 * e_p + 1e-9
    assert rel_l2(got_c, got_p) <= 1e-6


# ---------------------------------------------------------------------------
# non-separable G_uv (2D table)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["line", "scatter", "mixed"])
@pytest.mark.parametrize("dtype", ["c64", "bf16"])
def test_table2d_matches_oracle(kind, dtype):
    d = dev()
    G2 = synth.default_table_2d()
    w = small_workload([900, 0, 333, 41], kind=kind, seed=51)
    w.uvw[4] = [np.inf, 10.0, 1.5]
    sub_np = synth.subgrid_stack(4)
    sub_c64 = torch.from_numpy(sub_np).to(d)
    if dtype == "c64":
        sub, scale, ref_sub = sub_c64, None, sub_np.astype(np.complex128)
    else:
        sub, scale = dg.pack_subgrids(sub_c64, dtype)
        codes, sc = oracle.quantize(sub_np, dtype)
        ref_sub = oracle.dequantize(codes, sc, dtype)
    uvw = torch.from_numpy(w.uvw).to(d)
    offs = torch.from_numpy(w.vis_offsets).to(d)
    with dg.DegridPlan(dtype=dtype, device=d, g_uv2=G2) as p:
        assert p.table2d
        got = p.degrid(sub, uvw, offs, scale=scale).cpu().numpy()
        assert p.status() == 1
        # the coordinate step uses the 2D table's oversampling
        c, _ = oracle.coords(w.uvw, SHAPE, 8, G2.shape[0], 4, 128)
        np.testing.assert_array_equal(p.coords(uvw).cpu().numpy(), c)
    ref, bad = oracle.degrid_2d(G2, G_W, ref_sub, w.uvw, w.vis_offsets)
    assert bad == 1 and got[4] == 0
    assert rel_l2(got, ref) <= 2e-6       # kernel error (the oracle reads the stored values)


@pytest.mark.parametrize("kind", ["line", "scatter", "mixed"])
def test_table2d_adjoint_matches_oracle(kind):
    d = dev()
    shape = (40, 72, 4)
    rng = np.random.default_rng(53)
    G2 = rng.standard_normal((32, 32, 8, 8))          # a non-separable table
    w = small_workload([640, 0, 257, 33], kind=kind, shape=shape, seed=53)
    w.uvw[6] = [np.nan, 10.0, 1.5]
    y = synth.adjoint_vis(w.n_vis)
    uvw = torch.from_numpy(w.uvw).to(d)
    offs = torch.from_numpy(w.vis_offsets).to(d)
    sub_np = synth.subgrid_stack(4, shape)
    with dg.DegridPlan(shape=shape, device=d, g_uv2=G2) as p:
        got = p.grid(torch.from_numpy(y).to(d), uvw, offs, w.n_subgrids).cpu().numpy()
        assert p.status() == 1
        ds = p.degrid(torch.from_numpy(sub_np).to(d), uvw, offs).cpu().numpy()
        assert p.status() == 1
    ref, bad = oracle.grid_2d(G2, G_W, shape, w.n_subgrids, w.uvw, w.vis_offsets, y)
    assert bad == 1
    assert rel_l2(got, ref) <= TOL["c64"]
    # the GPU pair is an adjoint pair: <D s, y> = <s, G y>
    lhs = np.vdot(ds.astype(np.complex128), y.astype(np.complex128))
    rhs = np.vdot(sub_np.astype(np.complex128), got.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_table2d_separable_equals_separable_path():
    # G[fv][fu][b][a] = g[fv][b] g[fu][a]: the 2D path reproduces the
    # separable one to FP32 rounding
    d = dev()
    g = synth.gcf_table(8, 64, 2.3 * 8)
    G2 = g[:, None, :, None] * g[None, :, None, :]
    w = small_workload([1500, 700], kind="mixed", seed=52)
    sub, uvw, offs = upload(w, synth.subgrid_stack(2))
    with dg.DegridPlan(device=d, g_uv2=G2) as p2, dg.DegridPlan(device=d, g_uv=g) as p1:
        a = p2.degrid(sub, uvw, offs).cpu().numpy()
        b = p1.degrid(sub, uvw, offs).cpu().numpy()
    assert rel_l2(a, b) <= 1e-6


# ---------------------------------------------------------------------------
# adjoint and autograd
# ---------------------------------------------------------------------------

def test_adjoint_matches_oracle(plan):
    d = dev()
    shape = (64, 48, 4)
    w = small_workload([700, 0, 1500], kind="mixed", shape=shape, seed=9)
    y = synth.adjoint_vis(w.n_vis)
    with dg.DegridPlan(shape=shape, device=d) as p:
        got = p.grid(torch.from_numpy(y).to(d), torch.from_numpy(w.uvw).to(d),
                     torch.from_numpy(w.vis_offsets).to(d), w.n_subgrids).cpu().numpy()
        ref, _ = oracle.grid(G_UV, G_W, shape, w.n_subgrids, w.uvw, w.vis_offsets, y)
        assert rel_l2(got, ref) <= TOL["c64"]
        # accumulate mode adds to what is there
        base = torch.ones((w.n_subgrids,) + shape, dtype=torch.complex64, device=d)
        acc = p.grid(torch.from_numpy(y).to(d), torch.from_numpy(w.uvw).to(d),
                     torch.from_numpy(w.vis_offsets).to(d), w.n_subgrids, out=base,
                     accumulate=True).cpu().numpy()
        assert rel_l2(acc - 1, ref) <= TOL["c64"]


def test_adjoint_output_off_a_16_byte_boundary():
    # an output 8 bytes past a 16-byte boundary takes the float2 run-end adds
    # (the aligned nz = 4 output takes 16-byte vector reductions): both give
    # the oracle's gridding, in overwrite and in accumulate mode
    d = dev()
    shape = (64, 48, 4)
    w = small_workload([1800, 0, 900], kind="mixed", shape=shape, seed=19)
    y = torch.from_numpy(synth.adjoint_vis(w.n_vis)).to(d)
    uvw, offs = torch.from_numpy(w.uvw).to(d), torch.from_numpy(w.vis_offsets).to(d)
    ref, _ = oracle.grid(G_UV, G_W, shape, w.n_subgrids, w.uvw, w.vis_offsets, synth.adjoint_vis(w.n_vis))
    n = w.n_subgrids * int(np.prod(shape))
    buf = torch.full((n + 1,), float("nan"), dtype=torch.complex64, device=d)
    out = buf[1:].view((w.n_subgrids,) + shape)
    assert out.data_ptr() % 16 == 8
    with dg.DegridPlan(shape=shape, device=d) as p:
        got = p.grid(y, uvw, offs, w.n_subgrids, out=out).cpu().numpy()
        aligned = p.grid(y, uvw, offs, w.n_subgrids).cpu().numpy()
        out.fill_(1.0)
        acc = p.grid(y, uvw, offs, w.n_subgrids, out=out, accumulate=True).cpu().numpy()
        assert p.status() == 0
    assert rel_l2(got, ref) <= TOL["c64"]
    assert rel_l2(aligned, ref) <= TOL["c64"]
    assert rel_l2(acc - 1, ref) <= TOL["c64"]
    assert np.all(got[ref == 0] == 0)


@pytest.mark.parametrize("kind", ["line", "scatter", "mixed"])
def test_adjoint_all_list_kinds_with_invalid_points(kind):
    # runs of every length (scatter: a new footprint at nearly every
    # visibility), ragged batch tails, an empty subgrid, invalid points
    d = dev()
    shape = (40, 72, 4)
    w = small_workload([1033, 0, 64, 517], kind=kind, shape=shape, seed=21)
    w.uvw[3] = [np.nan, 10.0, 1.5]
    w.uvw[1040] = [20.0, 80.0, 1.5]
    w.uvw[1200] = [10.0, 10.0, 2.5]
    y = synth.adjoint_vis(w.n_vis)
    with dg.DegridPlan(shape=shape, device=d) as p:
        got = p.grid(torch.from_numpy(y).to(d), torch.from_numpy(w.uvw).to(d),
                     torch.from_numpy(w.vis_offsets).to(d), w.n_subgrids).cpu().numpy()
        assert p.status() == 3
    ref, bad = oracle.grid(G_UV, G_W, shape, w.n_subgrids, w.uvw, w.vis_offsets, y)
    assert bad == 3
    assert rel_l2(got, ref) <= TOL["c64"]
    assert np.all(got[1] == 0)                   # the empty subgrid stays zero


@pytest.mark.parametrize("shape,counts,kind", [
    ((16, 16, 4), [3000, 0, 2500, 0, 0, 800], "mixed"),     # zeroed in the kernel, empty subgrids
    ((512, 512, 4), [40000, 0], "line"),                     # most bands untouched
    ((40, 72, 4), [2000, 1, 0, 700], "scatter"),             # a new footprint at nearly every visibility
    ((512, 512, 4), [300, 0, 200, 0, 0, 0, 0, 9], "line"),   # fewer items than bands: memset first
])
def test_adjoint_overwrites_a_dirty_output(shape, counts, kind):
    # accumulate = 0 overwrites whatever the output held: every element is
    # the oracle's gridding, untouched ones exactly zero (the kernel zeroes
    # the stack band by band beside the sums, or a memset does when the call
    # has fewer work items than bands); twice in a row, and replayed from a
    # CUDA graph over a refilled output
    d = dev()
    w = small_workload(counts, kind=kind, shape=shape, seed=57)
    y = synth.adjoint_vis(w.n_vis, seed=58)
    ref, bad = oracle.grid(G_UV, G_W, shape, w.n_subgrids, w.uvw, w.vis_offsets, y)
    assert bad == 0
    yd = torch.from_numpy(y).to(d)
    uvw = torch.from_numpy(w.uvw).to(d)
    offs = torch.from_numpy(w.vis_offsets).to(d)
    out = torch.full((w.n_subgrids,) + shape, float("nan"), dtype=torch.complex64, device=d)
    zero = ref == 0
    with dg.DegridPlan(shape=shape, device=d) as p:
        for _ in range(2):
            out.fill_(float("nan"))
            got = p.grid(yd, uvw, offs, w.n_subgrids, out=out).cpu().numpy()
            assert p.status() == 0
            assert rel_l2(got, ref) <= TOL["c64"]
            assert np.all(got[zero] == 0)
        g = torch.cuda.CUDAGraph()
        st = torch.cuda.Stream(device=d)
        with torch.cuda.stream(st):
            with torch.cuda.graph(g, stream=st):
                p.grid(yd, uvw, offs, w.n_subgrids, out=out)
        for _ in range(2):
            out.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert rel_l2(got, ref) <= TOL["c64"]
            assert np.all(got[zero] == 0)
        assert p.status() == 0


def test_adjoint_dot_product_identity_on_gpu(plan):
    d = dev()
    w = synth.workload("line1_20k")
    sub_np = synth.subgrid_stack(1)
    sub, uvw, offs = upload(w, sub_np)
    y = synth.adjoint_vis(w.n_vis)
    ds = plan.degrid(sub, uvw, offs).cpu().numpy().astype(np.complex128)
    gy = plan.grid(torch.from_numpy(y).to(d), uvw, offs, 1).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(ds, y.astype(np.complex128))
    rhs = np.vdot(sub_np.astype(np.complex128), gy)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_autograd_gradient_is_adjoint_of_residual(plan):
    d = dev()
    w = small_workload([4000, 2000], kind="line", seed=11)
    sub_np = synth.subgrid_stack(2)
    y = synth.adjoint_vis(w.n_vis)
    sub = torch.from_numpy(sub_np).to(d).requires_grad_(True)
    uvw = torch.from_numpy(w.uvw).to(d)
    offs = torch.from_numpy(w.vis_offsets).to(d)
    vis = dg.DegridFn.apply(sub, uvw, offs, plan)
    loss = (vis - torch.from_numpy(y).to(d)).abs().pow(2).sum()
    loss.backward()
    got = sub.grad.cpu().numpy()
    ref_vis, _ = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), w.uvw, w.vis_offsets)
    ref, _ = oracle.grid(G_UV, G_W, SHAPE, 2, w.uvw, w.vis_offsets, 2 * (ref_vis - y))
    assert rel_l2(got, ref) <= 1e-5


# ---------------------------------------------------------------------------
# scheduler, edge cases, graphs
# ---------------------------------------------------------------------------

def test_tunings_give_bitwise_identical_results(plan):
    w = small_workload([5000, 255, 256, 257, 0, 1, 31, 33], kind="mixed", seed=12)
    sub, uvw, offs = upload(w, synth.subgrid_stack(8))
    outs = []
    saved = plan.tuning()
    try:
        for chunk, warps, bps in [(32, 1, 1), (256, 8, 0), (4096, 4, 2), (96, 2, 0)]:
            plan.set_tuning(chunk, warps, bps)
            outs.append(plan.degrid(sub, uvw, offs).cpu().numpy())
    finally:
        plan.set_tuning(saved["chunk"], saved["warps_per_block"], saved["blocks_per_sm"])
    for o in outs[1:]:
        np.testing.assert_array_equal(o.view(np.uint64), outs[0].view(np.uint64))


def test_one_subgrid_at_a_time_matches_batched(plan):
    w = small_workload([900, 2100, 64], kind="mixed", seed=13)
    sub_np = synth.subgrid_stack(3)
    sub, uvw, offs = upload(w, sub_np)
    batched = plan.degrid(sub, uvw, offs).cpu().numpy()
    d = dev()
    for s in range(3):
        lo, hi = w.vis_offsets[s], w.vis_offsets[s + 1]
        one = plan.degrid(sub[s:s + 1].contiguous(), uvw[lo:hi].contiguous(),
                          torch.tensor([0, hi - lo], dtype=torch.int64, device=d)).cpu().numpy()
        np.testing.assert_array_equal(one.view(np.uint64), batched[lo:hi].view(np.uint64))


def test_empty_and_degenerate_inputs(plan):
    d = dev()
    sub = torch.zeros((2,) + SHAPE, dtype=torch.complex64, device=d)
    uvw = torch.zeros((0, 3), dtype=torch.float64, device=d)
    offs = torch.zeros(3, dtype=torch.int64, device=d)
    assert plan.degrid(sub, uvw, offs).numel() == 0
    g = plan.grid(torch.zeros(0, dtype=torch.complex64, device=d), uvw, offs, 2)
    assert torch.count_nonzero(g).item() == 0
    # a single visibility
    w = small_workload([1], seed=14)
    sub_np = synth.subgrid_stack(1)
    s1, u1, o1 = upload(w, sub_np)
    got = plan.degrid(s1, u1, o1).cpu().numpy()
    ref, _ = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), w.uvw, w.vis_offsets)
    assert rel_l2(got, ref) <= TOL["c64"]
    assert plan.status() == 0


def test_malformed_offsets_are_reported(plan):
    d = dev()
    w = small_workload([100, 100], seed=15)
    sub, uvw, _ = upload(w, synth.subgrid_stack(2))
    bad = torch.tensor([0, 150, 120], dtype=torch.int64, device=d)   # ends short of N, decreasing
    plan.degrid(sub, uvw, torch.tensor([0, 150, 200], dtype=torch.int64, device=d))
    assert plan.status() == 0
    plan.degrid(sub, uvw, bad)
    with pytest.raises(dg.DegridError) as e:
        plan.status()
    assert e.value.status == dg.DG_ERR_OFFSETS
    assert plan.status() == 0      # cleared


def test_argument_errors_raise(plan):
    d = dev()
    sub = torch.zeros((1,) + SHAPE, dtype=torch.complex64, device=d)
    uvw = torch.zeros((4, 3), dtype=torch.float64, device=d)
    with pytest.raises((TypeError, ValueError)):
        plan.degrid(sub, uvw.float(), torch.tensor([0, 4], device=d))
    with pytest.raises((TypeError, ValueError)):
        plan.degrid(sub, uvw, torch.tensor([0, 4], dtype=torch.int64, device=d)[None])
    with dg.DegridPlan(dtype="bf16", device=d) as p:
        with pytest.raises(ValueError):
            p.degrid(torch.zeros((1,) + SHAPE + (2,), dtype=torch.bfloat16, device=d), uvw,
                     torch.tensor([0, 4], dtype=torch.int64, device=d))
    # outputs and inputs of the wrong size are refused on the host, before
    # anything is launched (a short buffer would be written past its end)
    offs = torch.tensor([0, 4], dtype=torch.int64, device=d)
    y = torch.zeros(4, dtype=torch.complex64, device=d)
    bad_calls = [
        lambda: plan.degrid(sub, uvw, offs, out=torch.empty(3, dtype=torch.complex64, device=d)),
        lambda: plan.degrid(sub, uvw, offs, out=torch.empty(4, dtype=torch.float32, device=d)),
        lambda: plan.grid(y, uvw, offs, 1, out=torch.empty((1, 8, 8, 4), dtype=torch.complex64, device=d)),
        lambda: plan.grid(y[:3], uvw, offs, 1),
        lambda: plan.coords(uvw, out=torch.empty((3, 6), dtype=torch.int32, device=d)),
        lambda: plan.coords(uvw, out=torch.empty((4, 6), dtype=torch.int64, device=d)),
        lambda: plan.coords(uvw.flatten()),
        lambda: plan.degrid_host(sub.cpu(), uvw.cpu(), offs.cpu(), out=torch.empty(3, dtype=torch.complex64)),
        lambda: dg.pack_subgrids(sub.real.contiguous(), "bf16"),
    ]
    for k, call in enumerate(bad_calls):
        with pytest.raises((TypeError, ValueError)):
            call()
    assert plan.status() == 0


def test_cuda_graph_replay_is_identical(plan):
    d = dev()
    w = small_workload([3000, 500, 4500], kind="mixed", seed=16)
    sub, uvw, offs = upload(w, synth.subgrid_stack(3))
    ref = plan.degrid(sub, uvw, offs)           # sizes the scratch before capture
    out = torch.empty_like(ref)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(device=d)
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.degrid(sub, uvw, offs, out=out)
    for _ in range(3):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out.view(torch.float32), ref.view(torch.float32))


def test_capture_of_a_smaller_call_that_halves_its_chunk():
    # a call sizes the plan's chunk table for every smaller call: after a
    # warm-up with N_big visibilities (chunk 256 kept), a call with fewer
    # visibilities that halves its chunk to 128, and so needs more items, is
    # captured in a CUDA graph without allocating, and replays bitwise
    import ctypes
    from paper_2102_12739_gb300 import _native
    d = dev()
    sms = torch.cuda.get_device_properties(d).multi_processor_count
    n_big = 512 * 16 * sms + 1000
    n_small = 512 * 16 * sms - 1000
    lib = _native.load()
    c, k = ctypes.c_int(), ctypes.c_int64()
    assert lib.degrid_schedule_reserve(sms, 256, 2, n_small, ctypes.byref(c), ctypes.byref(k)) == 0
    assert c.value == 128
    assert lib.degrid_schedule_reserve(sms, 256, 2, n_big, ctypes.byref(c), ctypes.byref(k)) == 0
    assert c.value == 256
    big = small_workload([n_big // 2, n_big - n_big // 2], kind="line", seed=41)
    small = small_workload([n_small // 2, n_small - n_small // 2], kind="line", seed=42)
    sub_np = synth.subgrid_stack(2)
    sub = torch.from_numpy(sub_np).to(d)
    y = torch.from_numpy(synth.adjoint_vis(n_small)).to(d)
    with dg.DegridPlan(device=d) as p:
        p.set_tuning(256, 8, 0)
        _, uvw_b, offs_b = upload(big, sub_np)
        p.degrid(sub, uvw_b, offs_b)                # warm-up at the largest size
        p.grid(torch.from_numpy(synth.adjoint_vis(n_big)).to(d), uvw_b, offs_b, 2)
        assert p.status() == 0
        _, uvw, offs = upload(small, sub_np)
        out = torch.empty(n_small, dtype=torch.complex64, device=d)
        gout = torch.empty((2,) + SHAPE, dtype=torch.complex64, device=d)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=d)
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                p.degrid(sub, uvw, offs, out=out)
                p.grid(y, uvw, offs, 2, out=gout)
        g.replay()
        torch.cuda.synchronize()
        assert p.status() == 0
        ref = p.degrid(sub, uvw, offs)
        gref = p.grid(y, uvw, offs, 2)
        assert torch.equal(out.view(torch.float32), ref.view(torch.float32))
        assert rel_l2(gout.cpu().numpy(), gref.cpu().numpy()) <= 1e-6   # float atomics: order varies
    want, _ = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), small.uvw, small.vis_offsets)
    assert rel_l2(out.cpu().numpy(), want) <= TOL["c64"]


def test_autotune_picks_a_candidate_and_caches_it(plan, tmp_path, monkeypatch):
    monkeypatch.setenv("DEGRID_TUNE_CACHE", str(tmp_path / "tune.json"))
    w = small_workload([6000, 3000], kind="line", seed=17)
    sub, uvw, offs = upload(w, synth.subgrid_stack(2))
    saved = plan.tuning()
    try:
        cands = [(128, 4, 0), (256, 8, 0, 9), (512, 8, 1)]
        res = dg.autotune(plan, sub, uvw, offs, candidates=cands, iters=2)
        assert not res["cached"] and len(res["timings"]) == 3
        assert plan.tuning() == res["tuning"]
        again = dg.autotune(plan, sub, uvw, offs, candidates=cands, iters=2)
        assert again["cached"] and again["tuning"] == res["tuning"]
        ref, _ = oracle.degrid(G_UV, G_W, synth.subgrid_stack(2).astype(np.complex128), w.uvw,
                               w.vis_offsets)
        assert rel_l2(plan.degrid(sub, uvw, offs).cpu().numpy(), ref) <= TOL["c64"]
    finally:
        plan.set_tuning(saved["chunk"], saved["warps_per_block"], saved["blocks_per_sm"])
        plan.set_direct_runs(saved["direct_runs"])


def test_adjoint_dense_lines_full_size_every_subgrid(plan):
    # the gridding workload at full size: 32 subgrids x 100,000 visibilities,
    # the whole output stack against the oracle's gridding (and per subgrid)
    d = dev()
    w = synth.workload("diff32_100k")
    y = synth.adjoint_vis(w.n_vis)
    g = plan.grid(torch.from_numpy(y).to(d), torch.from_numpy(w.uvw).to(d),
                  torch.from_numpy(w.vis_offsets).to(d), w.n_subgrids).cpu().numpy()
    assert plan.status() == 0
    ref, bad = oracle.grid(G_UV, G_W, SHAPE, w.n_subgrids, w.uvw, w.vis_offsets, y)
    assert bad == 0
    assert rel_l2(g, ref) <= TOL["c64"]
    for s in range(w.n_subgrids):
        assert rel_l2(g[s], ref[s]) <= TOL["c64"], s


def test_diff32_gradient_matches_fp64_central_differences():
    # 32 subgrids x 100,000 random-line visibilities, L = ||D s - y||^2: the
    # autograd gradient (the gridding kernel on 2 (D s - y), FP32) against
    # FP64 central differences of L taken with the oracle, on 64 entries that
    # footprints touch (real parts for even picks, imaginary parts for odd).
    # Only the visibilities whose footprint covers the perturbed entry change
    # L, so the difference is formed over those (every other term of L is
    # the same on both sides and cancels); L is quadratic, so the difference
    # is exact up to FP64 rounding for any step.  The bound is relative to
    # the sum of the magnitudes of the entry's gradient terms, the scale the
    # FP32 rounding of forward and gridding is relative to.
    d = dev()
    w = synth.workload("diff32_100k")
    sub_np = w.subgrids()
    sub = torch.from_numpy(sub_np).to(d)
    uvw = torch.from_numpy(w.uvw).to(d)
    offs = torch.from_numpy(w.vis_offsets).to(d)
    y_np = synth.adjoint_vis(w.n_vis)
    y = torch.from_numpy(y_np).to(d)
    with dg.DegridPlan(device=d) as p:
        s_req = sub.clone().requires_grad_(True)
        vis = dg.DegridFn.apply(s_req, uvw, offs, p)
        (vis - y).abs().pow(2).sum().backward()
        grad = s_req.grad.cpu().numpy()
        assert p.status() == 0

    rng = np.random.default_rng(29)
    picks = rng.choice(w.n_vis, 64, replace=False)
    cs, bad = oracle.coords(w.uvw, SHAPE)
    assert bad == 0
    h = 0.5
    worst = 0.0
    for k, i in enumerate(picks):
        s = int(np.searchsorted(w.vis_offsets, i, side="right") - 1)
        x0, y0, z0 = cs[i, 0], cs[i, 1], cs[i, 2]
        e = (int(y0 + rng.integers(8)), int(x0 + rng.integers(8)), int(z0 + rng.integers(4)))
        lo, hi = int(w.vis_offsets[s]), int(w.vis_offsets[s + 1])
        c = cs[lo:hi]
        cover = ((c[:, 1] <= e[0]) & (e[0] < c[:, 1] + 8) & (c[:, 0] <= e[1]) & (e[1] < c[:, 0] + 8) &
                 (c[:, 2] <= e[2]) & (e[2] < c[:, 2] + 4))
        A = lo + np.nonzero(cover)[0]
        assert A.size > 0
        step = h if k % 2 == 0 else 1j * h
        base = sub_np[s].astype(np.complex128)
        lp_lm = []
        for sign in (1, -1):
            pert = base.copy()
            pert[e] += sign * step
            v, _ = oracle.degrid(G_UV, G_W, pert[None], w.uvw[A], [0, A.size])
            r = v - y_np[A].astype(np.complex128)
            lp_lm.append(np.sum(r.real ** 2 + r.imag ** 2))
        fd = (lp_lm[0] - lp_lm[1]) / (2 * h)
        # the entry's weights d_i (degridding of a unit entry) and residuals r_i
        unit = np.zeros((1,) + SHAPE, dtype=np.complex128)
        unit[(0,) + e] = 1.0
        dw, _ = oracle.degrid(G_UV, G_W, unit, w.uvw[A], [0, A.size])
        r0, _ = oracle.degrid(G_UV, G_W, base[None], w.uvw[A], [0, A.size])
        r0 = r0 - y_np[A].astype(np.complex128)
        scale = float(np.sum(2 * np.abs(dw.real) * np.abs(r0)))
        g = grad[(s,) + e].real if k % 2 == 0 else grad[(s,) + e].imag
        worst = max(worst, abs(fd - g) / scale)
    assert worst <= 1e-5, worst


def test_many_subgrids_take_the_two_kernel_schedule():
    # more than 4096 subgrids: the scan and the chunk table are two kernels
    # (one block scans all counts) instead of one; small 16 x 16 x 4 subgrids,
    # ragged and empty lists, element by element against the oracle
    # (at chunk 128 the tiny lists form a sparse class claimed first and the
    # long ones stay dense; the long lists keep the call from halving its
    # chunk, as calls too small for two items per warp do)
    d = dev()
    shape = (16, 16, 4)
    rng = np.random.default_rng(71)
    counts = rng.integers(0, 24, 5000)
    counts[[0, 17, 4999]] = 0
    counts[[5, 2500, 4998]] = [400000, 300000, 17000]
    w = small_workload(list(counts), kind="scatter", shape=shape, seed=71)
    sub_np = synth.subgrid_stack(len(counts), shape=shape)
    sub, uvw, offs = upload(w, sub_np)
    ref, bad = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), w.uvw, w.vis_offsets)
    assert bad == 0
    outs = []
    with dg.DegridPlan(shape=shape, device=d) as p:
        for chunk in (32, 64, 128):
            p.set_tuning(chunk, 8, 0)
            got = p.degrid(sub, uvw, offs).cpu().numpy()
            assert p.status() == 0
            assert rel_l2(got, ref) <= TOL["c64"]
            outs.append(got)
    for o in outs[1:]:
        np.testing.assert_array_equal(o.view(np.uint64), outs[0].view(np.uint64))


@pytest.mark.parametrize("nz", [5, 8])
@pytest.mark.parametrize("dtype", ["c64", "f16", "bf16"])
def test_deep_w_axis_with_unaligned_footprints(nz, dtype):
    # nz > 4: a footprint starts at any z0 in [0, nz - 4], so its four w
    # samples are often not 16-byte aligned (the element-wise loads); planes
    # are not square.  A line whose w sweeps the whole axis (runs, and a
    # change of z0 inside runs of x, y) and scattered points; the direct arm
    # must give the cached path's bits, the adjoint the oracle's values.
    d = dev()
    shape = (40, 56, nz)
    ny, nx, _ = shape
    w = small_workload([1500, 0, 1200], kind="line", shape=shape, seed=80 + nz)
    rng = np.random.default_rng(90 + nz)
    w_hi = nz - 3 - 1e-3
    w.uvw[:1500, 2] = np.linspace(1.0, w_hi, 1500)
    w.uvw[1500:, 0] = rng.uniform(*synth.uv_box(nx), 1200)
    w.uvw[1500:, 1] = rng.uniform(*synth.uv_box(ny), 1200)
    w.uvw[1500:, 2] = rng.uniform(1.0, w_hi, 1200)
    c, bad = oracle.coords(w.uvw, shape)
    assert bad == 0 and len(np.unique(c[:, 2])) == nz - 3
    sub_np = synth.subgrid_stack(3, shape=shape)
    sub, uvw, offs = upload(w, sub_np)
    codes, scale = (sub, None) if dtype == "c64" else dg.pack_subgrids(sub, dtype)
    ref, _ = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), w.uvw, w.vis_offsets)
    with dg.DegridPlan(shape=shape, dtype=dtype, device=d) as p:
        got = p.degrid(codes, uvw, offs, scale=scale).cpu().numpy()
        p.set_direct_runs(1)
        direct = p.degrid(codes, uvw, offs, scale=scale).cpu().numpy()
        assert p.status() == 0
    assert rel_l2(got, ref) <= TOL[dtype]
    np.testing.assert_array_equal(direct.view(np.uint32), got.view(np.uint32))
    if dtype == "c64":
        y = synth.adjoint_vis(w.n_vis)
        with dg.DegridPlan(shape=shape, device=d) as p:
            g = p.grid(torch.from_numpy(y).to(d), uvw, offs, 3).cpu().numpy()
        gref, _ = oracle.grid(G_UV, G_W, shape, 3, w.uvw, w.vis_offsets, y)
        assert rel_l2(g, gref) <= TOL["c64"]


def test_two_plans_on_two_streams_in_flight_at_once():
    # one plan per stream (plans share no scratch): calls in flight on two
    # streams at once give the results of the same calls made one after the
    # other (bit for bit for the degridding)
    d = dev()
    wa = small_workload([3000, 0, 1200], kind="mixed", seed=91)
    wb = small_workload([500, 2500], kind="scatter", seed=92)
    sa, ua, oa = upload(wa, synth.subgrid_stack(3, seed=93))
    sb, ub, ob = upload(wb, synth.subgrid_stack(2, seed=94))
    ya = torch.from_numpy(synth.adjoint_vis(wa.n_vis, seed=95)).to(d)
    with dg.DegridPlan(device=d) as pa, dg.DegridPlan(device=d, gather=True) as pb:
        ref = [pa.degrid(sa, ua, oa), pb.degrid(sb, ub, ob), pa.grid(ya, ua, oa, 3)]
        torch.cuda.synchronize()
        s1, s2 = torch.cuda.Stream(d), torch.cuda.Stream(d)
        s1.wait_stream(torch.cuda.current_stream(d))
        s2.wait_stream(torch.cuda.current_stream(d))
        outs = []
        for _ in range(16):
            with torch.cuda.stream(s1):
                xa = pa.degrid(sa, ua, oa)
                ga = pa.grid(ya, ua, oa, 3)
            with torch.cuda.stream(s2):
                xb = pb.degrid(sb, ub, ob)
            outs.append((xa, xb, ga))
        torch.cuda.synchronize()
        assert pa.status() == 0 and pb.status() == 0
    gref = ref[2].cpu().numpy()
    for xa, xb, ga in outs:
        for g, r in ((xa, ref[0]), (xb, ref[1])):
            assert torch.equal(torch.view_as_real(g).view(torch.int32), torch.view_as_real(r).view(torch.int32))
        # the gridding adds with atomics: the order of the FP32 additions varies
        assert rel_l2(ga.cpu().numpy(), gref) <= 1e-6


def test_plans_of_different_sizes_from_several_host_threads():
    # plans are independent: four host threads, each with its own plan and
    # stream, CTAs of different sizes (so different shared-memory sizes of one
    # kernel instance) and one on the gather kernel, call at the same time;
    # every result matches the single-threaded one bit for bit
    import threading
    d = dev()
    w = small_workload([2000, 700, 0, 1500], kind="mixed", seed=97)
    sub, uvw, offs = upload(w, synth.subgrid_stack(4, seed=98))
    with dg.DegridPlan(device=d) as p0:
        ref = p0.degrid(sub, uvw, offs).cpu()
    torch.cuda.synchronize()
    errors, outs = [], {}

    def worker(tag, warps, gather):
        try:
            torch.cuda.set_device(d)
            s = torch.cuda.Stream(d)
            with dg.DegridPlan(device=d, gather=gather) as p, torch.cuda.stream(s):
                p.set_tuning(256, warps, 0)
                res = [p.degrid(sub, uvw, offs) for _ in range(20)]
                s.synchronize()
                assert p.status() == 0
                outs[tag] = [r.cpu() for r in res]
        except Exception as e:  # reported by the main thread
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(k, warps, gather))
               for k, (warps, gather) in enumerate([(2, False), (8, False), (4, False), (8, True)])]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert len(outs) == len(threads)
    for res in outs.values():
        for r in res:
            assert torch.equal(torch.view_as_real(r).view(torch.int32), torch.view_as_real(ref).view(torch.int32))


def test_sparse_and_dense_lists_at_every_chunk_size():
    # lists on both sides of each chunk size's sparse threshold (64 x chunk
    # visibilities: the sparse ones are cut into items of 64 and claimed
    # first), so every chunk size classes them differently; two long lists
    # keep the call large enough that no chunk size is halved.  The same bits
    # come out every time, and they match the oracle (sampled; the gridding
    # over the whole stack)
    d = dev()
    counts = [100, 1_500_000, 20000, 5000, 40000, 0, 300, 16383, 16384, 8191, 8192, 1, 1_000_000]
    w = small_workload(counts, kind="mixed", seed=99)
    sub_np = synth.subgrid_stack(len(counts), seed=100)
    sub, uvw, offs = upload(w, sub_np)
    outs = []
    with dg.DegridPlan(device=d) as p:
        # chunk 64: one class; 128, 256: thresholds 8192, 16384; 1024 is
        # halved to 512 for this call (threshold 32768)
        for chunk, warps in ((64, 8), (128, 4), (256, 8), (1024, 8), (256, 2)):
            p.set_tuning(chunk, warps, 0)
            o = p.degrid(sub, uvw, offs).cpu().numpy()
            assert p.status() == 0
            outs.append(o)
        p.set_tuning(256, 8, 0)
        yv = synth.adjoint_vis(w.n_vis, seed=101)
        g = p.grid(torch.from_numpy(yv).to(d), uvw, offs, len(counts)).cpu().numpy()
        assert p.status() == 0
    for o in outs[1:]:
        np.testing.assert_array_equal(o.view(np.uint64), outs[0].view(np.uint64))
    rng = np.random.default_rng(102)
    picks = []
    for s_ in range(len(counts)):
        lo, hi = w.vis_offsets[s_], w.vis_offsets[s_ + 1]
        if hi > lo:
            picks += [lo, hi - 1] + list(rng.integers(lo, hi, 300))
    idx, ref = oracle_degrid_sample(w, lambda s_: sub_np[s_], np.unique(picks))
    assert rel_l2(outs[0][idx], ref) <= TOL["c64"]
    gref, _ = oracle.grid(G_UV, G_W, synth.SUBGRID_SHAPE, len(counts), w.uvw, w.vis_offsets, yv)
    assert rel_l2(g, gref) <= TOL["c64"]
