"""degrid_execute_noalloc against degrid_execute (GPU only).

degrid_execute_noalloc serves callers that cannot allocate device memory
once they are running (real-time pipelines that must stay out of the CUDA
allocator, hosts whose device memory belongs to another allocator).  It takes
no plan and draws all its scratch from one fixed array inside the library, so
two things need checking: that it computes what the plan-based call
computes, and that the array's leftovers from one call do not leak into the
next.  Both calls run the same summing kernel and the results do not depend
on how the visibilities are cut into work items, so every comparison is bit
for bit.  The tests make calls in a row with different inputs (different
subgrid counts, invalid visibilities in different places, every storage type
with its per-subgrid scales) and calls at the limits of the fixed array
(1,024 subgrids, most of them empty; a call just below the visibility
limit).  They set up all of their own inputs, so they run the same alone in
a fresh process or after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2102_12739_gb300 as dg  # noqa: E402
from paper_2102_12739_gb300 import _native, synth  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPE = synth.SUBGRID_SHAPE


def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch.device("cuda", 0)


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _inputs(counts, seed, bad_rows):
    parts = [synth.random_line(c, np.random.default_rng([200 + seed, s])) for s, c in enumerate(counts)]
    uvw = np.ascontiguousarray(np.concatenate(parts))
    for r in bad_rows:
        uvw[r] = [np.nan, 10.0, 1.5]
    sub = synth.subgrid_stack(len(counts))
    return sub, uvw, synth.offsets_from_counts(counts)


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


def _noalloc(lib, d, g_uv_dev, g_w_dev, dtype, shape, n_sub, sub, scale, uvw, offs, n, out, status):
    stream = torch.cuda.current_stream(d)
    return lib.degrid_execute_noalloc(
        ctypes.c_void_p(stream.cuda_stream), shape[1], shape[0], shape[2],
        _vp(g_uv_dev), g_uv_dev.shape[0], _vp(g_w_dev), g_w_dev.shape[0], dtype,
        n_sub, _vp(sub), _vp(scale), _vp(uvw), _vp(offs), n, _vp(out), _vp(status))


def _tables(d):
    g_uv, g_w = synth.default_tables()
    # the FP32 tables a plan would hold (double -> float, round to nearest)
    return (torch.from_numpy(g_uv.astype(np.float32)).to(d),
            torch.from_numpy(g_w.astype(np.float32)).to(d))


def test_noalloc_matches_degrid_execute_on_two_calls():
    d = _device()
    torch.cuda.set_device(d)
    lib = _native.load()
    g_uv_dev, g_w_dev = _tables(d)
    status = torch.full((2,), -1, dtype=torch.int64, device=d)
    calls = [([3000, 0, 1777, 40], 1, [5, 3100]),
             ([25_000, 9000], 2, [24_999])]
    with dg.DegridPlan(device=d) as plan:
        for counts, seed, bad_rows in calls:
            sub_np, uvw_np, offs_np = _inputs(counts, seed, bad_rows)
            sub = torch.from_numpy(sub_np).to(d)
            uvw = torch.from_numpy(uvw_np).to(d)
            offs = torch.from_numpy(offs_np).to(d)
            n = int(offs_np[-1])
            ref = plan.degrid(sub, uvw, offs).cpu().numpy()
            assert plan.status() == len(bad_rows)

            out = torch.empty(n, dtype=torch.complex64, device=d)
            rc = _noalloc(lib, d, g_uv_dev, g_w_dev, _native.DG_C64, SHAPE, len(counts), sub, None,
                          uvw, offs, n, out, status)
            assert rc == _native.DG_OK, _native.status_string(rc)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_array_equal(_bits(got), _bits(ref))
            assert np.all(got[bad_rows] == 0)
            st = status.cpu().numpy()
            assert st[0] == len(bad_rows)       # this call's count only
            assert st[1] == 0


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_noalloc_reduced_precision_storage_matches_bitwise(dtype):
    # FP16 / BF16 codes with one scale per subgrid (subgrids at different
    # scales), two calls in a row, against plans of the same storage type
    d = _device()
    torch.cuda.set_device(d)
    lib = _native.load()
    g_uv_dev, g_w_dev = _tables(d)
    status = torch.full((2,), -1, dtype=torch.int64, device=d)
    code = _native.DG_C32_F16 if dtype == "f16" else _native.DG_C32_BF16
    calls = [([4000, 1, 2500], 3, [7]),
             ([0, 6000, 300, 70], 4, [6100, 6369])]
    with dg.DegridPlan(dtype=dtype, device=d) as plan:
        for counts, seed, bad_rows in calls:
            sub_np, uvw_np, offs_np = _inputs(counts, seed, bad_rows)
            sub_np[1] *= 1e-3
            codes, scale = dg.pack_subgrids(torch.from_numpy(sub_np).to(d), dtype)
            uvw = torch.from_numpy(uvw_np).to(d)
            offs = torch.from_numpy(offs_np).to(d)
            n = int(offs_np[-1])
            ref = plan.degrid(codes, uvw, offs, scale=scale).cpu().numpy()
            assert plan.status() == len(bad_rows)
            out = torch.empty(n, dtype=torch.complex64, device=d)
            rc = _noalloc(lib, d, g_uv_dev, g_w_dev, code, SHAPE, len(counts), codes, scale, uvw, offs,
                          n, out, status)
            assert rc == _native.DG_OK, _native.status_string(rc)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(_bits(out.cpu().numpy()), _bits(ref))
            assert status.cpu().numpy()[0] == len(bad_rows)
            # a scale is required for these storage types
            assert _noalloc(lib, d, g_uv_dev, g_w_dev, code, SHAPE, len(counts), codes, None, uvw, offs,
                            n, out, status) == _native.DG_ERR_DTYPE


def test_noalloc_at_the_subgrid_limit_with_mostly_empty_lists():
    # 1,024 subgrids (the most the array schedules), 1,000 of them empty,
    # small 16 x 16 x 4 subgrids; then a call with fewer subgrids, whose
    # schedule must not see the previous call's items
    d = _device()
    torch.cuda.set_device(d)
    lib = _native.load()
    g_uv_dev, g_w_dev = _tables(d)
    shape = (16, 16, 4)
    rng = np.random.default_rng(5)
    counts = np.zeros(1024, dtype=np.int64)
    busy = rng.choice(1024, 24, replace=False)
    counts[busy] = rng.integers(1, 30_000, 24)
    counts[1023] = 5
    status = torch.zeros(2, dtype=torch.int64, device=d)
    with dg.DegridPlan(shape=shape, device=d) as plan:
        for cts in (counts, counts[:300]):
            parts = [synth.random_line(int(c), np.random.default_rng([300, s]), shape)
                     for s, c in enumerate(cts)]
            uvw_np = np.ascontiguousarray(np.concatenate(parts))
            offs_np = synth.offsets_from_counts(cts)
            sub = torch.from_numpy(synth.subgrid_stack(len(cts), shape=shape)).to(d)
            uvw = torch.from_numpy(uvw_np).to(d)
            offs = torch.from_numpy(offs_np).to(d)
            n = int(offs_np[-1])
            ref = plan.degrid(sub, uvw, offs).cpu().numpy()
            assert plan.status() == 0
            out = torch.full((n,), float("nan"), dtype=torch.complex64, device=d)
            rc = _noalloc(lib, d, g_uv_dev, g_w_dev, _native.DG_C64, shape, len(cts), sub, None, uvw,
                          offs, n, out, status)
            assert rc == _native.DG_OK, _native.status_string(rc)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(_bits(out.cpu().numpy()), _bits(ref))
            assert status.cpu().numpy().tolist() == [0, 0]


def test_noalloc_just_below_the_visibility_limit():
    # 2^25 - 3 visibilities (the array's item capacity nearly used up) on
    # three dense lines, coordinates generated on the device
    d = _device()
    torch.cuda.set_device(d)
    lib = _native.load()
    g_uv_dev, g_w_dev = _tables(d)
    n = _native_max_vis() - 3
    counts = [n // 3, n // 3, n - 2 * (n // 3)]
    offs_np = synth.offsets_from_counts(counts)
    uvw = torch.empty((n, 3), dtype=torch.float64, device=d)
    for s, c in enumerate(counts):
        synth.random_line_on_device(uvw, int(offs_np[s]), c, np.random.default_rng([400, s]))
    offs = torch.from_numpy(offs_np).to(d)
    sub = synth.subgrid_stack_on_device(3, d)
    status = torch.zeros(2, dtype=torch.int64, device=d)
    with dg.DegridPlan(device=d) as plan:
        ref = plan.degrid(sub, uvw, offs)
        assert plan.status() == 0
    out = torch.empty(n, dtype=torch.complex64, device=d)
    rc = _noalloc(lib, d, g_uv_dev, g_w_dev, _native.DG_C64, SHAPE, 3, sub, None, uvw, offs, n, out, status)
    assert rc == _native.DG_OK, _native.status_string(rc)
    torch.cuda.synchronize()
    assert torch.equal(out.view(torch.int32), ref.view(torch.int32))
    assert status.cpu().numpy().tolist() == [0, 0]


def _native_max_vis():
    import re
    import os
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "degrid.h")
    m = re.search(r"#define\s+DG_NOALLOC_MAX_VIS\s+\(1 << (\d+)\)", open(hdr).read())
    return 1 << int(m.group(1))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    d = _device()
    lib = _native.load()
    dummy = torch.zeros(16, dtype=torch.float64, device=d)
    p = _vp(dummy)
    too_many_vis = (1 << 25) + 1
    rc = lib.degrid_execute_noalloc(None, 512, 512, 4, p, 16384, p, 128, _native.DG_C64, 1, p, None,
                                    p, p, too_many_vis, p, None)
    assert rc == _native.DG_ERR_SCRATCH_LIMIT
    assert "scratch" in _native.status_string(rc)
    rc = lib.degrid_execute_noalloc(None, 512, 512, 4, p, 16384, p, 1024, _native.DG_C64, 1, p, None,
                                    p, p, 10, p, None)
    assert rc == _native.DG_ERR_SCRATCH_LIMIT      # w table beyond the 512 rows it stages
    rc = lib.degrid_execute_noalloc(None, 512, 512, 4, p, 16384, p, 128, _native.DG_C64, 1025, p,
                                    None, p, p, 10, p, None)
    assert rc == _native.DG_ERR_SCRATCH_LIMIT
