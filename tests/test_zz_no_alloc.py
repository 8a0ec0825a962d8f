"""degrid_execute_noalloc against degrid_execute (GPU only).

degrid_execute_noalloc serves callers that cannot allocate device memory
once they are running (real-time pipelines that must stay out of the CUDA
allocator, hosts whose device memory belongs to another allocator).  It takes
no plan and draws all its scratch from one fixed array inside the library, so
two things need checking: that it computes what the plan-based call
computes, and that the array's leftovers from one call do not leak into the
next.  The test therefore makes two calls in a row with different inputs
(different subgrid counts, invalid visibilities in different places) and
compares each with degrid_execute on the same inputs, within the relative L2
tolerance of the complex64 parity tests.  It sets up all of its own inputs,
so it runs the same alone in a fresh process or after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2102_12739_gb300 as dg  # noqa: E402
from paper_2102_12739_gb300 import _native, synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 2e-6          # relative L2, as for every complex64 parity test
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


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_degrid_execute_on_two_calls():
    d = _device()
    torch.cuda.set_device(d)
    lib = _native.load()
    g_uv, g_w = synth.default_tables()
    # the FP32 tables a plan would hold (double -> float, round to nearest)
    g_uv_dev = torch.from_numpy(g_uv.astype(np.float32)).to(d)
    g_w_dev = torch.from_numpy(g_w.astype(np.float32)).to(d)
    status = torch.full((2,), -1, dtype=torch.int64, device=d)
    stream = torch.cuda.current_stream(d)
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
            rc = lib.degrid_execute_noalloc(
                ctypes.c_void_p(stream.cuda_stream), SHAPE[1], SHAPE[0], SHAPE[2],
                _vp(g_uv_dev), g_uv.shape[0], _vp(g_w_dev), g_w.shape[0], _native.DG_C64,
                len(counts), _vp(sub), None, _vp(uvw), _vp(offs), n, _vp(out), _vp(status))
            assert rc == _native.DG_OK, _native.status_string(rc)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert _rel_l2(got, ref) <= TOL
            assert np.all(got[bad_rows] == 0)
            st = status.cpu().numpy()
            assert st[0] == len(bad_rows)       # this call's count only
            assert st[1] == 0


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
