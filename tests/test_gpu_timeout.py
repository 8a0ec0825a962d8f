"""The bounded device-side wait that gives up (GPU only).

The gather kernel waits on an mbarrier for the tensor copies of each stage
of footprints, with a limit on the polls; a wait that runs out records a
flag that degrid_get_status reports as DG_ERR_TIMEOUT, waits (with the full
limit) for the warp's copies still in flight and ends the warp.  The library
variant "timeout" gives that wait a limit of zero polls from a warp's fourth
stage on, so it runs out while the stage's copies are in flight.  Nothing
faults and nothing hangs: every copy was issued for a valid box and lands.

Checked in a child process that loads the variant: the status is
DG_ERR_TIMEOUT; every visibility the kernel wrote before its warp gave up
equals the FP64 oracle (the others keep the caller's sentinel); and the
context and the plan stay usable: the footprint-cache kernel (no mbarrier
waits) then gives every visibility, with a clean status.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def check_timeout_variant():
    import torch

    import oracle
    import paper_2102_12739_gb300 as dg
    from paper_2102_12739_gb300 import _native, synth
    from tests.test_gpu_parity import G_UV, G_W, rel_l2, small_workload, upload

    from paper_2102_12739_gb300 import build
    assert _native.lib_path() == build.variant_path("timeout")
    d = torch.device("cuda", 0)
    w = small_workload([3000, 0, 2000, 517], kind="scatter", seed=61)
    sub_np = synth.subgrid_stack(4)
    sub, uvw, offs = upload(w, sub_np)
    ref, bad = oracle.degrid(G_UV, G_W, sub_np.astype(np.complex128), w.uvw, w.vis_offsets)
    assert bad == 0
    with dg.DegridPlan(device=d, gather=True) as p:
        out = torch.full((w.n_vis,), float("nan"), dtype=torch.complex64, device=d)
        p.degrid(sub, uvw, offs, out=out)
        try:
            p.status()
            raise AssertionError("the wait did not run out")
        except dg.DegridError as e:
            assert e.status == _native.DG_ERR_TIMEOUT, e
        got = out.cpu().numpy()
        written = ~np.isnan(got.real)
        n_written = int(written.sum())
        # each warp sums its first three stages of four visibilities, then gives up
        assert 0 < n_written < w.n_vis, n_written
        assert rel_l2(got[written], ref[written]) <= 2e-6
        assert np.max(np.abs(got[written] - ref[written])) <= 1e-5
        # the status was read and cleared; the context and the plan still work
        assert p.status() == 0
        p.set_gather(False)
        full = p.degrid(sub, uvw, offs).cpu().numpy()
        assert p.status() == 0
        assert rel_l2(full, ref) <= 2e-6
    print("timeout ok: %d of %d visibilities written before the waits gave up" % (n_written, w.n_vis))


def test_a_bounded_wait_that_runs_out_reports_timeout():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2102_12739_gb300 import build
    build.build_variant("timeout")
    env = dict(os.environ, DEGRID_LIBRARY_VARIANT="timeout")
    r = subprocess.run([sys.executable, "-c", "from tests.test_gpu_timeout import check_timeout_variant as c; c()"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-25:])
    assert r.returncode == 0, tail
    assert "timeout ok" in r.stdout, tail
