"""The subgrid producer on the GPU against its FP64 oracle (GPU only).

The producer makes the stack degridding reads: for subgrid s the w-plane
grids of the tapered sky image (improved w-stacking), a window of N x N uv
cells at nz w-planes.  Its CUDA path (a screen kernel, a batched FFT, a
window kernel) is checked on every cell against oracle.predict, at small
sizes with every kind of offset and at the full 512 x 512 x 4 size of the
degridding workloads, and independently of the oracle against the analytic
visibility of a point source.  The last test runs the whole pipeline: sky
image -> subgrids -> visibilities, against the oracle's subgrids degridded by
the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import predict as P  # noqa: E402
import paper_2102_12739_gb300 as dg  # noqa: E402
from paper_2102_12739_gb300 import _native, synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 2e-6          # relative L2, as for the complex64 degridding


def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch.device("cuda", 0)


def rel_l2(got, ref):
    return float(np.linalg.norm(np.asarray(got) - ref) / np.linalg.norm(ref))


def run(image, theta, uv, w, nz, taper=None, per_pass=4):
    d = dev()
    n = image.shape[0]
    with dg.SubgridPredictor(n=n, nz=nz, subgrids_per_pass=per_pass, device=d) as pr:
        out = pr.predict(torch.from_numpy(np.ascontiguousarray(image, dtype=np.complex64)).to(d), theta,
                         torch.from_numpy(np.ascontiguousarray(uv, dtype=np.int32)).to(d),
                         torch.from_numpy(np.ascontiguousarray(w, dtype=np.float64)).to(d),
                         taper=None if taper is None else torch.from_numpy(taper).to(d))
        return out.cpu().numpy()


@pytest.mark.parametrize("n,nz,theta,per_pass", [(64, 4, 0.3, 2), (48, 3, 1.9, 4), (16, 1, 0.05, 1)])
def test_small_stacks_every_cell(n, nz, theta, per_pass):
    # positive, negative and wrapping cell offsets, large and negative w,
    # a ragged last pass, pixels outside the unit circle (theta 1.9)
    rng = np.random.default_rng(n)
    img = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    taper = rng.uniform(0.5, 2.0, (n, n)).astype(np.float32)
    uv = np.array([[0, 0], [5, -3], [-n - 7, 2 * n + 1], [n // 2, -n // 2], [1, 1]], dtype=np.int32)
    w = np.array([[0.0, 1.0], [1234.5, 17.25], [-5000.0, -80.0], [31.0, 0.0], [250000.0, 900.0]])
    got = run(img, theta, uv, w, nz, taper, per_pass)
    ref = P.predict(img, theta, np.concatenate([uv, w], axis=1), nz=nz, taper=taper)
    for s in range(len(uv)):
        assert rel_l2(got[s], ref[s]) <= TOL, (s, rel_l2(got[s], ref[s]))


def test_passes_of_more_than_256_subgrids():
    # a pass of 300 subgrids: the screen kernel splits the subgrids' w in
    # tiles of 256; plane spacings equal within runs and changing between
    # them (the step screen is reused, then made again), and a second pass
    n, nz, S, per_pass = 16, 2, 340, 300
    rng = np.random.default_rng(11)
    img = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    uv = rng.integers(-40, 40, size=(S, 2)).astype(np.int32)
    w = np.stack([rng.uniform(-3000.0, 3000.0, S), np.repeat([25.0, 40.0, 25.0, 7.5], S // 4)], axis=1)
    got = run(img, 0.4, uv, w, nz, per_pass=per_pass)
    ref = P.predict(img, 0.4, np.concatenate([uv, w], axis=1), nz=nz)
    assert rel_l2(got, ref) <= TOL
    for s in (0, 255, 256, 299, 300, S - 1):
        assert rel_l2(got[s], ref[s]) <= TOL, s


def test_full_size_stack_every_cell_and_a_point_source():
    # 16 subgrids of 512 x 512 x 4 from the model sky: every cell against the
    # oracle; then one unit source, against its analytic visibility
    n, S = 512, 16
    img = synth.sky_image(n)
    taper = synth.image_taper(n)
    uv, w = synth.predict_offsets(S)
    got = run(img, synth.PREDICT_THETA, uv, w, 4, taper, per_pass=6)
    ref = P.predict(img, synth.PREDICT_THETA, np.concatenate([uv, w], axis=1), nz=4, taper=taper)
    for s in range(S):
        assert rel_l2(got[s], ref[s]) <= TOL, (s, rel_l2(got[s], ref[s]))
    a0, b0 = 400, 77
    one = np.zeros((n, n), dtype=np.complex64)
    one[b0, a0] = 1.0
    uv1 = np.array([[3, -9]], dtype=np.int32)
    w1 = np.array([[2500.0, 50.0]])
    g = run(one, synth.PREDICT_THETA, uv1, w1, 4)[0]
    th = synth.PREDICT_THETA
    l0, m0 = (a0 - n // 2) * th / n, (b0 - n // 2) * th / n
    n0 = np.sqrt(1 - l0 * l0 - m0 * m0)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u = (x - n // 2 + 3) / th
    v = (y - n // 2 - 9) / th
    for c in range(4):
        want = np.exp(-2j * np.pi * (u * l0 + v * m0 + (2500.0 + 50.0 * c) * (n0 - 1)))
        assert np.max(np.abs(g[:, :, c] - want)) <= 2e-6


def test_untapered_equals_unit_taper_and_arguments_are_checked():
    d = dev()
    n = 32
    rng = np.random.default_rng(3)
    img = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    uv = np.array([[1, 2]], dtype=np.int32)
    w = np.array([[10.0, 2.0]])
    a = run(img, 0.5, uv, w, 4)
    b = run(img, 0.5, uv, w, 4, taper=np.ones((n, n), dtype=np.float32))
    np.testing.assert_array_equal(a.view(np.uint64), b.view(np.uint64))
    lib = _native.load()
    import ctypes
    h = ctypes.c_void_p()
    assert lib.subgrid_predict_plan_create(ctypes.byref(h), 31, 4, 1, 0) == _native.DG_ERR_ARG
    assert lib.subgrid_predict_plan_create(ctypes.byref(h), 32, 0, 1, 0) == _native.DG_ERR_ARG
    with dg.SubgridPredictor(n=n, nz=4, device=d) as pr:
        im = torch.from_numpy(img).to(d)
        uvt = torch.from_numpy(uv).to(d)
        wt = torch.from_numpy(w).to(d)
        with pytest.raises(dg.DegridError):
            pr.predict(im, 0.0, uvt, wt)
        with pytest.raises(dg.DegridError):
            pr.predict(im, float("nan"), uvt, wt)
        empty = pr.predict(im, 0.5, uvt[:0], wt[:0])
        assert empty.shape == (0, n, n, 4)


def test_sky_to_visibilities_pipeline():
    # the producer's subgrids degridded on the GPU, against the oracle's
    # subgrids degridded by the oracle, on lines of visibilities
    d = dev()
    n, S = 512, 4
    img = synth.sky_image(n)
    taper = synth.image_taper(n)
    uv, w = synth.predict_offsets(S)
    w_lines = synth.lines_workload("pipeline", [30_000] * S)
    with dg.SubgridPredictor(n=n, nz=4, device=d) as pr, dg.DegridPlan(device=d) as plan:
        sub = pr.predict(torch.from_numpy(img).to(d), synth.PREDICT_THETA, torch.from_numpy(uv).to(d),
                         torch.from_numpy(w).to(d), taper=torch.from_numpy(taper).to(d))
        vis = plan.degrid(sub, torch.from_numpy(w_lines.uvw).to(d),
                          torch.from_numpy(w_lines.vis_offsets).to(d)).cpu().numpy()
        assert plan.status() == 0
    ref_sub = P.predict(img, synth.PREDICT_THETA, np.concatenate([uv, w], axis=1), nz=4, taper=taper)
    g_uv, g_w = synth.default_tables()
    ref, bad = oracle.degrid(g_uv, g_w, ref_sub, w_lines.uvw, w_lines.vis_offsets)
    assert bad == 0
    assert rel_l2(vis, ref) <= 4e-6
