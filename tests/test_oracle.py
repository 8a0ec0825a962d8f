"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test targets a different way the oracle could be wrong: the snapping
rule (hand-derived cases), table orientation and axis order (one-hot tables,
brute force from the Kaiser-Bessel closed form), dropped or duplicated terms
(constant subgrid closed form, brute force), linearity, the adjoint pairing
(dot-product identity), integer-shift invariance, out-of-bounds handling and
the gradient convention (finite differences).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2102_12739_gb300 import synth
from tests import _brute

HERE = os.path.dirname(os.path.abspath(__file__))
SHAPE = (512, 512, 4)
G_UV, G_W = synth.default_tables()


def load_coord_cases():
    uvw, expect = [], []
    with open(os.path.join(HERE, "golden", "coords_cases.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            uvw.append([float.fromhex(t) for t in tok[:3]])
            expect.append([int(t) for t in tok[3:9]])
    return np.array(uvw), np.array(expect, dtype=np.int32)


def test_coords_hand_cases():
    uvw, expect = load_coord_cases()
    got, bad = oracle.coords(uvw, SHAPE)
    np.testing.assert_array_equal(got, expect)
    assert bad == int((expect[:, 0] < 0).sum())


def small_random_uvw(rng, n, shape, on_grid=False, dense=False):
    ny, nx, _ = shape
    ulo, uhi = synth.uv_box(nx)
    vlo, vhi = synth.uv_box(ny)
    if dense:
        start = np.array([rng.uniform(ulo, uhi), rng.uniform(vlo, vhi), rng.uniform(1.0, 1.99)])
        end = np.array([rng.uniform(ulo, uhi), rng.uniform(vlo, vhi), rng.uniform(1.0, 1.99)])
        return synth.line(n, start, end)
    u = rng.uniform(ulo, uhi, n)
    v = rng.uniform(vlo, vhi, n)
    w = rng.uniform(1.0, 1.99, n)
    if on_grid:
        u, v, w = np.rint(u), np.rint(v), np.ones(n)
    return np.stack([u, v, w], axis=1)


def random_subgrids(rng, S, shape):
    re = rng.standard_normal((S,) + shape)
    im = rng.standard_normal((S,) + shape)
    return re + 1j * im


def test_delta_gcf_on_grid_returns_addressed_sample():
    # Delta tables: the only non-zero weight sits at offset 0 (row f=0,
    # column W/2-1), so an on-grid visibility returns the sample it addresses.
    shape = (32, 48, 4)
    g_uv = np.zeros_like(G_UV)
    g_uv[0, 3] = 1.0
    g_w = np.zeros_like(G_W)
    g_w[0, 1] = 1.0
    rng = np.random.default_rng(10)
    sub = random_subgrids(rng, 2, shape)
    uvw = small_random_uvw(rng, 300, shape, on_grid=True)
    offs = np.array([0, 170, 300])
    vis, bad = oracle.degrid(g_uv, g_w, sub, uvw, offs)
    assert bad == 0
    s_of = np.repeat([0, 1], [170, 130])
    u, v = uvw[:, 0].astype(int), uvw[:, 1].astype(int)
    # w = 1.0 sits on plane 1: z0 = 0 and column 1 of the w table is offset 0.
    np.testing.assert_array_equal(vis, sub[s_of, v, u, 1])


def test_one_hot_tables_pin_orientation():
    # One non-zero entry (row f*, column k*) per table.  A visibility whose
    # fractional offsets equal f*/O on every axis returns the single sample at
    # start + k* on every axis; any other fraction returns 0.  Swapping the
    # table's rows and columns, or u and v, or the start offset breaks this.
    shape = (40, 56, 4)
    fu_star, ku_star, fw_star, kw_star = 5321, 6, 77, 2
    g_uv = np.zeros_like(G_UV)
    g_uv[fu_star, ku_star] = 1.0
    g_w = np.zeros_like(G_W)
    g_w[fw_star, kw_star] = 1.0
    rng = np.random.default_rng(11)
    sub = random_subgrids(rng, 1, shape)
    n = 200
    iu = rng.integers(3, shape[1] - 4, n)
    iv = rng.integers(3, shape[0] - 4, n)
    u = iu + fu_star / 16384.0
    v = iv + fu_star / 16384.0
    w = 1.0 + fw_star / 128.0
    uvw = np.stack([u, v, np.full(n, w)], axis=1)
    uvw[n // 2:, 0] += 1.0 / 16384.0   # second half: wrong u fraction -> 0
    vis, bad = oracle.degrid(g_uv, g_w, sub, uvw, [0, n])
    assert bad == 0
    x = iu - 3 + ku_star
    y = iv - 3 + ku_star
    z = 0 + kw_star
    expect = sub[0, y, x, z]
    expect[n // 2:] = 0
    np.testing.assert_array_equal(vis, expect)


def test_constant_subgrid_is_product_of_row_sums():
    shape = (24, 24, 4)
    c = 0.75 - 1.25j
    sub = np.full((1,) + shape, c)
    rng = np.random.default_rng(12)
    n = 400
    fu = rng.integers(0, 16384, n)
    fv = rng.integers(0, 16384, n)
    fw = rng.integers(0, 128, n)
    iu = rng.integers(3, shape[1] - 4, n)
    iv = rng.integers(3, shape[0] - 4, n)
    uvw = np.stack([iu + fu / 16384.0, iv + fv / 16384.0, 1.0 + fw / 128.0], axis=1)
    vis, bad = oracle.degrid(G_UV, G_W, sub, uvw, [0, n])
    assert bad == 0
    expect = c * G_UV[fu].sum(1) * G_UV[fv].sum(1) * G_W[fw].sum(1)
    np.testing.assert_allclose(vis, expect, rtol=1e-14, atol=0)


def test_linearity():
    shape = (40, 40, 4)
    rng = np.random.default_rng(13)
    s1 = random_subgrids(rng, 2, shape)
    s2 = random_subgrids(rng, 2, shape)
    uvw = np.concatenate([small_random_uvw(rng, 250, shape),
                          small_random_uvw(rng, 250, shape, dense=True)])
    offs = [0, 250, 500]
    a, b = 0.3 - 2.0j, -1.7 + 0.25j
    lhs, _ = oracle.degrid(G_UV, G_W, a * s1 + b * s2, uvw, offs)
    r1, _ = oracle.degrid(G_UV, G_W, s1, uvw, offs)
    r2, _ = oracle.degrid(G_UV, G_W, s2, uvw, offs)
    rhs = a * r1 + b * r2
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)


def test_adjoint_dot_product_identity():
    shape = (48, 40, 4)
    rng = np.random.default_rng(14)
    S = 3
    sub = random_subgrids(rng, S, shape)
    parts = [small_random_uvw(rng, 300, shape), small_random_uvw(rng, 500, shape, dense=True),
             small_random_uvw(rng, 1, shape)]
    uvw = np.concatenate(parts)
    offs = synth.offsets_from_counts([300, 500, 1])
    y = rng.standard_normal(801) + 1j * rng.standard_normal(801)
    d, _ = oracle.degrid(G_UV, G_W, sub, uvw, offs)
    g, _ = oracle.grid(G_UV, G_W, shape, S, uvw, offs, y)
    lhs = np.vdot(d, y)          # <D s, y> = sum conj(Ds) y
    rhs = np.vdot(sub, g)        # <s, G y>
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("dense", [False, True])
def test_brute_force_degrid_and_grid(dense):
    shape = (16, 20, 4)
    rng = np.random.default_rng(15 + dense)
    S = 2
    sub = random_subgrids(rng, S, shape)
    parts = [small_random_uvw(rng, 60, shape, dense=dense) for _ in range(S)]
    # a few invalid ones: outside in u, in v and in w
    parts[1][:3] = [[1.0, 8.0, 1.5], [8.0, 14.9, 1.5], [8.0, 8.0, 2.2]]
    uvw = np.concatenate(parts)
    offs = [0, 60, 120]
    vis, bad = oracle.degrid(G_UV, G_W, sub, uvw, offs)
    assert bad == 3
    y = rng.standard_normal(120) + 1j * rng.standard_normal(120)
    g, _ = oracle.grid(G_UV, G_W, shape, S, uvw, offs, y)
    for s in range(S):
        rows = slice(offs[s], offs[s + 1])
        D = _brute.dense_matrix(uvw[rows], shape)
        ref = D @ sub[s].ravel()
        assert np.linalg.norm(vis[rows] - ref) <= 1e-12 * np.linalg.norm(ref)
        gref = D.T @ y[rows]
        assert np.linalg.norm(g[s].ravel() - gref) <= 1e-12 * np.linalg.norm(gref)
    assert np.all(vis[60:63] == 0)


def test_touched_counts_match_brute_force():
    shape = (16, 20, 4)
    rng = np.random.default_rng(17)
    uvw = np.concatenate([small_random_uvw(rng, 40, shape),
                          small_random_uvw(rng, 40, shape, dense=True)])
    offs = [0, 40, 80]
    got = oracle.touched(shape, 2, uvw, offs)
    for s in range(2):
        m = _brute.footprint_mask(uvw[offs[s]:offs[s + 1]], shape)
        assert got[s] == int(m.any(axis=0).sum())


def test_integer_shift_invariance_is_bitwise():
    shape = (32, 40, 4)
    rng = np.random.default_rng(18)
    sub = random_subgrids(rng, 1, shape)
    uvw = small_random_uvw(rng, 300, shape)
    uvw[:, 0] = np.clip(uvw[:, 0], 3.5, shape[1] - 5.5)
    shifted = np.roll(sub, 1, axis=2)       # s'[y][x+1][z] = s[y][x][z]
    uvw2 = uvw.copy()
    uvw2[:, 0] += 1.0
    a, _ = oracle.degrid(G_UV, G_W, sub, uvw, [0, 300])
    b, _ = oracle.degrid(G_UV, G_W, shifted, uvw2, [0, 300])
    np.testing.assert_array_equal(a, b)


def test_out_of_bounds_and_empty_subgrids():
    shape = (32, 32, 4)
    rng = np.random.default_rng(19)
    sub = random_subgrids(rng, 3, shape)
    uvw = small_random_uvw(rng, 10, shape)
    uvw[2] = [np.nan, 10, 1.5]
    uvw[5] = [10, -40.0, 1.5]
    uvw[7] = [10, 10, 0.5]
    offs = [0, 0, 10, 10]          # first and last subgrid hold no visibilities
    vis, bad = oracle.degrid(G_UV, G_W, sub, uvw, offs)
    assert bad == 3
    assert vis[2] == 0 and vis[5] == 0 and vis[7] == 0
    ref, _ = oracle.degrid(G_UV, G_W, sub[1:2], np.delete(uvw, [2, 5, 7], axis=0), [0, 7])
    np.testing.assert_array_equal(np.delete(vis, [2, 5, 7]), ref)
    with pytest.raises(ValueError):
        oracle.degrid(G_UV, G_W, sub, uvw, [0, 5, 4, 10])


def test_gradient_matches_central_differences():
    # L(s) = ||D s - y||^2 is quadratic, so FP64 central differences are exact
    # up to rounding; the complex gradient dL/dRe + i dL/dIm equals G(2(Ds - y)).
    shape = (16, 16, 4)
    rng = np.random.default_rng(20)
    sub = random_subgrids(rng, 1, shape)
    uvw = small_random_uvw(rng, 80, shape, dense=True)
    y = rng.standard_normal(80) + 1j * rng.standard_normal(80)

    def loss(s):
        d, _ = oracle.degrid(G_UV, G_W, s, uvw, [0, 80])
        return float(np.sum(np.abs(d - y) ** 2))

    d, _ = oracle.degrid(G_UV, G_W, sub, uvw, [0, 80])
    grad, _ = oracle.grid(G_UV, G_W, shape, 1, uvw, [0, 80], 2 * (d - y))
    touched = np.flatnonzero(np.abs(grad.ravel()) > 1e-3)
    pick = rng.choice(touched, size=16, replace=False)
    h = 1e-3
    for flat in pick:
        for unit in (1.0, 1j):
            sp = sub.copy().ravel()
            sm = sub.copy().ravel()
            sp[flat] += h * unit
            sm[flat] -= h * unit
            fd = (loss(sp.reshape(sub.shape)) - loss(sm.reshape(sub.shape))) / (2 * h)
            an = grad.ravel()[flat].real if unit == 1.0 else grad.ravel()[flat].imag
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


def test_tables_against_library_bessel():
    # The generator's own I0 series against numpy's i0 (a different method),
    # and the table orientation: row 0 peaks at column W/2 - 1 with value 1.
    x = np.linspace(0.0, 20.0, 301)
    np.testing.assert_allclose(synth.bessel_i0(x), np.i0(x), rtol=1e-13)
    assert G_UV.shape == (16384, 8) and G_W.shape == (128, 4)
    assert G_UV[0, 3] == 1.0 and G_W[0, 1] == 1.0
    f = np.arange(16384)
    ref = _brute.kb_closed_form((np.arange(8)[None, :] - 3) - f[:, None] / 16384.0, 8, 18.4)
    np.testing.assert_allclose(G_UV, ref, rtol=1e-13, atol=1e-300)


def test_quantize_matches_library_rounding():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(21)
    x = rng.standard_normal(200_000).astype(np.float32)
    # exact ties for bf16 (half an ulp at 1.0 is 2^-8) and fp16
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.5 + 2 ** -9,
                     1 + 2 ** -11, 1 + 3 * 2 ** -11, 0.0, -0.0], dtype=np.float32)
    x = np.concatenate([x, ties])
    want_bf = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(oracle.bf16_bits_rn(x), want_bf)
    assert oracle.bf16_bits_rn(np.array([1 + 2 ** -8], np.float32))[0] == 0x3F80
    assert oracle.bf16_bits_rn(np.array([1 + 3 * 2 ** -8], np.float32))[0] == 0x3F82
    want_h = torch.from_numpy(x).to(torch.float16).numpy()
    np.testing.assert_array_equal(x.astype(np.float16).view(np.uint16), want_h.view(np.uint16))


def test_quantize_scale_and_range():
    rng = np.random.default_rng(22)
    sub = (rng.standard_normal((3, 8, 8, 4)) + 1j * rng.standard_normal((3, 8, 8, 4))).astype(np.complex64)
    sub[2] = 0
    for dt in ("f16", "bf16"):
        codes, scale = oracle.quantize(sub, dt)
        comp = sub.view(np.float32).reshape(sub.shape + (2,))
        np.testing.assert_array_equal(scale[:2], np.abs(comp[:2]).reshape(2, -1).max(1))
        assert scale[2] == 0 and np.all(codes[2] == 0)
        deq = oracle.dequantize(codes, scale, dt)
        err = np.abs(deq - sub) / np.repeat(np.maximum(scale, 1e-30), 256).reshape(sub.shape)
        tol = 2 ** -11 if dt == "f16" else 2 ** -8
        assert err[:2].max() <= tol * np.sqrt(2)


# ---------------------------------------------------------------------------
# Non-separable G_uv (oracle.degrid_2d): G[fv][fu][b][a], oversampling 64
# ---------------------------------------------------------------------------

O2D = 64


def _onehot_positions(O):
    fv, fu = np.meshgrid(np.arange(O), np.arange(O), indexing="ij")
    return (3 * fv + fu) % 8, (5 * fu + 2 * fv + 1) % 8      # (b*, a*) per (fv, fu)


def test_2d_one_hot_blocks_pin_orientation():
    # Every (fv, fu) block has its single 1 at a different (b*, a*) that is
    # not symmetric in fv/fu or in b/a, so swapping the offsets, the block's
    # axes or the start offset picks the wrong sample.
    shape = (40, 56, 4)
    bstar, astar = _onehot_positions(O2D)
    G = np.zeros((O2D, O2D, 8, 8))
    fv_i, fu_i = np.meshgrid(np.arange(O2D), np.arange(O2D), indexing="ij")
    G[fv_i, fu_i, bstar, astar] = 1.0
    g_w = np.zeros_like(G_W)
    g_w[77, 2] = 1.0
    rng = np.random.default_rng(41)
    sub = random_subgrids(rng, 1, shape)
    n = 500
    iu = rng.integers(3, shape[1] - 4, n)
    iv = rng.integers(3, shape[0] - 4, n)
    fu = rng.integers(0, O2D, n)
    fv = rng.integers(0, O2D, n)
    uvw = np.stack([iu + fu / O2D, iv + fv / O2D, np.full(n, 1.0 + 77 / 128.0)], axis=1)
    vis, bad = oracle.degrid_2d(G, g_w, sub, uvw, [0, n])
    assert bad == 0
    expect = sub[0, iv - 3 + bstar[fv, fu], iu - 3 + astar[fv, fu], 2]
    np.testing.assert_array_equal(vis, expect)


def test_2d_separable_table_matches_separable_oracle():
    # G[fv][fu][b][a] = g[fv][b] g[fu][a] is the separable method: the two
    # oracles agree to FP64 rounding (the weight products round differently)
    g = synth.gcf_table(8, O2D, 2.3 * 8)
    G = g[:, None, :, None] * g[None, :, None, :]
    rng = np.random.default_rng(42)
    shape = (48, 40, 4)
    sub = random_subgrids(rng, 2, shape)
    parts = [synth.random_line(300, np.random.default_rng([42, s]), shape) for s in range(2)]
    uvw = np.concatenate(parts)
    sep, bad1 = oracle.degrid(g, G_W, sub, uvw, [0, 300, 600])
    two, bad2 = oracle.degrid_2d(G, G_W, sub, uvw, [0, 300, 600])
    assert bad1 == bad2 == 0
    assert np.max(np.abs(two - sep)) <= 1e-13 * np.max(np.abs(sep))


def test_2d_diagonal_kernel_closed_form():
    # G = identity block for every offset pair: a non-separable kernel whose
    # degridded value is the sum of the samples on the footprint's diagonal
    # y0 + b, x0 + b (times the w weights)
    shape = (32, 32, 4)
    G = np.broadcast_to(np.eye(8), (O2D, O2D, 8, 8)).copy()
    rng = np.random.default_rng(43)
    sub = random_subgrids(rng, 1, shape)
    n = 300
    iu = rng.integers(3, shape[1] - 4, n)
    iv = rng.integers(3, shape[0] - 4, n)
    fw = rng.integers(0, 128, n)
    uvw = np.stack([iu + rng.integers(0, O2D, n) / O2D, iv + rng.integers(0, O2D, n) / O2D,
                    1.0 + fw / 128.0], axis=1)
    vis, bad = oracle.degrid_2d(G, G_W, sub, uvw, [0, n])
    assert bad == 0
    b = np.arange(8)
    diag = sub[0][(iv - 3)[:, None] + b, (iu - 3)[:, None] + b]      # [n][8][nz]
    expect = np.einsum("nbc,nc->n", diag[:, :, :4], G_W[fw])
    np.testing.assert_allclose(vis, expect, rtol=1e-13, atol=1e-13)


def test_2d_constant_subgrid_is_block_sum():
    shape = (24, 24, 4)
    c = -0.5 + 2.0j
    sub = np.full((1,) + shape, c)
    rng = np.random.default_rng(44)
    G = rng.standard_normal((O2D, O2D, 8, 8))
    n = 300
    fu, fv, fw = rng.integers(0, O2D, n), rng.integers(0, O2D, n), rng.integers(0, 128, n)
    iu = rng.integers(3, shape[1] - 4, n)
    iv = rng.integers(3, shape[0] - 4, n)
    uvw = np.stack([iu + fu / O2D, iv + fv / O2D, 1.0 + fw / 128.0], axis=1)
    uvw[7] = [np.nan, 5.0, 1.5]
    vis, bad = oracle.degrid_2d(G, G_W, sub, uvw, [0, n])
    assert bad == 1 and vis[7] == 0
    expect = c * G[fv, fu].sum(axis=(1, 2)) * G_W[fw].sum(1)
    expect[7] = 0
    np.testing.assert_allclose(vis, expect, rtol=1e-12, atol=1e-12)


def test_2d_adjoint_dot_product_identity():
    # <D s, y> = <s, G y> for the 2D table with a random (non-separable) G
    shape = (28, 36, 4)
    rng = np.random.default_rng(45)
    G = rng.standard_normal((O2D, O2D, 8, 8))
    sub = random_subgrids(rng, 2, shape)
    parts = [synth.piecewise_list(150, np.random.default_rng([45, s]), shape) for s in range(2)]
    uvw = np.concatenate(parts)
    uvw[5] = [np.nan, 4.0, 1.5]
    offs = [0, 150, 300]
    y = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    ds, bad1 = oracle.degrid_2d(G, G_W, sub, uvw, offs)
    gy, bad2 = oracle.grid_2d(G, G_W, shape, 2, uvw, offs, y)
    assert bad1 == bad2 == 1
    lhs = np.vdot(ds, y)
    rhs = np.vdot(sub, gy)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_2d_adjoint_one_hot_block_scatters_one_sample():
    # one visibility, one-hot block (b*, a*) and one-hot w row: exactly one
    # subgrid element receives y, at the footprint start + (b*, a*, k*)
    shape = (24, 24, 4)
    bstar, astar = _onehot_positions(O2D)
    G = np.zeros((O2D, O2D, 8, 8))
    fv_i, fu_i = np.meshgrid(np.arange(O2D), np.arange(O2D), indexing="ij")
    G[fv_i, fu_i, bstar, astar] = 1.0
    g_w = np.zeros_like(G_W)
    g_w[5, 3] = 1.0
    fu, fv = 17, 42
    uvw = np.array([[9 + fu / O2D, 11 + fv / O2D, 1.0 + 5 / 128.0]])
    out, bad = oracle.grid_2d(G, g_w, shape, 1, uvw, [0, 1], np.array([2.5 - 1.5j]))
    assert bad == 0
    nz = np.argwhere(out != 0)
    assert nz.tolist() == [[0, 11 - 3 + bstar[fv, fu], 9 - 3 + astar[fv, fu], 3]]
    assert out[0, 11 - 3 + bstar[fv, fu], 9 - 3 + astar[fv, fu], 3] == 2.5 - 1.5j
