"""Brute-force dense-matrix degridding for tiny grids (test helper).

Independent of both the oracle and the library: the weight of grid point
(y, x, z) for a visibility is evaluated from the Kaiser-Bessel closed form
(numpy's ``i0``), not read from the oversampled tables.  The footprint of a
support-W kernel around the snapped position p/O (p = rint(q O), numpy's
``rint`` rounds half to even) is the W grid points whose offset from p/O lies
in (-W/2, W/2].  A visibility whose footprint leaves the subgrid on any axis
contributes nothing.
"""
import numpy as np


def kb_closed_form(t, support, beta):
    t = np.asarray(t, dtype=np.float64)
    r = 1.0 - (2.0 * t / support) ** 2
    val = np.i0(beta * np.sqrt(np.clip(r, 0.0, None))) / np.i0(beta)
    return np.where(np.abs(t) <= support / 2, val, 0.0)


def axis_weights(q, n, support, oversample, beta):
    """Weights over grid points 0..n-1, or None if the footprint leaves [0, n)."""
    if not np.isfinite(q):
        return None
    snapped = np.rint(q * oversample) / oversample
    pts = np.arange(-2 * support, n + 2 * support, dtype=np.float64)
    off = pts - snapped
    inside = (off > -support / 2) & (off <= support / 2)
    used = pts[inside]
    if used.min() < 0 or used.max() > n - 1:
        return None
    w = np.zeros(n)
    w[used.astype(np.int64)] = kb_closed_form(off[inside], support, beta)
    return w


def dense_matrix(uvw, shape, uv=(8, 16384, 18.4), wk=(4, 128, 9.2)):
    """Dense weight matrix [n_vis][ny*nx*nz] (float64)."""
    ny, nx, nz = shape
    rows = []
    for q in np.asarray(uvw, dtype=np.float64).reshape(-1, 3):
        wu = axis_weights(q[0], nx, *uv)
        wv = axis_weights(q[1], ny, *uv)
        ww = axis_weights(q[2], nz, *wk)
        if wu is None or wv is None or ww is None:
            rows.append(np.zeros(ny * nx * nz))
        else:
            rows.append(np.einsum("y,x,z->yxz", wv, wu, ww).ravel())
    return np.array(rows).reshape(-1, ny * nx * nz)


def footprint_mask(uvw, shape, uv=(8, 16384, 18.4), wk=(4, 128, 9.2)):
    """Boolean [n_vis][ny*nx*nz]: grid points inside each valid footprint."""
    ny, nx, nz = shape
    rows = []
    for q in np.asarray(uvw, dtype=np.float64).reshape(-1, 3):
        ws = [axis_weights(q[0], nx, *uv), axis_weights(q[1], ny, *uv),
              axis_weights(q[2], nz, *wk)]
        if any(w is None for w in ws):
            rows.append(np.zeros(ny * nx * nz, dtype=bool))
            continue
        mu, mv, mw = [np.zeros_like(w, dtype=bool) for w in ws]
        for m, qq, n, (W, O, _) in ((mu, q[0], nx, uv), (mv, q[1], ny, uv), (mw, q[2], nz, wk)):
            snapped = np.rint(qq * O) / O
            pts = np.arange(n, dtype=np.float64)
            m[:] = (pts - snapped > -W / 2) & (pts - snapped <= W / 2)
        rows.append(np.einsum("y,x,z->yxz", mv, mu, mw).ravel())
    return np.array(rows)
