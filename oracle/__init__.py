"""FP64 CPU oracle for 3D degridding -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library (``paper_2102_12739_gb300``)
never touches it, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain double-precision loops, see its
header for the readings of the paper it encodes); this module compiles it
with gcc on first use and wraps it with ctypes.  It also holds the reference
for the per-subgrid FP16/BF16 storage format (``quantize``), written with
numpy from the IEEE-754 definitions.  ``oracle.predict`` (numpy, FP64) is
the reference of the step upstream of degridding that produces the subgrid
stack (the w-plane grids of improved w-stacking).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_I64 = ctypes.c_int64
_I32 = ctypes.c_int
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, OpenMP, strict FP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB lets the mutation test load a deliberately broken copy.
            path = os.environ.get("ORACLE_LIB") or build()
            lib = ctypes.CDLL(path)
            lib.oracle_coords.restype = _I64
            lib.oracle_coords.argtypes = [_I32] * 7 + [_P, _I64, _P]
            lib.oracle_degrid.restype = _I64
            lib.oracle_degrid.argtypes = ([_I32] * 3 + [_P, _I32, _I32, _P, _I32, _I32,
                                                        _I32, _P, _P, _P, _I64, _P])
            lib.oracle_degrid_2d.restype = _I64
            lib.oracle_degrid_2d.argtypes = lib.oracle_degrid.argtypes
            lib.oracle_grid.restype = _I64
            lib.oracle_grid.argtypes = ([_I32] * 3 + [_P, _I32, _I32, _P, _I32, _I32,
                                                      _I32, _P, _P, _I64, _P, _P, _I32])
            lib.oracle_grid_2d.restype = _I64
            lib.oracle_grid_2d.argtypes = lib.oracle_grid.argtypes
            lib.oracle_touched.restype = _I64
            lib.oracle_touched.argtypes = [_I32] * 8 + [_P, _P, _I64, _P]
            lib.oracle_set_threads.restype = None
            lib.oracle_set_threads.argtypes = [_I32]
            lib.oracle_max_threads.restype = _I32
            lib.oracle_max_threads.argtypes = []
            _lib = lib
    return _lib


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape_tail=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _complex_to_pairs(a) -> np.ndarray:
    """complex array -> contiguous float64 (..., 2); exact for complex64/128."""
    a = np.asarray(a)
    if np.iscomplexobj(a):
        return np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1), dtype=np.float64)
    return np.ascontiguousarray(a, dtype=np.float64)


def _tables(g_uv, g_w):
    g_uv = np.ascontiguousarray(g_uv, dtype=np.float64)
    g_w = np.ascontiguousarray(g_w, dtype=np.float64)
    return g_uv, g_w


def coords(uvw, shape, uv_support=8, uv_oversample=16384, w_support=4, w_oversample=128):
    """(x0, y0, z0, fu, fv, fw) per visibility, int32 [n][6]; -1 if invalid.

    Returns (coords, n_invalid).
    """
    ny, nx, nz = shape
    uvw = _f64(uvw).reshape(-1, 3)
    out = np.empty((uvw.shape[0], 6), dtype=np.int32)
    bad = _load().oracle_coords(nx, ny, nz, uv_support, uv_oversample, w_support,
                                w_oversample, _ptr(uvw), uvw.shape[0], _ptr(out))
    return out, int(bad)


def degrid(g_uv, g_w, subgrids, uvw, vis_offsets):
    """Degridded visibilities, complex128 [n], and the invalid count.

    subgrids: complex [S][ny][nx][nz] (promoted exactly to float64);
    uvw: float64 [n][3]; vis_offsets: int64 [S + 1].
    """
    g_uv, g_w = _tables(g_uv, g_w)
    sub = _complex_to_pairs(subgrids)
    S, ny, nx, nz = sub.shape[:4]
    uvw = _f64(uvw).reshape(-1, 3)
    offs = np.ascontiguousarray(vis_offsets, dtype=np.int64)
    assert offs.shape == (S + 1,)
    out = np.empty((uvw.shape[0], 2), dtype=np.float64)
    bad = _load().oracle_degrid(nx, ny, nz, _ptr(g_uv), g_uv.shape[1], g_uv.shape[0],
                                _ptr(g_w), g_w.shape[1], g_w.shape[0], S, _ptr(sub),
                                _ptr(uvw), _ptr(offs), uvw.shape[0], _ptr(out))
    if bad < 0:
        raise ValueError("oracle_degrid: invalid vis_offsets")
    return out[:, 0] + 1j * out[:, 1], int(bad)


def degrid_2d(g_uv2, g_w, subgrids, uvw, vis_offsets):
    """Degridding with a non-separable G_uv table g_uv2 [O][O][W][W] indexed
    [fv][fu][b][a]; complex128 [n] and the invalid count."""
    g_uv2 = np.ascontiguousarray(g_uv2, dtype=np.float64)
    O, O2, W, W2 = g_uv2.shape
    assert O == O2 and W == W2
    g_w = np.ascontiguousarray(g_w, dtype=np.float64)
    sub = _complex_to_pairs(subgrids)
    S, ny, nx, nz = sub.shape[:4]
    uvw = _f64(uvw).reshape(-1, 3)
    offs = np.ascontiguousarray(vis_offsets, dtype=np.int64)
    assert offs.shape == (S + 1,)
    out = np.empty((uvw.shape[0], 2), dtype=np.float64)
    bad = _load().oracle_degrid_2d(nx, ny, nz, _ptr(g_uv2), W, O, _ptr(g_w), g_w.shape[1],
                                   g_w.shape[0], S, _ptr(sub), _ptr(uvw), _ptr(offs),
                                   uvw.shape[0], _ptr(out))
    if bad < 0:
        raise ValueError("oracle_degrid_2d: invalid vis_offsets")
    return out[:, 0] + 1j * out[:, 1], int(bad)


def grid(g_uv, g_w, shape, n_subgrids, uvw, vis_offsets, vis, out=None):
    """Adjoint of ``degrid``: complex128 [S][ny][nx][nz] and the invalid count.

    If ``out`` (complex128, C-contiguous) is given the result is added to it.
    """
    g_uv, g_w = _tables(g_uv, g_w)
    ny, nx, nz = shape
    uvw = _f64(uvw).reshape(-1, 3)
    offs = np.ascontiguousarray(vis_offsets, dtype=np.int64)
    y = _complex_to_pairs(vis).reshape(-1, 2)
    accumulate = out is not None
    if out is None:
        out = np.empty((n_subgrids, ny, nx, nz), dtype=np.complex128)
    assert out.dtype == np.complex128 and out.flags.c_contiguous
    buf = out.view(np.float64)
    bad = _load().oracle_grid(nx, ny, nz, _ptr(g_uv), g_uv.shape[1], g_uv.shape[0],
                              _ptr(g_w), g_w.shape[1], g_w.shape[0], n_subgrids,
                              _ptr(uvw), _ptr(offs), uvw.shape[0], _ptr(y), _ptr(buf),
                              int(accumulate))
    if bad < 0:
        raise ValueError("oracle_grid: invalid vis_offsets")
    return out, int(bad)


def grid_2d(g_uv2, g_w, shape, n_subgrids, uvw, vis_offsets, vis, out=None):
    """Adjoint of ``degrid_2d``: complex128 [S][ny][nx][nz] and the invalid
    count (added to ``out`` if given)."""
    g_uv2 = np.ascontiguousarray(g_uv2, dtype=np.float64)
    O, O2, W, W2 = g_uv2.shape
    assert O == O2 and W == W2
    g_w = np.ascontiguousarray(g_w, dtype=np.float64)
    ny, nx, nz = shape
    uvw = _f64(uvw).reshape(-1, 3)
    offs = np.ascontiguousarray(vis_offsets, dtype=np.int64)
    y = _complex_to_pairs(vis).reshape(-1, 2)
    accumulate = out is not None
    if out is None:
        out = np.empty((n_subgrids, ny, nx, nz), dtype=np.complex128)
    assert out.dtype == np.complex128 and out.flags.c_contiguous
    buf = out.view(np.float64)
    bad = _load().oracle_grid_2d(nx, ny, nz, _ptr(g_uv2), W, O, _ptr(g_w), g_w.shape[1],
                                 g_w.shape[0], n_subgrids, _ptr(uvw), _ptr(offs), uvw.shape[0],
                                 _ptr(y), _ptr(buf), int(accumulate))
    if bad < 0:
        raise ValueError("oracle_grid_2d: invalid vis_offsets")
    return out, int(bad)


def touched(shape, n_subgrids, uvw, vis_offsets, uv_support=8, uv_oversample=16384,
            w_support=4, w_oversample=128):
    """Distinct subgrid elements touched per subgrid, int64 [S]."""
    ny, nx, nz = shape
    uvw = _f64(uvw).reshape(-1, 3)
    offs = np.ascontiguousarray(vis_offsets, dtype=np.int64)
    out = np.zeros(n_subgrids, dtype=np.int64)
    total = _load().oracle_touched(nx, ny, nz, uv_support, uv_oversample, w_support,
                                   w_oversample, n_subgrids, _ptr(uvw), _ptr(offs),
                                   uvw.shape[0], _ptr(out))
    if total < 0:
        raise ValueError("oracle_touched: invalid vis_offsets")
    return out


# ---------------------------------------------------------------------------
# Reduced-precision subgrid storage (per-subgrid scale to max |component|)
# ---------------------------------------------------------------------------

def bf16_bits_rn(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit patterns (uint16), round to nearest, ties to even.

    bfloat16 keeps the top 16 bits of the IEEE-754 binary32 pattern; rounding
    adds 0x7FFF plus the lowest kept bit before truncating.  NaNs map to a
    quiet NaN.
    """
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)
    nan = np.isnan(np.asarray(x, dtype=np.float32))
    r[nan] = 0x7FC0
    return r


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


def quantize(subgrids: np.ndarray, dtype: str):
    """Store complex64 subgrids as FP16 or BF16 pairs with a per-subgrid scale.

    scale[s] = max over subgrid s of max(|Re|, |Im|) (exact in FP32); each
    component is divided by the scale in FP32 (IEEE division, round to
    nearest) and rounded to nearest-even in the target format; an all-zero
    subgrid gets scale 0 and zero codes.  Returns (codes uint16
    [S][ny][nx][nz][2], scale float32 [S]).
    """
    sub = np.ascontiguousarray(subgrids, dtype=np.complex64)
    S = sub.shape[0]
    comp = sub.view(np.float32).reshape(sub.shape + (2,))
    scale = np.abs(comp).reshape(S, -1).max(axis=1).astype(np.float32)
    safe = np.where(scale > 0, scale, np.float32(1.0)).astype(np.float32)
    bshape = (S,) + (1,) * (comp.ndim - 1)
    q = (comp / safe.reshape(bshape)).astype(np.float32)
    q[scale == 0] = 0.0
    if dtype == "f16":
        codes = q.astype(np.float16).view(np.uint16)
    elif dtype == "bf16":
        codes = bf16_bits_rn(q)
    else:
        raise ValueError(dtype)
    return codes, scale


def dequantize(codes: np.ndarray, scale: np.ndarray, dtype: str) -> np.ndarray:
    """Exact FP64 value of the stored subgrids: code * scale, complex128."""
    if dtype == "f16":
        f = np.asarray(codes, dtype=np.uint16).view(np.float16).astype(np.float64)
    elif dtype == "bf16":
        f = bf16_bits_to_f32(codes).astype(np.float64)
    else:
        raise ValueError(dtype)
    S = f.shape[0]
    f = f * np.asarray(scale, dtype=np.float64).reshape((S,) + (1,) * (f.ndim - 1))
    return f[..., 0] + 1j * f[..., 1]
