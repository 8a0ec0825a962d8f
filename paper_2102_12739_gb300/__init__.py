"""GB300-native 3D degridding (arXiv:2102.12739).

The compute path is the CUDA library ``libdegrid.so`` (C ABI in
``include/degrid.h``); this module only marshals torch tensors into its
calls.  PyTorch supplies device memory, streams and autograd.  There is no
CPU fallback: without the library (or a GPU) every compute call raises.

Main objects:
  DegridPlan        GCF tables on the device + scratch + tuning
  DegridPlan.degrid visibilities from a subgrid stack (degrid_execute)
  DegridPlan.grid   the adjoint (grid_adjoint_execute)
  DegridPlan.coords per-visibility start points and GCF rows
  pack_subgrids     complex64 -> FP16/BF16 storage with per-subgrid scale
  DegridFn          torch.autograd.Function, backward = adjoint kernel
  autotune          pick chunk / warps / blocks per SM by timing
  SubgridPredictor  the subgrid stack from a sky image (the w-plane grids of
                    improved w-stacking, upstream of degridding)
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import synth
from ._native import (DG_C32_BF16, DG_C32_F16, DG_C64, DG_ERR_OFFSETS, DG_OK,  # noqa: F401
                      DegridError, SIGNATURES, check, lib_path, load, status_string)

__all__ = ["DegridPlan", "DegridFn", "DegridError", "pack_subgrids", "degrid", "autotune",
           "measure_fp32_peak", "measure_l2_read_bw", "measure_l2_reduce_bw", "synth", "load", "lib_path", "SIGNATURES",
           "SubgridPredictor"]

DTYPES = {"c64": DG_C64, "f16": DG_C32_F16, "bf16": DG_C32_BF16}


def _torch():
    import torch
    return torch


def _vp(t) -> Optional[ctypes.c_void_p]:
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream, device):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t, name, dtype, device, shape=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name} must live on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


class DegridPlan:
    """GCF tables and scratch for one subgrid shape, storage type and device.

    shape   (ny, nx, nz) of every subgrid; default (512, 512, 4)
    g_uv    float64 [O_uv][8] oversampled uv GCF (default: Kaiser-Bessel,
            oversampling 16384); row f, column k = kernel at offset
            (k - 3) - f / O_uv
    g_w     float64 [O_w][4] w GCF (default: Kaiser-Bessel, oversampling 128)
    dtype   subgrid storage: "c64", "f16" or "bf16"
    device  CUDA device (index, string or torch.device); default current
    """

    def __init__(self, shape=synth.SUBGRID_SHAPE, g_uv=None, g_w=None, dtype: str = "c64",
                 device=None, compensated: bool = False, g_uv2=None, gather: bool = False):
        torch = _torch()
        lib = load()
        if dtype not in DTYPES:
            raise ValueError(f"dtype must be one of {sorted(DTYPES)}")
        if g_uv is None or g_w is None:
            d_uv, d_w = synth.default_tables()
            g_uv = d_uv if g_uv is None else g_uv
            g_w = d_w if g_w is None else g_w
        self.g_uv = np.ascontiguousarray(g_uv, dtype=np.float64)
        self.g_w = np.ascontiguousarray(g_w, dtype=np.float64)
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        device = torch.device(device)
        if device.type != "cuda":
            raise ValueError("DegridPlan needs a CUDA device")
        if device.index is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = device
        self.shape = tuple(int(x) for x in shape)
        self.dtype = dtype
        ny, nx, nz = self.shape
        h = ctypes.c_void_p()
        self.table2d = g_uv2 is not None
        if self.table2d:
            # non-separable G_uv [O][O][8][8] indexed [fv][fu][b][a]
            self.g_uv2 = np.ascontiguousarray(g_uv2, dtype=np.float64)
            O = self.g_uv2.shape[0]
            if self.g_uv2.shape != (O, O, 8, 8):
                raise ValueError("g_uv2 must have shape [O][O][8][8]")
            st = lib.degrid_plan_create_2d(ctypes.byref(h), nx, ny, nz,
                                           self.g_uv2.ctypes.data_as(ctypes.c_void_p), O,
                                           self.g_w.ctypes.data_as(ctypes.c_void_p),
                                           self.g_w.shape[1], self.g_w.shape[0], DTYPES[dtype],
                                           device.index)
            check(st, "degrid_plan_create_2d")
        else:
            st = lib.degrid_plan_create(ctypes.byref(h), nx, ny, nz,
                                        self.g_uv.ctypes.data_as(ctypes.c_void_p),
                                        self.g_uv.shape[1], self.g_uv.shape[0],
                                        self.g_w.ctypes.data_as(ctypes.c_void_p),
                                        self.g_w.shape[1], self.g_w.shape[0], DTYPES[dtype],
                                        device.index)
            check(st, "degrid_plan_create")
        self._h = h
        if compensated:
            self.set_compensated(True)
        if gather:
            self.set_gather(True)

    # -- lifetime --------------------------------------------------------
    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("plan has been closed")
        return self._h

    def close(self) -> None:
        h, self._h = getattr(self, "_h", None), None
        if h is not None:
            load().degrid_plan_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- tuning ----------------------------------------------------------
    def set_tuning(self, chunk: int = 0, warps_per_block: int = 0, blocks_per_sm: int = -1) -> None:
        check(load().degrid_plan_set_tuning(self.handle, chunk, warps_per_block, blocks_per_sm),
              "degrid_plan_set_tuning")

    def tuning(self) -> dict:
        c, w, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(load().degrid_plan_get_tuning(self.handle, ctypes.byref(c), ctypes.byref(w),
                                            ctypes.byref(b)), "degrid_plan_get_tuning")
        return {"chunk": c.value, "warps_per_block": w.value, "blocks_per_sm": b.value,
                "direct_runs": self.direct_runs, "gather": self.gather}

    def set_compensated(self, enabled: bool = True) -> None:
        """Compensated (TwoSum) reduction of the lane partials in degrid()."""
        check(load().degrid_plan_set_compensated(self.handle, 1 if enabled else 0),
              "degrid_plan_set_compensated")

    @property
    def compensated(self) -> bool:
        v = ctypes.c_int()
        check(load().degrid_plan_get_compensated(self.handle, ctypes.byref(v)),
              "degrid_plan_get_compensated")
        return bool(v.value)

    def set_direct_runs(self, min_runs: int) -> None:
        """Halves of 32 visibilities with at least min_runs footprint runs are
        summed directly instead of through the footprint cache (1..33; 33 =
        never).  Results are bitwise the same either way."""
        check(load().degrid_plan_set_direct_runs(self.handle, int(min_runs)),
              "degrid_plan_set_direct_runs")

    @property
    def direct_runs(self) -> int:
        v = ctypes.c_int()
        check(load().degrid_plan_get_direct_runs(self.handle, ctypes.byref(v)),
              "degrid_plan_get_direct_runs")
        return v.value

    def set_gather(self, enabled: bool = True) -> None:
        """Sum through the gather kernel (every footprint streamed into shared
        memory; for scattered coverage).  Results are bitwise the same as the
        footprint-cache path.  Needs nz = 4 and a separable G_uv table."""
        check(load().degrid_plan_set_gather(self.handle, 1 if enabled else 0),
              "degrid_plan_set_gather")

    def set_host_direct(self, enabled: bool = True) -> None:
        """Let degrid_host() read pinned host inputs in place (default), or
        always copy them."""
        check(load().degrid_plan_set_host_direct(self.handle, 1 if enabled else 0),
              "degrid_plan_set_host_direct")

    @property
    def host_direct(self) -> bool:
        v = ctypes.c_int()
        check(load().degrid_plan_get_host_direct(self.handle, ctypes.byref(v)),
              "degrid_plan_get_host_direct")
        return bool(v.value)

    @property
    def gather(self) -> bool:
        v = ctypes.c_int()
        check(load().degrid_plan_get_gather(self.handle, ctypes.byref(v)), "degrid_plan_get_gather")
        return bool(v.value)

    def enable_timing(self, n_slots: int = 4096) -> None:
        """Record a CUDA event pair around the main kernel of each of the next
        calls (cycling through n_slots pairs); n_slots = 0 turns timing off."""
        check(load().degrid_plan_enable_timing(self.handle, int(n_slots)),
              "degrid_plan_enable_timing")

    def kernel_times_ms(self, n: int) -> list:
        """Durations of the most recent (up to n) timed main-kernel launches,
        oldest first (synchronises on the newest)."""
        buf = (ctypes.c_float * max(int(n), 1))()
        cnt = ctypes.c_int()
        check(load().degrid_plan_kernel_times_ms(self.handle, buf, int(n), ctypes.byref(cnt)),
              "degrid_plan_kernel_times_ms")
        return [float(buf[i]) for i in range(cnt.value)]

    # -- helpers ---------------------------------------------------------
    def _subgrid_view(self, subgrids):
        torch = _torch()
        ny, nx, nz = self.shape
        if self.dtype == "c64":
            if subgrids.dtype == torch.complex64:
                _need(subgrids, "subgrids", torch.complex64, self.device)
                if tuple(subgrids.shape[1:]) != (ny, nx, nz):
                    raise ValueError(f"subgrids must be [S, {ny}, {nx}, {nz}] complex64")
                return subgrids, subgrids.shape[0]
            _need(subgrids, "subgrids", torch.float32, self.device)
        else:
            want = torch.float16 if self.dtype == "f16" else torch.bfloat16
            _need(subgrids, "subgrids", want, self.device)
        if tuple(subgrids.shape[1:]) != (ny, nx, nz, 2):
            raise ValueError(f"subgrids must be [S, {ny}, {nx}, {nz}, 2]")
        return subgrids, subgrids.shape[0]

    def _common(self, uvw, vis_offsets, n_subgrids):
        torch = _torch()
        _need(uvw, "uvw", torch.float64, self.device)
        if uvw.dim() != 2 or uvw.shape[1] != 3:
            raise ValueError("uvw must be [N, 3] float64")
        _need(vis_offsets, "vis_offsets", torch.int64, self.device, (n_subgrids + 1,))
        return uvw.shape[0]

    # -- compute ---------------------------------------------------------
    def degrid(self, subgrids, uvw, vis_offsets, scale=None, out=None, stream=None):
        """Visibilities complex64 [N] from the subgrid stack (degrid_execute)."""
        torch = _torch()
        sub, S = self._subgrid_view(subgrids)
        n = self._common(uvw, vis_offsets, S)
        if self.dtype != "c64":
            if scale is None:
                raise ValueError("scale is required for f16/bf16 subgrids")
            _need(scale, "scale", torch.float32, self.device, (S,))
        if out is None:
            out = torch.empty(n, dtype=torch.complex64, device=self.device)
        else:
            _need(out, "out", torch.complex64, self.device, (n,))
        st = load().degrid_execute(self.handle, _stream_handle(stream, self.device), S, _vp(sub),
                                   _vp(scale) if self.dtype != "c64" else None, _vp(uvw),
                                   _vp(vis_offsets), n, _vp(out))
        check(st, "degrid_execute")
        return out

    def degrid_host(self, subgrids, uvw, vis_offsets, scale=None, out=None):
        """degrid() on HOST data (degrid_execute_host); returns when the
        complex64 [N] host output is complete.  With pinned (page-locked)
        subgrids, coordinates and output the kernel reads and writes them in
        place over the host link; otherwise the call copies the inputs in
        subgrid groups, overlapping the copies with the sums.

        Inputs are CPU torch tensors or numpy arrays (subgrids complex64, or
        for f16/bf16 plans the uint16 code pairs [S, ny, nx, nz, 2] with a
        float32 scale [S]).
        """
        torch = _torch()

        def cpu(x, dtype, name):
            if not isinstance(x, torch.Tensor):
                x = torch.from_numpy(np.ascontiguousarray(x))
            if x.device.type != "cpu" or x.dtype != dtype or not x.is_contiguous():
                raise TypeError(f"{name} must be a contiguous CPU {dtype} tensor")
            return x

        sub_dtype = torch.complex64 if self.dtype == "c64" else (
            torch.float16 if self.dtype == "f16" else torch.bfloat16)
        if self.dtype != "c64" and isinstance(subgrids, np.ndarray):
            subgrids = torch.from_numpy(np.ascontiguousarray(subgrids).view(np.int16)).view(sub_dtype)
        sub = cpu(subgrids, sub_dtype, "subgrids")
        S = sub.shape[0]
        uvw = cpu(uvw, torch.float64, "uvw")
        offs = cpu(vis_offsets, torch.int64, "vis_offsets")
        n = uvw.shape[0]
        if offs.shape != (S + 1,) or uvw.shape != (n, 3):
            raise ValueError("vis_offsets must be [S + 1] and uvw [N, 3]")
        sc = None
        if self.dtype != "c64":
            if scale is None:
                raise ValueError("scale is required for f16/bf16 subgrids")
            sc = cpu(scale, torch.float32, "scale")
        if out is None:
            out = torch.empty(n, dtype=torch.complex64, pin_memory=True)
        else:
            out = cpu(out, torch.complex64, "out")
            if out.shape != (n,):
                raise ValueError("out must be [N]")
        st = load().degrid_execute_host(self.handle, S, _vp(sub), _vp(sc), _vp(uvw), _vp(offs), n,
                                        _vp(out))
        check(st, "degrid_execute_host")
        return out

    def grid(self, vis, uvw, vis_offsets, n_subgrids: int, out=None, accumulate: bool = False,
             stream=None):
        """Adjoint: complex64 [S, ny, nx, nz] from visibilities (grid_adjoint_execute)."""
        torch = _torch()
        n = self._common(uvw, vis_offsets, n_subgrids)
        _need(vis, "vis", torch.complex64, self.device, (n,))
        if out is None:
            out = torch.empty((n_subgrids,) + self.shape, dtype=torch.complex64, device=self.device)
            accumulate = False
        else:
            _need(out, "out", torch.complex64, self.device, (n_subgrids,) + self.shape)
        st = load().grid_adjoint_execute(self.handle, _stream_handle(stream, self.device),
                                         n_subgrids, _vp(uvw), _vp(vis_offsets), n, _vp(vis),
                                         _vp(out), int(bool(accumulate)))
        check(st, "grid_adjoint_execute")
        return out

    def coords(self, uvw, out=None, stream=None):
        """int32 [N, 6] = (x0, y0, z0, fu, fv, fw), -1 rows for invalid."""
        torch = _torch()
        _need(uvw, "uvw", torch.float64, self.device)
        if uvw.dim() != 2 or uvw.shape[1] != 3:
            raise ValueError("uvw must be [N, 3] float64")
        n = uvw.shape[0]
        if out is None:
            out = torch.empty((n, 6), dtype=torch.int32, device=self.device)
        else:
            _need(out, "out", torch.int32, self.device, (n, 6))
        st = load().degrid_coords_execute(self.handle, _stream_handle(stream, self.device),
                                          _vp(uvw), n, _vp(out))
        check(st, "degrid_coords_execute")
        return out

    def status(self, stream=None) -> int:
        """Synchronise and return (then clear) the invalid-visibility count.

        Raises DegridError(DG_ERR_OFFSETS) if a call saw malformed offsets.
        """
        n = ctypes.c_int64()
        st = load().degrid_get_status(self.handle, _stream_handle(stream, self.device),
                                      ctypes.byref(n))
        check(st, "degrid_get_status")
        return int(n.value)


def pack_subgrids(subgrids, dtype: str, stream=None):
    """complex64 [S, ny, nx, nz] -> (codes [S, ny, nx, nz, 2] in float16 or
    bfloat16, scale float32 [S]) via degrid_pack_subgrids."""
    torch = _torch()
    if dtype not in ("f16", "bf16"):
        raise ValueError("dtype must be 'f16' or 'bf16'")
    if subgrids.dtype != torch.complex64 or not subgrids.is_contiguous() or not subgrids.is_cuda:
        raise ValueError("subgrids must be a contiguous complex64 CUDA tensor")
    S = subgrids.shape[0]
    elems = subgrids[0].numel() if S else 0
    tdt = torch.float16 if dtype == "f16" else torch.bfloat16
    codes = torch.empty(tuple(subgrids.shape) + (2,), dtype=tdt, device=subgrids.device)
    scale = torch.empty(S, dtype=torch.float32, device=subgrids.device)
    st = load().degrid_pack_subgrids(_stream_handle(stream, subgrids.device), DTYPES[dtype], S,
                                     elems, _vp(subgrids), _vp(codes), _vp(scale))
    check(st, "degrid_pack_subgrids")
    return codes, scale


def measure_fp32_peak(device: int = 0, packed: bool = True) -> float:
    """FP32 FMA throughput of `device` in TFLOP/s, measured by
    degrid_measure_fp32_peak (packed FFMA2 chains, or scalar FFMA)."""
    out = ctypes.c_double(0.0)
    check(load().degrid_measure_fp32_peak(int(device), 1 if packed else 0, ctypes.byref(out)),
          "degrid_measure_fp32_peak")
    return float(out.value)


def measure_l2_read_bw(device: int = 0) -> float:
    """L2-to-SM read bandwidth of `device` in GB/s, measured by
    degrid_measure_l2_read_bw."""
    out = ctypes.c_double(0.0)
    check(load().degrid_measure_l2_read_bw(int(device), ctypes.byref(out)),
          "degrid_measure_l2_read_bw")
    return float(out.value)


def measure_l2_reduce_bw(device: int = 0) -> float:
    """Rate of tensor reduce-adds of 2 KB footprint tiles into an L2-resident
    stack, GB/s of added data (degrid_measure_l2_reduce_bw)."""
    out = ctypes.c_double(0.0)
    check(load().degrid_measure_l2_reduce_bw(int(device), ctypes.byref(out)),
          "degrid_measure_l2_reduce_bw")
    return float(out.value)


def degrid(plan: DegridPlan, subgrids, uvw, vis_offsets, scale=None):
    """Functional form of DegridPlan.degrid."""
    return plan.degrid(subgrids, uvw, vis_offsets, scale=scale)


def _make_fn():
    torch = _torch()

    class DegridFn(torch.autograd.Function):
        """vis = Degrid(subgrids); backward returns Grid(grad_vis).

        The degridding weights are real, so the adjoint needs no conjugation
        and, with PyTorch's convention for complex gradients
        (grad = dL/dRe + i dL/dIm), the gradient of a real loss with respect
        to the subgrids is the gridding of the visibility gradient.
        """

        @staticmethod
        def forward(ctx, subgrids, uvw, vis_offsets, plan):
            ctx.plan = plan
            ctx.n_subgrids = subgrids.shape[0]
            ctx.save_for_backward(uvw, vis_offsets)
            return plan.degrid(subgrids, uvw, vis_offsets)

        @staticmethod
        def backward(ctx, grad_vis):
            uvw, vis_offsets = ctx.saved_tensors
            grad = ctx.plan.grid(grad_vis.contiguous(), uvw, vis_offsets, ctx.n_subgrids)
            return grad, None, None, None

    return DegridFn


class _LazyFn:
    _fn = None

    def __getattr__(self, name):
        if _LazyFn._fn is None:
            _LazyFn._fn = _make_fn()
        return getattr(_LazyFn._fn, name)


DegridFn = _LazyFn()


def autotune(plan: DegridPlan, subgrids, uvw, vis_offsets, scale=None, **kw):
    """Time tuning candidates on the given inputs and keep the fastest."""
    from .tune import autotune as _autotune
    return _autotune(plan, subgrids, uvw, vis_offsets, scale=scale, **kw)


class SubgridPredictor:
    """The subgrid stack from an N x N sky image (subgrid_predict_execute):
    for subgrid s the cells (x - N/2 + u0_s, y - N/2 + v0_s) / theta of the
    w-planes w0_s + c dw_s, c < nz, of the tapered image's w-stacked
    Fourier transform, complex64 [S, N, N, nz] -- the layout DegridPlan
    reads.

    n, nz              image / subgrid side and w-planes per subgrid
    subgrids_per_pass  subgrids transformed together (work buffer size)
    device             CUDA device
    """

    def __init__(self, n: int = 512, nz: int = 4, subgrids_per_pass: int = 16, device=None):
        torch = _torch()
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        device = torch.device(device)
        if device.type != "cuda":
            raise ValueError("SubgridPredictor needs a CUDA device")
        if device.index is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device, self.n, self.nz = device, int(n), int(nz)
        h = ctypes.c_void_p()
        check(load().subgrid_predict_plan_create(ctypes.byref(h), self.n, self.nz, int(subgrids_per_pass),
                                                 device.index), "subgrid_predict_plan_create")
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            load().subgrid_predict_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def predict(self, image, theta: float, uv_offsets, w_planes, taper=None, out=None, stream=None):
        """image complex64 [N, N]; uv_offsets int32 [S, 2]; w_planes float64
        [S, 2] (w0, dw); taper float32 [N, N] or None -- all on the device."""
        torch = _torch()
        if self._h is None:
            raise RuntimeError("SubgridPredictor is closed")
        n = self.n
        _need(image, "image", torch.complex64, self.device, (n, n))
        if taper is not None:
            _need(taper, "taper", torch.float32, self.device, (n, n))
        _need(uv_offsets, "uv_offsets", torch.int32, self.device)
        S = uv_offsets.shape[0]
        if tuple(uv_offsets.shape) != (S, 2):
            raise ValueError("uv_offsets must be [S, 2] int32")
        _need(w_planes, "w_planes", torch.float64, self.device, (S, 2))
        if out is None:
            out = torch.empty((S, n, n, self.nz), dtype=torch.complex64, device=self.device)
        else:
            _need(out, "out", torch.complex64, self.device, (S, n, n, self.nz))
        st = load().subgrid_predict_execute(self._h, _stream_handle(stream, self.device), float(theta),
                                            _vp(image), _vp(taper), S, _vp(uv_offsets), _vp(w_planes),
                                            _vp(out))
        check(st, "subgrid_predict_execute")
        return out
