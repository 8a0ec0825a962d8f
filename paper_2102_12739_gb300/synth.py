"""Seeded synthetic workloads for 3D degridding.

This module only *generates inputs*: subgrid stacks, per-subgrid visibility
coordinate lists, the precomputed oversampled GCF tables and adjoint
visibilities.  It holds none of the degridding arithmetic (no snapping of
coordinates, no footprint sums), so both the CUDA path and the FP64 oracle
can consume its outputs without sharing any of the method's code.

Shapes follow the paper's statement of the problem (Section "Implementation"):
S subgrids of 512 x 512 x 4 complex samples, a uv GCF of support 8 x 8 and a
w GCF of support 4, and per subgrid a list of N_vis,S coordinates [u, v, w].
The paper's tests put the visibilities of a subgrid on a line with constant
du, dv, dw; the batched workload adds segments and circular arcs so that the
visibility counts per subgrid spread over three orders of magnitude (the
load-balancing scenario of the paper's Results section, Fig. 2).

Conventions (also used by the library):
  * subgrid stack: complex64 C-order [S][ny][nx][nz], y <-> v, x <-> u,
    z <-> w;
  * coordinates: float64 [N][3] = (u, v, w) in subgrid pixel units, origin at
    element (0, 0, 0); lists of consecutive subgrids are concatenated and
    delimited by int64 ``vis_offsets`` [S + 1];
  * GCF tables: float64 [oversample][support]; row f, column k holds the
    kernel value at grid offset (k - support/2 + 1) - f/oversample.

Seeds: subgrids 0, coordinates 1, counts and list structure 2, adjoint
visibilities 3, the sky image of the subgrid producer 4.  Each subgrid / list draws from its own stream
``default_rng([seed, s])`` so that any one of them can be regenerated alone.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SEED_SUBGRID = 0
SEED_UVW = 1
SEED_STRUCTURE = 2
SEED_ADJOINT = 3
SEED_SKY = 4

UV_SUPPORT = 8
UV_OVERSAMPLE = 16384
W_SUPPORT = 4
W_OVERSAMPLE = 128
# Kaiser-Bessel shape parameter: 2.3 x support (uv from the workload
# definition; the same rule is applied to w).
UV_BETA = 2.3 * UV_SUPPORT
W_BETA = 2.3 * W_SUPPORT

SUBGRID_SHAPE = (512, 512, 4)  # (ny, nx, nz)
# Sampling box that keeps every 8x8x4 footprint inside a 512x512x4 subgrid
# with half a pixel of margin: start = floor(snap(q)) - 3 must lie in
# [0, n - 8], and for w the footprint must cover planes 0..3.
W_LO, W_HI = 1.0, 1.99


def uv_box(n: int) -> tuple[float, float]:
    """Sampling interval for u (n = nx) or v (n = ny)."""
    return 3.5, n - 4.5


# ---------------------------------------------------------------------------
# GCF tables (precomputed inputs, "Implementation" section bullet list)
# ---------------------------------------------------------------------------

def bessel_i0(x: np.ndarray) -> np.ndarray:
    """Modified Bessel function I0 by its power series sum_k ((x/2)^k / k!)^2.

    Evaluated term by term in float64 until the terms stop changing the sum;
    for the arguments used here (|x| <= 20) about 50 terms suffice.
    """
    x = np.asarray(x, dtype=np.float64)
    half = 0.5 * x
    term = np.ones_like(x)
    total = np.ones_like(x)
    for k in range(1, 200):
        term = term * (half / k) ** 2
        total = total + term
        if np.all(term <= 1e-18 * total):
            break
    return total


def kaiser_bessel(x: np.ndarray, support: int, beta: float) -> np.ndarray:
    """Peak-normalised Kaiser-Bessel window on |x| <= support/2, else 0."""
    x = np.asarray(x, dtype=np.float64)
    t = 2.0 * x / support
    inside = np.abs(x) <= support / 2
    arg = beta * np.sqrt(np.clip(1.0 - t * t, 0.0, None))
    return np.where(inside, bessel_i0(arg) / bessel_i0(np.array(beta)), 0.0)


def gcf_table(support: int, oversample: int, beta: float) -> np.ndarray:
    """Oversampled 1D GCF table, float64 [oversample][support].

    Row f, column k: KB((k - support/2 + 1) - f/oversample).
    """
    f = np.arange(oversample, dtype=np.float64)[:, None]
    k = np.arange(support, dtype=np.float64)[None, :]
    offs = (k - support // 2 + 1) - f / oversample
    return np.ascontiguousarray(kaiser_bessel(offs, support, beta))


def gcf_table_2d(support: int, oversample: int, beta: float) -> np.ndarray:
    """Oversampled non-separable G_uv: a circularly symmetric Kaiser-Bessel
    kernel, float64 [oversample][oversample][support][support] indexed
    [fv][fu][b][a], holding KB(sqrt(x^2 + y^2)) at x = (a - support/2 + 1) -
    fu/oversample, y = (b - support/2 + 1) - fv/oversample (0 beyond radius
    support/2)."""
    f = np.arange(oversample, dtype=np.float64)
    k = np.arange(support, dtype=np.float64)
    off = (k[None, :] - support // 2 + 1) - f[:, None] / oversample        # [f][k]
    y = off[:, None, :, None]                                             # [fv][1][b][1]
    x = off[None, :, None, :]                                             # [1][fu][1][a]
    r = np.sqrt(x * x + y * y)
    return np.ascontiguousarray(kaiser_bessel(r, support, beta))


TABLE2D_OVERSAMPLE = 64


def default_table_2d(oversample: int = TABLE2D_OVERSAMPLE) -> np.ndarray:
    """Circular Kaiser-Bessel G_uv table [O][O][8][8] (beta as the 1D table)."""
    return gcf_table_2d(UV_SUPPORT, oversample, UV_BETA)


def default_tables() -> tuple[np.ndarray, np.ndarray]:
    """(g_uv [16384][8], g_w [128][4]) Kaiser-Bessel tables, float64."""
    return (gcf_table(UV_SUPPORT, UV_OVERSAMPLE, UV_BETA),
            gcf_table(W_SUPPORT, W_OVERSAMPLE, W_BETA))


# ---------------------------------------------------------------------------
# Subgrids
# ---------------------------------------------------------------------------

def subgrid(s: int, shape=SUBGRID_SHAPE, seed: int = SEED_SUBGRID) -> np.ndarray:
    """Subgrid s: i.i.d. complex Gaussian (Re, Im ~ N(0, 1)), complex64."""
    rng = np.random.default_rng([seed, s])
    re_im = rng.standard_normal(size=tuple(shape) + (2,), dtype=np.float32)
    return re_im.view(np.complex64)[..., 0]


def subgrid_stack(n_subgrids: int, shape=SUBGRID_SHAPE, seed: int = SEED_SUBGRID,
                  out: Optional[np.ndarray] = None) -> np.ndarray:
    """Stack of subgrids, complex64 [S][ny][nx][nz]."""
    if out is None:
        out = np.empty((n_subgrids,) + tuple(shape), dtype=np.complex64)
    for s in range(n_subgrids):
        out[s] = subgrid(s, shape, seed)
    return out


# ---------------------------------------------------------------------------
# Coordinate lists
# ---------------------------------------------------------------------------

def _uniform_point(rng, shape):
    ny, nx, _ = shape
    ulo, uhi = uv_box(nx)
    vlo, vhi = uv_box(ny)
    return np.array([rng.uniform(ulo, uhi), rng.uniform(vlo, vhi),
                     rng.uniform(W_LO, W_HI)])


def line(n: int, start: np.ndarray, end: np.ndarray) -> np.ndarray:
    """n points start + j * step, step = (end - start) / (n - 1), float64 [n][3]."""
    if n == 0:
        return np.zeros((0, 3))
    step = (end - start) / max(n - 1, 1)
    j = np.arange(n, dtype=np.float64)[:, None]
    return start[None, :] + j * step[None, :]


def random_line(n: int, rng, shape=SUBGRID_SHAPE) -> np.ndarray:
    """The paper's test list: a line with random start and constant step."""
    start = _uniform_point(rng, shape)
    end = _uniform_point(rng, shape)
    return line(n, start, end)


def arc(n: int, rng, shape=SUBGRID_SHAPE) -> np.ndarray:
    """Circular arc in uv that lies wholly inside the sampling box; w linear."""
    ny, nx, _ = shape
    ulo, uhi = uv_box(nx)
    vlo, vhi = uv_box(ny)
    rmax = 0.5 * min(uhi - ulo, vhi - vlo)
    r = rng.uniform(min(5.0, 0.5 * rmax), rmax)
    cu = rng.uniform(ulo + r, uhi - r)
    cv = rng.uniform(vlo + r, vhi - r)
    th0 = rng.uniform(0.0, 2 * math.pi)
    span = rng.uniform(0.1, 2 * math.pi)
    w0, w1 = rng.uniform(W_LO, W_HI), rng.uniform(W_LO, W_HI)
    t = np.arange(n, dtype=np.float64) / max(n - 1, 1)
    th = th0 + span * t
    out = np.empty((n, 3))
    out[:, 0] = np.clip(cu + r * np.cos(th), ulo, uhi)
    out[:, 1] = np.clip(cv + r * np.sin(th), vlo, vhi)
    out[:, 2] = w0 + (w1 - w0) * t
    return out


def piecewise_list(n: int, rng, shape=SUBGRID_SHAPE) -> np.ndarray:
    """1-8 pieces, each a line segment or a circular arc (probability 1/2)."""
    k = int(rng.integers(1, 9))
    sizes = np.full(k, n // k, dtype=np.int64)
    sizes[: n % k] += 1
    pieces = []
    for m in sizes:
        if rng.uniform() < 0.5:
            pieces.append(random_line(int(m), rng, shape))
        else:
            pieces.append(arc(int(m), rng, shape))
    return np.concatenate(pieces, axis=0) if pieces else np.zeros((0, 3))


def scattered_list(n: int, rng, shape=SUBGRID_SHAPE) -> np.ndarray:
    """n points uniform in the valid box: no two consecutive visibilities
    share a footprint (sparse uv coverage)."""
    ny, nx, _ = shape
    ulo, uhi = uv_box(nx)
    vlo, vhi = uv_box(ny)
    return np.stack([rng.uniform(ulo, uhi, n), rng.uniform(vlo, vhi, n),
                     rng.uniform(W_LO, W_HI, n)], axis=1)


def offsets_from_counts(counts) -> np.ndarray:
    counts = np.asarray(counts, dtype=np.int64)
    out = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=out[1:])
    return out


def adjoint_vis(n_vis: int, seed: int = SEED_ADJOINT) -> np.ndarray:
    """Seeded complex Gaussian visibilities for the adjoint, complex64 [N]."""
    rng = np.random.default_rng(seed)
    re_im = rng.standard_normal(size=(n_vis, 2), dtype=np.float32)
    return re_im.view(np.complex64)[:, 0].copy()


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    """Inputs of one degridding call (everything except the subgrid data).

    ``subgrids()`` materialises the complex64 stack on demand (it can be
    several GB); ``subgrid(s)`` regenerates one subgrid alone.
    """
    name: str
    n_subgrids: int
    shape: tuple
    uvw: np.ndarray          # float64 [N][3]
    vis_offsets: np.ndarray  # int64 [S + 1]
    ids: Optional[np.ndarray] = None   # global subgrid ids (a shard of a larger job)

    @property
    def n_vis(self) -> int:
        return int(self.vis_offsets[-1])

    def counts(self) -> np.ndarray:
        return np.diff(self.vis_offsets)

    def subgrid(self, s: int) -> np.ndarray:
        return subgrid(int(self.ids[s]) if self.ids is not None else s, self.shape)

    def subgrids(self) -> np.ndarray:
        if self.ids is None:
            return subgrid_stack(self.n_subgrids, self.shape)
        out = np.empty((self.n_subgrids,) + tuple(self.shape), dtype=np.complex64)
        for s in range(self.n_subgrids):
            out[s] = self.subgrid(s)
        return out

    def subgrid_nbytes(self, elem_bytes: int = 8) -> int:
        ny, nx, nz = self.shape
        return self.n_subgrids * ny * nx * nz * elem_bytes


def lines_workload(name: str, counts, shape=SUBGRID_SHAPE, ids=None) -> Workload:
    """Every subgrid's list is its own random line (the paper's test case).

    With `ids`, the subgrids are those global ids of a larger job (their
    values and lists are the ones that job would have).
    """
    counts = [int(c) for c in counts]
    gid = list(range(len(counts))) if ids is None else [int(i) for i in ids]
    parts = [random_line(c, np.random.default_rng([SEED_UVW, g]), shape)
             for g, c in zip(gid, counts)]
    uvw = np.ascontiguousarray(np.concatenate(parts, axis=0)) if parts else np.zeros((0, 3))
    return Workload(name, len(counts), tuple(shape), uvw, offsets_from_counts(counts),
                    None if ids is None else np.asarray(gid, dtype=np.int64))


def scattered_workload(name: str, counts, shape=SUBGRID_SHAPE) -> Workload:
    """Every subgrid's list is scattered uniformly over the valid box."""
    counts = [int(c) for c in counts]
    parts = [scattered_list(c, np.random.default_rng([SEED_UVW, s]), shape)
             for s, c in enumerate(counts)]
    uvw = np.ascontiguousarray(np.concatenate(parts, axis=0)) if parts else np.zeros((0, 3))
    return Workload(name, len(counts), tuple(shape), uvw, offsets_from_counts(counts))


def batched_counts(n_subgrids: int, lo: float = 1e3, hi: float = 1e6) -> np.ndarray:
    """Visibility counts log-uniform in [lo, hi], rounded to integers."""
    rng = np.random.default_rng(SEED_STRUCTURE)
    e = rng.uniform(math.log10(lo), math.log10(hi), size=n_subgrids)
    return np.rint(10.0 ** e).astype(np.int64)


def batched_workload(name: str, n_subgrids: int, lo: float = 1e3, hi: float = 1e6,
                     shape=SUBGRID_SHAPE) -> Workload:
    """Uneven load: log-uniform counts, lists of segments and arcs."""
    counts = batched_counts(n_subgrids, lo, hi)
    parts = [piecewise_list(int(c), np.random.default_rng([SEED_UVW, s]), shape)
             for s, c in enumerate(counts)]
    uvw = np.ascontiguousarray(np.concatenate(parts, axis=0))
    return Workload(name, n_subgrids, tuple(shape), uvw, offsets_from_counts(counts))


def workload(name: str) -> Workload:
    """Named workloads.

    line1_20k      1 subgrid, 20,000 visibilities on one line
    lines64_250k   64 subgrids, 250,000 visibilities each (16M): the
                   throughput workload
    lines16_250k   its first 16 subgrids (4M visibilities; profiling case)
    batched512     512 subgrids, log-uniform counts in [1e3, 1e6]
    batched64      64 subgrids of the same recipe (profiling case)
    diff32_100k    32 subgrids, 100,000 visibilities each (adjoint)
    scatter16_250k 16 subgrids, 250,000 scattered visibilities each (4M; no
                   footprint shared by consecutive visibilities)
    """
    if name == "line1_20k":
        return lines_workload(name, [20_000])
    if name == "lines64_250k":
        return lines_workload(name, [250_000] * 64)
    if name == "lines16_250k":
        return lines_workload(name, [250_000] * 16)
    if name == "batched512":
        return batched_workload(name, 512)
    if name == "batched64":
        return batched_workload(name, 64)
    if name == "diff32_100k":
        return lines_workload(name, [100_000] * 32)
    if name == "scatter16_250k":
        return scattered_workload(name, [250_000] * 16)
    raise KeyError(name)


# ---- inputs of the subgrid producer (the step upstream of degridding) -----

def sky_image(n: int = 512, n_sources: int = 300, seed: int = SEED_SKY) -> np.ndarray:
    """A model sky, complex64 [n][n] (row <-> m, column <-> l): point sources
    of log-uniform flux in [1e-3, 1] at random pixels plus weak Gaussian
    background, with a small imaginary part (a polarisation-like leak)."""
    rng = np.random.default_rng(seed)
    img = (1e-4 * rng.standard_normal((n, n)) + 1e-5j * rng.standard_normal((n, n)))
    b = rng.integers(0, n, n_sources)
    a = rng.integers(0, n, n_sources)
    flux = 10.0 ** rng.uniform(-3, 0, n_sources)
    np.add.at(img, (b, a), flux * (1 + 0.01j * rng.standard_normal(n_sources)))
    return img.astype(np.complex64)


def image_taper(n: int = 512) -> np.ndarray:
    """A smooth positive image-plane correction, float32 [n][n] (an input of
    the producer like the image: the inverse of a separable bell)."""
    x = (np.arange(n) - n // 2) / (n / 2)
    bell = np.cos(0.45 * np.pi * x) ** 2 + 0.05
    return (1.0 / np.outer(bell, bell)).astype(np.float32)


PREDICT_THETA = 0.1             # image width in direction cosines (about 5.7 degrees)


def predict_offsets(n_subgrids: int, dw: float = 100.0):
    """Subgrid parameters of the producer workload: every subgrid the full
    n x n cell window (u0 = v0 = 0) of one stack of w-planes, the stacks
    consecutive (w0_s = (s - S/2) * 4 dw, planes dw apart): int32 [S][2]
    and float64 [S][2]."""
    uv = np.zeros((n_subgrids, 2), dtype=np.int32)
    w = np.stack([(np.arange(n_subgrids) - n_subgrids // 2) * 4.0 * dw, np.full(n_subgrids, dw)], axis=1)
    return uv, np.ascontiguousarray(w, dtype=np.float64)


# ---- inputs generated on the device ----------------------------------------
# For sizes the host should not hold (stacks of thousands of subgrids, more
# than 2^31 visibilities).  The values are inputs like the rest: tests copy
# the rows and subgrids they check back to the host and hand them to the
# oracle.  torch is imported here only, so the module stays numpy-only for
# the oracle's users.

def subgrid_stack_on_device(n_subgrids: int, device, shape=SUBGRID_SHAPE, seed: int = SEED_SUBGRID):
    """complex64 [S][ny][nx][nz] on `device`, i.i.d. complex Gaussian (torch's
    generator for that device, seeded)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    return torch.randn((n_subgrids,) + tuple(shape) + (2,), generator=gen, device=device,
                       dtype=torch.float32).view(torch.complex64)[..., 0].contiguous()


_SLAB = 1 << 27     # rows per temporary: 1 GiB of float64


def fill_line_on_device(uvw, lo: int, n: int, start, end) -> None:
    """Rows [lo, lo + n) of the device tensor uvw (float64 [N][3]) := the line
    start + j * step, step = (end - start) / (n - 1), as in `line`."""
    import torch
    step = [(float(e) - float(s)) / max(n - 1, 1) for s, e in zip(start, end)]
    for a in range(0, n, _SLAB):
        m = min(_SLAB, n - a)
        j = torch.arange(a, a + m, dtype=torch.float64, device=uvw.device)
        for k in range(3):
            uvw[lo + a: lo + a + m, k] = j * step[k] + float(start[k])


def fill_scattered_on_device(uvw, lo: int, n: int, shape=SUBGRID_SHAPE, seed: int = SEED_UVW) -> None:
    """Rows [lo, lo + n) of uvw := points uniform in the valid box, as in
    `scattered_list` (torch's generator for the device, seeded)."""
    import torch
    ny, nx, _ = shape
    box = (uv_box(nx), uv_box(ny), (W_LO, W_HI))
    gen = torch.Generator(device=uvw.device)
    gen.manual_seed(seed)
    for a in range(0, n, _SLAB):
        m = min(_SLAB, n - a)
        r = torch.rand((m, 3), dtype=torch.float64, device=uvw.device, generator=gen)
        for k in range(3):
            r[:, k] = r[:, k] * (box[k][1] - box[k][0]) + box[k][0]
        uvw[lo + a: lo + a + m] = r


def random_line_on_device(uvw, lo: int, n: int, rng, shape=SUBGRID_SHAPE) -> None:
    """Rows [lo, lo + n) of uvw := a line with random ends, as in `random_line`."""
    start = _uniform_point(rng, shape)
    end = _uniform_point(rng, shape)
    fill_line_on_device(uvw, lo, n, start, end)
