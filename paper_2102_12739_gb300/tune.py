"""Autotuner for the persistent degridding kernel.

The paper picks N_b, the visibilities per thread block, by hand and finds
that the best value depends on the step du, dv, dw while N_b = 32 is good
enough, and it switches between kernel variants by list length (Section
"Results").  Here the knobs are the chunk size (visibilities per work item),
warps per CTA, resident CTAs per SM and the summing arm (footprint cache only;
the direct per-visibility arm for halves with many short runs, which wins
when footprints overlap but their w rows change often; or the gather kernel,
which streams every footprint through shared memory and wins when footprints
are scattered); this module times a
small grid of candidates on the caller's own inputs with CUDA events and
keeps the fastest on the plan.  Results are cached in a JSON file
keyed by GPU name, storage type and a coarse description of the inputs, so a
later call with similar inputs reuses them without timing.

The cache file is ``$DEGRID_TUNE_CACHE`` if set, else
``~/.cache/gb300_degrid/tune.json``; ``DEGRID_TUNE=0`` disables timing (the
cache is still read).
"""
from __future__ import annotations

import json
import math
import os
from typing import Iterable, Optional

NEVER = 33          # DG_DIRECT_RUNS_NEVER
SHORT = 9           # DG_DIRECT_RUNS_SHORT

DEFAULT_CANDIDATES = [
    (chunk, warps, 0, direct, 0)
    for chunk in (128, 256, 512, 1024)
    for warps in (4, 8)
    for direct in (NEVER, SHORT)
] + [(chunk, 8, 0, NEVER, 1) for chunk in (128, 256, 512)]

_KEYS = ("chunk", "warps_per_block", "blocks_per_sm", "direct_runs", "gather")


def _apply(plan, t: dict) -> None:
    plan.set_tuning(t["chunk"], t["warps_per_block"], t["blocks_per_sm"])
    plan.set_direct_runs(t.get("direct_runs", NEVER))
    plan.set_gather(bool(t.get("gather", 0)))


def _cache_path() -> str:
    return os.environ.get("DEGRID_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gb300_degrid", "tune.json"))


def _load_cache() -> dict:
    try:
        with open(_cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store_cache(cache: dict) -> None:
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def cache_key(plan, n_subgrids: int, n_vis: int) -> str:
    """GPU, storage type, G_uv table kind, reduction, subgrid shape and the
    orders of magnitude of S and N."""
    import torch
    name = torch.cuda.get_device_name(plan.device)
    ny, nx, nz = plan.shape
    return "%s|%s|%s|%s|%dx%dx%d|S~2^%d|N~2^%d" % (
        name, plan.dtype, "2d" if getattr(plan, "table2d", False) else "sep",
        "comp" if plan.compensated else "plain", ny, nx, nz,
        int(math.log2(max(n_subgrids, 1))), int(math.log2(max(n_vis, 1))))


def autotune(plan, subgrids, uvw, vis_offsets, scale=None,
             candidates: Optional[Iterable] = None, iters: int = 5, use_cache: bool = True):
    """Time `candidates` (chunk, warps_per_block, blocks_per_sm[, direct_runs[,
    gather]]) and keep the best; a candidate without direct_runs or gather
    keeps the plan's.  Candidates the plan cannot run (the gather kernel on a
    plan with a 2D table) are skipped.

    Returns {"tuning": {...}, "ms": best median kernel ms, "timings": [...]}.
    """
    import torch
    S = int(vis_offsets.shape[0]) - 1
    n = int(uvw.shape[0])
    key = cache_key(plan, S, n)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        before = plan.tuning()
        try:
            _apply(plan, cache[key]["tuning"])
            return dict(cache[key], tuning=plan.tuning(), cached=True)
        except Exception:
            # a tuning this plan cannot take (an old or foreign entry): the
            # part of it already applied is undone, then it is timed again
            _apply(plan, before)
    if os.environ.get("DEGRID_TUNE", "1") == "0":
        return {"tuning": plan.tuning(), "ms": None, "timings": [], "cached": False}
    cands = list(candidates) if candidates is not None else list(DEFAULT_CANDIDATES)
    before_timing = plan.tuning()
    out = torch.empty(n, dtype=torch.complex64, device=plan.device)
    plan.enable_timing(max(iters, 1))
    timings = []
    try:
        for cand in cands:
            chunk, warps, bps = cand[:3]
            direct = cand[3] if len(cand) > 3 else plan.direct_runs
            gather = int(cand[4]) if len(cand) > 4 else int(plan.gather)
            try:
                _apply(plan, {"chunk": chunk, "warps_per_block": warps, "blocks_per_sm": bps,
                              "direct_runs": direct, "gather": gather})
            except Exception:
                _apply(plan, before_timing)
                continue
            for _ in range(2):                      # warm-up (also sizes scratch)
                plan.degrid(subgrids, uvw, vis_offsets, scale=scale, out=out)
            for _ in range(iters):
                plan.degrid(subgrids, uvw, vis_offsets, scale=scale, out=out)
            ms = sorted(plan.kernel_times_ms(iters))
            timings.append({"chunk": chunk, "warps_per_block": warps, "blocks_per_sm": bps,
                            "direct_runs": direct, "gather": gather, "ms": ms[len(ms) // 2]})
    finally:
        plan.enable_timing(0)
    if not timings:
        raise RuntimeError("autotune: no candidate could be timed")
    best = min(timings, key=lambda t: t["ms"])
    _apply(plan, best)
    result = {"tuning": {k: best[k] for k in _KEYS}, "ms": best["ms"], "timings": timings}
    if use_cache:
        cache[key] = {"tuning": result["tuning"], "ms": result["ms"]}
        _store_cache(cache)
    return dict(result, cached=False)
