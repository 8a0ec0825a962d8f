"""The autotuner's on-disk cache (host logic, no GPU): a cached tuning is
reused without timing when the plan can take it, and timed again when it
cannot (an entry the plan rejects, such as the gather kernel for a plan with
a 2D G_uv table); a corrupted cache file reads as empty."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2102_12739_gb300 import DegridError, tune  # noqa: E402


class FakePlan:
    """The plan calls the autotuner makes; refuses the gather kernel."""

    def __init__(self):
        self.device = torch.device("cpu")
        self.t = {"chunk": 256, "warps_per_block": 8, "blocks_per_sm": 0, "direct_runs": 33, "gather": False}
        self.timed = 0

    def set_tuning(self, chunk, warps, bps):
        self.t.update(chunk=chunk, warps_per_block=warps, blocks_per_sm=bps)

    def set_direct_runs(self, n):
        self.t["direct_runs"] = n

    def set_gather(self, on):
        if on:
            raise DegridError(6, "degrid_plan_set_gather")
        self.t["gather"] = False

    def tuning(self):
        return dict(self.t)

    def enable_timing(self, n):
        pass

    def degrid(self, *a, **k):
        self.timed += 1

    def kernel_times_ms(self, n):
        return [0.5 if self.t["chunk"] == 128 else 1.0] * n


@pytest.fixture
def cache_file(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("DEGRID_TUNE_CACHE", str(path))
    monkeypatch.setattr(tune, "cache_key", lambda plan, S, n: "key")
    return path


def call(plan):
    offs = np.array([0, 10], dtype=np.int64)
    uvw = np.zeros((10, 3))
    return tune.autotune(plan, None, uvw, offs, candidates=[(256, 8, 0, 33, 0), (128, 4, 0, 33, 0)], iters=2)


def test_a_usable_cached_tuning_is_reused_without_timing(cache_file):
    cache_file.write_text(json.dumps({"key": {"tuning": {"chunk": 512, "warps_per_block": 4, "blocks_per_sm": 0,
                                                         "direct_runs": 9, "gather": 0}, "ms": 0.2}}))
    plan = FakePlan()
    r = call(plan)
    assert r["cached"] and plan.timed == 0
    assert plan.t["chunk"] == 512 and plan.t["warps_per_block"] == 4 and plan.t["direct_runs"] == 9


def test_a_cached_tuning_the_plan_rejects_is_timed_again(cache_file):
    cache_file.write_text(json.dumps({"key": {"tuning": {"chunk": 512, "warps_per_block": 8, "blocks_per_sm": 0,
                                                         "direct_runs": 33, "gather": 1}, "ms": 0.1}}))
    plan = FakePlan()
    r = call(plan)
    assert not r["cached"] and plan.timed > 0
    assert r["tuning"]["chunk"] == 128 and plan.t["chunk"] == 128
    stored = json.loads(cache_file.read_text())["key"]["tuning"]
    assert stored["chunk"] == 128 and stored["gather"] == 0


def test_a_corrupted_cache_file_reads_as_empty(cache_file):
    cache_file.write_text("{not json")
    plan = FakePlan()
    r = call(plan)
    assert not r["cached"] and r["tuning"]["chunk"] == 128
    assert json.loads(cache_file.read_text())["key"]["tuning"]["chunk"] == 128


def test_a_refused_cached_tuning_leaves_the_plan_as_it_was(cache_file, monkeypatch):
    # with timing disabled the autotuner returns the plan's own tuning: no
    # part of the refused entry (its chunk, warps or direct-arm threshold)
    # may stay applied
    monkeypatch.setenv("DEGRID_TUNE", "0")
    cache_file.write_text(json.dumps({"key": {"tuning": {"chunk": 1024, "warps_per_block": 4, "blocks_per_sm": 3,
                                                         "direct_runs": 9, "gather": 1}, "ms": 0.1}}))
    plan = FakePlan()
    before = plan.tuning()
    r = call(plan)
    assert not r["cached"] and plan.timed == 0
    assert plan.tuning() == before and r["tuning"] == before
