"""The autotuner's search (coordinate descent over the launch-shape knobs, a change kept only
when it is at least 1.5% faster) and its per-shape cache, on a stand-in context whose step
times come from a cost function of its tuning: host logic only, no GPU."""

import json

import pytest

from paper_2212_00476_gb300 import autotune as AT
from paper_2212_00476_gb300 import zncc as Z


class FakeCtx:
    """What the tuner uses of a context: its shape, its tuning calls and its run call."""

    def __init__(self, W=64, H=32, D=16, win=9):
        self.W, self.H, self.D, self.win = W, H, D, win
        self.stream = None
        self.tuning = {}
        self.runs = 0

    def set_tuning(self, key, value):
        self.tuning[key] = value

    def zncc_run(self, *args):
        self.runs += 1


def install_timer(monkeypatch, cost):
    """Replaces the CUDA-event timer: a timing is cost(settings by name) of the context's current
    tuning (None for a shape the launch cannot use); returns the list of timed settings."""
    timed = []

    def fake_time(ctx, run, reps):
        run()
        settings = {AT.NAMES[k]: v for k, v in ctx.tuning.items()}
        timed.append(settings)
        return cost(settings)

    monkeypatch.setattr(AT, "_time", fake_time)
    return timed


def tune(ctx, path, **kw):
    return AT.tune(ctx, None, None, None, 20.0, 0.1, 3, Z.ZNCC_F32, cache=str(path), **kw)


BEST = {"row_minb2": 1, "row_spb": 4, "h_tq": 4, "v_tq": 0, "v_lpc": 2, "line_loads": 2, "ahat_join": 0}


def separable(settings):
    """1 ms plus 0.05 ms for every knob away from BEST (ample against the 1.5% threshold)."""
    return 1.0 + sum(0.05 for name, best in BEST.items() if settings.get(name, 0) != best)


def test_every_candidate_key_has_a_name_that_apply_maps_back():
    assert set(AT.CANDIDATES) <= set(AT.NAMES)
    for key, values in AT.CANDIDATES.items():
        assert 0 in values                      # the search starts from the automatic shapes
        ctx = FakeCtx()
        AT.apply(ctx, {AT.NAMES[key]: values[-1]})
        assert ctx.tuning == {key: values[-1]}


def test_coordinate_descent_finds_the_best_of_a_separable_landscape(monkeypatch, tmp_path):
    install_timer(monkeypatch, separable)
    ctx = FakeCtx()
    res = tune(ctx, tmp_path / "t.json")
    assert res["settings"] == BEST
    assert res["ms"] == pytest.approx(1.0)
    assert {AT.NAMES[k]: v for k, v in ctx.tuning.items()} == BEST     # left applied


def test_gains_below_the_threshold_are_not_taken(monkeypatch, tmp_path):
    # h_tq = 2 is 1% faster (below 1.5%), v_lpc = 2 is 3% faster
    def cost(s):
        return 1.0 - (0.01 if s.get("h_tq") == 2 else 0.0) - (0.03 if s.get("v_lpc") == 2 else 0.0)

    install_timer(monkeypatch, cost)
    res = tune(FakeCtx(), tmp_path / "t.json")
    assert res["settings"]["h_tq"] == 0
    assert res["settings"]["v_lpc"] == 2


def test_shapes_a_launch_cannot_use_are_skipped(monkeypatch, tmp_path):
    # eight lanes per chunk would be fastest but cannot launch; four is the best that can
    def cost(s):
        if s.get("h_tq") == 8:
            return None
        return {0: 1.0, 2: 0.95, 4: 0.9}[s.get("h_tq", 0)]

    install_timer(monkeypatch, cost)
    res = tune(FakeCtx(), tmp_path / "t.json")
    assert res["settings"]["h_tq"] == 4


def test_results_are_cached_per_shape_and_reapplied(monkeypatch, tmp_path):
    timed = install_timer(monkeypatch, separable)
    path = tmp_path / "t.json"
    first = tune(FakeCtx(), path)
    n = len(timed)
    assert n > 0
    data = json.loads(path.read_text())
    key = AT.shape_key(FakeCtx(), 3, Z.ZNCC_F32)
    assert data[key]["settings"] == BEST

    ctx = FakeCtx()                             # same shape: applied from the cache, not timed
    again = tune(ctx, path)
    assert len(timed) == n and again == first
    assert {AT.NAMES[k]: v for k, v in ctx.tuning.items()} == BEST

    tune(FakeCtx(W=128), path)                  # another shape: searched and stored beside it
    assert len(timed) > n
    assert len(json.loads(path.read_text())) == 2

    m = len(timed)
    tune(FakeCtx(), path, force=True)           # force: searched again
    assert len(timed) > m
