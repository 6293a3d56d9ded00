"""Host logic of the launch-shape autotuner (no GPU): candidate sets, the
choice of the fastest, and the on-disk cache (keyed by problem and GPU)."""
import json

import pytest
import torch

import paper_2210_12375_b300 as tode
from paper_2210_12375_b300 import tuning as at


def _field_and_inputs(B=1000, D=16):
    A = torch.zeros(B, D, D)
    y0 = torch.zeros(B, D)
    t0 = torch.zeros(B, dtype=torch.float64)
    t1 = torch.ones(B, dtype=torch.float64)
    return tode.Linear(A), y0, t0, t1


def test_candidates_cover_the_knobs():
    c = at.candidates("linear", 16, "fused")
    assert {o["group"] for o in c} == {4, 8, 16}
    assert {o["block"] for o in c} == {32, 64, 128, 256}
    assert {o["ctas_per_sm"] for o in c} == {0, 1, 2, 4}
    assert {o["order"] for o in c} == {0, 1}
    assert all("poll_every" in o for o in at.candidates("vdp", 2, "plain"))
    assert at.candidates("mlp", 32, "fused") == [{"order": 0}, {"order": 1}]
    wide = at.candidates("mlp", 64, "fused", with_adjoint=True)
    assert {(o["order"], o["ctas_per_sm"]) for o in wide} == {(0, 1), (0, 2), (1, 1), (1, 2)}


def test_autotune_picks_fastest_and_caches(tmp_path):
    at.set_cache_path(str(tmp_path / "tune.json"))
    at._mem.clear()
    try:
        f, y0, t0, t1 = _field_and_inputs()
        cost = lambda o: (1.0 + abs(o["group"] - 8) + 0.1 * o["ctas_per_sm"]
                          + abs(o["block"] - 128) / 1e4 - 0.01 * o["order"])
        best = at.autotune(f, y0, t0, t1, timer=cost)
        assert best == {"group": 8, "block": 128, "ctas_per_sm": 0, "order": 1}
        data = json.loads((tmp_path / "tune.json").read_text())
        (key, entry), = data.items()
        assert "linear|D16|B1024|float32|fused|fwd" in key
        assert entry["options"] == best and len(entry["tried"]) == 96

        def boom(o):
            raise AssertionError("the cache should answer")
        at._mem.clear()  # a new process: the file answers
        assert at.autotune(f, y0, t0, t1, timer=boom) == best
        assert at.autotune(f, y0[:900], t0[:900], t1[:900], timer=boom) == best  # same bucket
        with pytest.raises(AssertionError):
            at.autotune(f, y0, t0, t1, timer=boom, refresh=True)
    finally:
        at.set_cache_path(None)
        at._mem.clear()


def test_autotune_skips_refused_shapes(tmp_path):
    at.set_cache_path(None)
    at._mem.clear()
    f, y0, t0, t1 = _field_and_inputs(B=64)

    def picky(o):
        if o["group"] != 16:
            raise tode._abi.TodeError(tode._abi.TODE_EUNSUPPORTED, "test")
        return float(o["block"])
    assert at.autotune(f, y0, t0, t1, timer=picky)["group"] == 16
    at._mem.clear()
