"""Host logic of the schedule autotuner: coordinate descent over the knobs,
the wall-time budget, and the per-shape cache (the device timing is replaced
by a function of the knobs; no GPU involved)."""

import json

import numpy as np

import workloads as W
from paper_1104_0623_gb300 import tune


def fake_cost(params):
    # best at leaf 10, 64x64 tiles above 64, group 16, no shared-memory inversion
    tiles = abs(np.log2(params["gemm_small_max"]) - 6) if params["gemm_small_max"] else 3.0
    return (abs(params["leaf"] - 10) + tiles
            + abs(np.log2(params["energy_group"]) - 4) + params["invert_smem"] / 112 + 1.0)


def make_tuner(tmp_path, monkeypatch, calls):
    t = tune.Tuner(cache_path=str(tmp_path / "tune.json"))
    monkeypatch.setattr(t, "_device_name", lambda: "fake-gpu")

    def fake_time(mesh, energies, precision, batch, params, V=None):
        calls.append(dict(params))
        return fake_cost(params)
    monkeypatch.setattr(t, "_time", fake_time)
    return t


def test_coordinate_descent_finds_the_best_knobs_and_caches_them(tmp_path, monkeypatch):
    calls = []
    t = make_tuner(tmp_path, monkeypatch, calls)
    mesh = W.c3()[0]
    E = W.c3_energies()
    best = t.tune(mesh, E, "mixed_ff", 16)
    assert best == {"leaf": 10, "gemm_small_max": 64, "energy_group": 16, "invert_smem": 0}
    # every candidate is timed once; the default first
    assert calls[0] == tune.DEFAULTS
    assert len(calls) == len({tuple(sorted(c.items())) for c in calls})
    n = len(calls)
    # cached: a second call times nothing, and a new tuner reads the file
    assert t.tune(mesh, E, "mixed_ff", 16) == best and len(calls) == n
    calls2 = []
    t2 = make_tuner(tmp_path, monkeypatch, calls2)
    assert t2.tune(mesh, E, "mixed_ff", 16) == best and calls2 == []
    entry = json.load(open(tmp_path / "tune.json"))[t.key(mesh, "mixed_ff", 16)]
    assert entry["seconds_per_energy"] <= entry["default_seconds_per_energy"]
    # another shape or precision is tuned separately
    t.tune(W.c3()[1], E, "mixed_ff", 16)
    t.tune(mesh, E, "fp64", 16)
    assert len(json.load(open(tmp_path / "tune.json"))) == 3


def test_budget_stops_the_search_with_a_valid_choice(tmp_path, monkeypatch):
    calls = []
    t = make_tuner(tmp_path, monkeypatch, calls)
    t.budget_s = 0.0
    best = t.tune(W.c3()[0], W.c3_energies(), "mixed", 8)
    assert best == tune.DEFAULTS and len(calls) == 1
