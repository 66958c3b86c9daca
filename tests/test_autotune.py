"""Host logic of the launch-configuration autotuner: coordinate search over the knobs with
a stand-in timing function, the JSON cache (problem key, shape-level fall-back, atomic
writes) and the application of a cached choice to muster_params."""
import json
import os

import pytest

from paper_2412_14671_gb300 import autotune

SHAPE, N = (40, 48, 40), 4
PARAMS = dict(n_levels=2, window=5, n_squarings=6, deterministic=1)


def cost(p):
    # a stand-in device: flow_nf 1 is 10 % faster, chunk_pct 200 5 % faster, half batches slower
    ms = 100.0
    if p.get("flow_nf") == 1:
        ms *= 0.9
    if p.get("chunk_pct") == 200:
        ms *= 0.95
    if p.get("chunk_pct") == 400:
        ms *= 0.99  # below the 2 % threshold against 200
    if p.get("pair_batch"):
        ms *= 1.2
    return ms


def test_coordinate_search_and_cache(tmp_path):
    path = str(tmp_path / "tune.json")
    calls = []

    def measure(p):
        calls.append(p)
        return cost(p)

    res = autotune.tune(SHAPE, N, PARAMS, path=path, measure=measure)
    assert not res["cached"]
    assert res["choice"] == {"flow_nf": 1, "chunk_pct": 200, "pair_batch": "all"}
    assert res["ms"] == pytest.approx(100.0 * 0.9 * 0.95)
    # default, flow_nf 1, chunk 50/200/400, half batch
    assert len(calls) == 6 and len(res["trials"]) == 6
    # cached: no measurement the second time
    calls.clear()
    again = autotune.tune(SHAPE, N, PARAMS, path=path, measure=measure)
    assert again["cached"] and again["choice"] == res["choice"] and not calls
    data = json.load(open(path))
    key = autotune.problem_key(SHAPE, N, PARAMS, autotune.device_name())
    assert key in data and autotune.problem_key(SHAPE, None, PARAMS, autotune.device_name()) in data


def test_lookup_falls_back_to_the_shape_and_params_apply(tmp_path):
    path = str(tmp_path / "tune.json")
    autotune.tune(SHAPE, N, PARAMS, path=path, measure=cost)
    assert autotune.lookup(SHAPE, N, PARAMS, path) == {"flow_nf": 1, "chunk_pct": 200, "pair_batch": "all"}
    # another session count of the same shape takes the shape-level entry
    assert autotune.lookup(SHAPE, 7, PARAMS, path)["chunk_pct"] == 200
    # another window is another problem
    assert autotune.lookup(SHAPE, N, dict(PARAMS, window=7), path) is None
    p = autotune.tuned_params(SHAPE, N, PARAMS, path)
    assert p["flow_nf"] == 1 and p["chunk_pct"] == 200 and p["pair_batch"] == 0
    # explicit settings win over the cache
    assert autotune.tuned_params(SHAPE, N, dict(PARAMS, chunk_pct=50), path)["chunk_pct"] == 50
    # no entry: params unchanged
    assert autotune.tuned_params((8, 8, 8), 3, PARAMS, path) == PARAMS


def test_knob_params_and_keys():
    assert autotune.knob_params({"pair_batch": "half"}, 5) == {"pair_batch": 10}
    assert autotune.knob_params({"pair_batch": "all", "flow_nf": 2}, 5) == {"pair_batch": 0, "flow_nf": 2}
    k1 = autotune.problem_key(SHAPE, N, PARAMS, "dev")
    k2 = autotune.problem_key(SHAPE, N, dict(PARAMS, lr=0.3, alpha_ss=2.0), "dev")
    assert k1 == k2  # step sizes and weights do not change the launch configuration
    assert autotune.problem_key(SHAPE, N, dict(PARAMS, deterministic=0), "dev") != k1


def test_tune_needs_images_or_a_measure(tmp_path):
    with pytest.raises(ValueError):
        autotune.tune(SHAPE, N, PARAMS, path=str(tmp_path / "t.json"))


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert autotune.load_cache(str(path)) == {}
    res = autotune.tune(SHAPE, N, PARAMS, path=str(path), measure=cost)
    assert not res["cached"] and os.path.exists(path)
