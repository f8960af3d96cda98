"""Host logic of the batch autotuner: shape classes, the choice of the
fastest candidate and the cache file (no GPU)."""
import json

from paper_2407_10914_gb300 import autotune as A


def test_shape_class_rounds_to_two_digits():
    k1 = A.shape_class(19, "fp32", [(123456, 7890), (1000, 10)])
    k2 = A.shape_class(19, "fp32", [(124000, 7900), (490, 0)])
    assert k1 == k2 == "Q19-fp32-n2-F120000-S7900"
    assert A.shape_class(19, "fp16", [(5, 0)]) == "Q19-fp16-n1-F5-S0"
    assert A.shape_class(9, "fp32", [(0, 0)]).startswith("Q9-fp32-n1-F0")


def test_fastest_prefers_least_time_then_candidate_order():
    t = {c: 1.0 for c in A.CANDIDATES}
    assert A.fastest(t) == A.CANDIDATES[0]
    t[A.CANDIDATES[3]] = 0.5
    assert A.fastest(t) == A.CANDIDATES[3]


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    assert A.load_cache(p) == {}
    A.store_cache(p, "k1", {"config": [1, 256, 4], "ms_per_step": 2.0})
    A.store_cache(p, "k2", {"config": [0, 128, 1], "ms_per_step": 3.0})
    d = json.load(open(p))
    assert d["k1"]["config"] == [1, 256, 4] and d["k2"]["ms_per_step"] == 3.0
    open(p, "w").write("not json")
    assert A.load_cache(p) == {}


def test_tile_class_and_cached_tile(tmp_path):
    """The tile search's key and its cache: a cached shape among the
    candidates is returned without building or timing anything; one that
    is not a candidate is ignored."""
    key = A.tile_class(19, "fp32", (256, 256, 256), [(4588847, 2561392)])
    assert key == "tile-Q19-fp32-256x256x256-n1-F4600000-S2600000"
    p = str(tmp_path / "t.json")
    A.store_cache(p, key, {"tile": [64, 8, 8], "ms_per_step": 0.5,
                           "trials": {"64x8x8": 0.5}})

    def make(tile):
        raise AssertionError("a cached shape needs no trial")

    r = A.tune_tile(make, 19, key=key, cache_path=p)
    assert r["cached"] and r["tile"] == (64, 8, 8)
    A.store_cache(p, key, {"tile": [16, 4, 4], "ms_per_step": 0.5})
    built = []

    def make2(tile):
        built.append(tile)
        raise RuntimeError("stop")

    try:
        A.tune_tile(make2, 19, key=key, cache_path=p)
    except RuntimeError:
        pass
    assert built == [A.TILE_CANDIDATES[19][0]]
    assert all(t[0] >= 32 for q in A.TILE_CANDIDATES
               for t in A.TILE_CANDIDATES[q])
