"""The batch autotuner's host logic: candidates, choice, cache round trip."""

from paper_2508_01864_gb300 import batch


def test_candidates_and_pick():
    assert batch.candidates(16) == [16, 8, 4, 2, 1]
    assert batch.candidates(3) == [3, 1]
    assert batch.pick({16: 2.0, 8: 1.5, 4: 1.5, 2: 3.0}) == 8  # ties go to more rhs per CTA


def test_key_and_cache_round_trip(tmp_path, monkeypatch):
    k1 = batch.tune_key("GB300", 16, ["d1nu0.5", "d2nu1.5", "d1nu0.5"], 100000)
    k2 = batch.tune_key("GB300", 16, ["d2nu1.5", "d1nu0.5", "d1nu0.5"], 120000)
    assert k1 == k2  # order-free mix, same size bucket
    assert batch.tune_key("GB300", 8, ["d1nu0.5"], 100000) != k1
    path = tmp_path / "cache.json"
    monkeypatch.setenv("FGK_AUTOTUNE_CACHE", str(path))
    assert batch.load_cache() == {}
    batch.store_cache({k1: {"rhs_per_cta": 4}})
    batch.store_cache({"other": {"rhs_per_cta": 1}})
    c = batch.load_cache()
    assert c[k1]["rhs_per_cta"] == 4 and c["other"]["rhs_per_cta"] == 1
