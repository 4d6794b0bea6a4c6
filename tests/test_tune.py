"""Autotuner host logic (CPU): the rule of thumb, buckets and the cache."""
import os

from paper_1908_11740_gb300 import tune


def test_rule_of_thumb():
    # tiles about ten times the average extent: mean extent 3.3e-5 -> K ~ 3000
    assert tune.rule_k(3.3e-5) == 3030
    assert tune.rule_k(1e-3) == 100
    assert tune.rule_k(0.0) == 8192 and tune.rule_k(10.0) == 1


def test_buckets_group_similar_inputs():
    assert tune.bucket(30_000_000, 3.3e-5) == tune.bucket(20_000_000, 3.1e-5)
    assert tune.bucket(30_000_000, 3.3e-5) != tune.bucket(3_000_000, 3.3e-5)
    assert tune.bucket(30_000_000, 3.3e-5) != tune.bucket(30_000_000, 3.3e-4)


def test_cache_roundtrip(tmp_path):
    p = os.path.join(tmp_path, "c", "tune.json")
    c = tune.Cache(p)
    assert c.get("GB300", "k") is None
    c.put("GB300", "k", {"factor": 0.71, "block_target": 768})
    c2 = tune.Cache(p)
    assert c2.get("GB300", "k") == {"factor": 0.71, "block_target": 768}
    assert c2.get("other", "k") is None
