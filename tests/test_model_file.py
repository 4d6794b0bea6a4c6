"""The packaged predictor: layout and provenance (CPU only)."""
import json
import os

import numpy as np

import oracle.learned as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MODEL = os.path.join(ROOT, "paper_1908_11740_gb300", "models", "block_pairs_mlp.npz")


def test_packaged_model_layout_and_header():
    d = np.load(MODEL, allow_pickle=False)
    p = d["params"]
    assert p.dtype == np.float32 and p.shape == (L.PARAMS,)
    assert np.all(np.isfinite(p))
    h = json.loads(str(d["header"]))
    assert h["features"] == "eq2-histograms-k8-phi16-overlap-buckets-v1"
    assert "seed 29" in h["eval"]["workload"]        # evaluated on a seed it was not trained on
    assert "20-27" in h["train_joins"]


def test_packaged_model_predicts_sensible_counts():
    # a block with no entries spread over the buckets predicts few pairs; a
    # denser block (all buckets 100x) predicts more
    d = np.load(MODEL, allow_pickle=False)
    p = d["params"].astype(np.float64)
    lo = np.full((1, L.FEAT), np.log1p(2.0))
    hi = np.full((1, L.FEAT), np.log1p(200.0))
    assert L.mlp_forward(p, hi)[0] > L.mlp_forward(p, lo)[0]
