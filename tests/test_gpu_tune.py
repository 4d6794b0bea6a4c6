"""Autotuner on the GPU: measured choice, cache hit, and the tuned join is exact."""
import os

import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_tuner_measures_caches_and_stays_exact(tmp_path):
    from paper_1908_11740_gb300 import build, sj, tune

    build.build()
    ctx = sj.sj_create(0)
    try:
        R, S = inputs.gis_pair(60_000, 90_000, seed=41, median_extent=5e-4)
        dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
        m = tune.mean_extent(ctx, dR, dS)
        want_m = float((R[:, 2] - R[:, 0]).sum() + (R[:, 3] - R[:, 1]).sum() + (S[:, 2] - S[:, 0]).sum()
                       + (S[:, 3] - S[:, 1]).sum()) / (2 * (len(R) + len(S)))
        assert abs(m - want_m) <= 1e-6 * want_m
        best, results = tune.measure(ctx, dR, dS, factors=(0.5, 1.0, 2.0), blocks=(768, 1536), reps=1)
        assert len(results) == 6 and best["rule_k"] == tune.rule_k(m)
        cache = tune.Cache(os.path.join(tmp_path, "t.json"))
        g1, b1 = tune.tuned(ctx, dR, dS, cache=cache, device_name="test")
        g2, b2 = tune.tuned(ctx, dR, dS, cache=cache, device_name="test", measure_if_missing=False)
        assert (g1.nx, b1) == (g2.nx, b2)
        sj.sj_set_tuning(ctx, b1)
        got = sj.sj_join(ctx, dR, dS, g1).cpu().numpy()
        got = got[np.lexsort((got[:, 1], got[:, 0]))]
        np.testing.assert_array_equal(got, oracle.pbsm(R, S, 64))
    finally:
        sj.sj_destroy(ctx)
