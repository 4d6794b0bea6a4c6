"""Parity at full size for the batched workload: 256 independent joins, per
side log-uniform in [1e3, 2e6] rectangles (about 1.35e8 in all), uniform and
Gaussian-mixture centres, log-normal extents (median 1e-4), joined in one
batched call with the grid of every join from the rule of thumb (tile extent
about 10x the average rectangle extent).  Every join's pair set is compared
with the single-threaded oracle PBSM, and a second call (which replays the
captured graphs) must return the same result, as must the learned one-pass
sizing of the whole batch with the packaged model."""
import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sj():
    from paper_1908_11740_gb300 import build, sj as binding

    build.build()
    return binding


def srt(a):
    a = np.asarray(a, np.int32).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def test_batch_256_full_size(sj):
    joins = inputs.batch_pairs(n_joins=256)
    assert sum(len(r) + len(s) for r, s in joins) > 1e8
    Rs = [torch.from_numpy(r).cuda() for r, _ in joins]
    Ss = [torch.from_numpy(s).cuda() for _, s in joins]
    from paper_1908_11740_gb300 import learn

    ctx = sj.sj_create(0)
    model, _ = learn.load(ctx)
    try:
        pairs, offs = sj.sj_join_batch(ctx, Rs, Ss, None)
        torch.cuda.synchronize()
        got = pairs.cpu().numpy()
        again, offs2 = sj.sj_join_batch(ctx, Rs, Ss, None)
        torch.cuda.synchronize()
        assert list(offs2) == list(offs)
        got2 = again.cpu().numpy()
        sj.sj_set_model(ctx, model)
        one, offs3 = sj.sj_join_batch(ctx, Rs, Ss, None, opts=sj.make_opts("one_pass"))
        st = sj.sj_last_stats(ctx)
        assert st["one_pass"] == 1 and list(offs3) == list(offs)
        got3 = one.cpu().numpy()
    finally:
        sj.sj_set_model(ctx, None)
        model.free()
        sj.sj_destroy(ctx)
    for j, (r, s) in enumerate(joins):
        # the oracle's result does not depend on its grid: 128 x 128 keeps it quick
        want = oracle.pbsm(r, s, 128)
        np.testing.assert_array_equal(srt(got[offs[j]:offs[j + 1]]), want, err_msg=f"join {j}")
        np.testing.assert_array_equal(srt(got2[offs[j]:offs[j + 1]]), want, err_msg=f"join {j} (replay)")
        np.testing.assert_array_equal(srt(got3[offs[j]:offs[j + 1]]), want, err_msg=f"join {j} (one-pass)")
