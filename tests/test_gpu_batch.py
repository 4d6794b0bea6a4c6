"""Batched joins (sj_join_batch): every join of the batch against the
oracle, uneven sizes, explicit and rule-of-thumb grids, repeated calls that
replay the captured graphs, a too-small output buffer."""
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


@pytest.fixture(scope="module")
def ctx(sj):
    c = sj.sj_create(0)
    yield c
    sj.sj_destroy(c)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def srt(a):
    a = np.asarray(a, np.int32).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def _batch():
    joins = inputs.batch_pairs(n_joins=12, seed0=4000, n_min=50, n_max=30_000, median_extent=2e-3)
    joins.append(inputs.degenerate_pair(300, 200, seed=9))
    joins.append((np.zeros((0, 4), np.float32), inputs.uniform_pair(10, 10, seed=1)[1]))
    return joins


@pytest.mark.parametrize("grids_kind", ["explicit", "rule"])
def test_batch_matches_oracle(sj, ctx, grids_kind):
    joins = _batch()
    Rs = [dev(r) for r, _ in joins]
    Ss = [dev(s) for _, s in joins]
    grids = [sj.make_grid(k) for k in (8, 16, 33, 64, 5, 100, 3, 1, 40, 20, 7, 128, 9, 4)] \
        if grids_kind == "explicit" else None
    for rep in range(3):            # the second and third call replay the graphs
        pairs, offs = sj.sj_join_batch(ctx, Rs, Ss, grids)
        torch.cuda.synchronize()
        got = pairs.cpu().numpy()
        for j, (r, s) in enumerate(joins):
            want = oracle.brute(r, s) if len(r) * len(s) < 2e7 else oracle.sweep(r, s)
            np.testing.assert_array_equal(srt(got[offs[j]:offs[j + 1]]), want)


def test_batch_overflow_reports_offsets(sj, ctx):
    joins = _batch()[:4]
    Rs = [dev(r) for r, _ in joins]
    Ss = [dev(s) for _, s in joins]
    small = torch.empty((1, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(sj.SJError) as e:
        sj.sj_join_batch(ctx, Rs, Ss, None, out=small)
    assert e.value.status == sj.SJ_EOVERFLOW
    pairs, offs = sj.sj_join_batch(ctx, Rs, Ss, None)
    assert offs[-1] == sum(len(oracle.sweep(r, s)) for r, s in joins)


@pytest.mark.parametrize("kind", ["learned", "eq2", "undersized"])
def test_batch_one_pass_matches_oracle(sj, ctx, kind):
    """One-pass sizing of the whole batch: every join's range equals the
    oracle, with the packaged model, the Eq. 2 estimate, and a model that
    predicts no pairs (every block re-run exactly)."""
    import oracle.learned as L

    from paper_1908_11740_gb300 import learn

    joins = _batch()
    Rs = [dev(r) for r, _ in joins]
    Ss = [dev(s) for _, s in joins]
    model = None
    try:
        if kind == "learned":
            model, _ = learn.load(ctx)
            sj.sj_set_model(ctx, model)
            opts = sj.make_opts("one_pass")
        elif kind == "eq2":
            opts = sj.make_opts("one_pass_heur")
        else:
            model = sj.Model(ctx, np.zeros(L.PARAMS, np.float32))
            sj.sj_set_model(ctx, model)
            opts = sj.make_opts("one_pass", margin=0.0)
        for rep in range(2):
            pairs, offs = sj.sj_join_batch(ctx, Rs, Ss, None, opts=opts)
            st = sj.sj_last_stats(ctx)
            assert st["one_pass"] == 1
            if kind == "undersized":
                assert st["refit_items"] > 0
            got = pairs.cpu().numpy()
            for j, (r, s) in enumerate(joins):
                want = oracle.brute(r, s) if len(r) * len(s) < 2e7 else oracle.sweep(r, s)
                np.testing.assert_array_equal(srt(got[offs[j]:offs[j + 1]]), want)
        small = torch.empty((1, 2), dtype=torch.int32, device="cuda")
        with pytest.raises(sj.SJError) as e:
            sj.sj_join_batch(ctx, Rs, Ss, None, out=small, opts=opts)
        assert e.value.status == sj.SJ_EOVERFLOW
    finally:
        sj.sj_set_model(ctx, None)
        if model is not None:
            model.free()


@pytest.mark.parametrize("mode", ["two_pass", "one_pass_heur"])
def test_batch_sorted_output(sj, ctx, mode):
    """sort_output on a batch: every join's range comes back in (r, s) order,
    exactly the oracle's sorted pairs (no sorting on the host), in both
    sizing modes; a batch whose tiles exceed shared memory (joined join by
    join) is sorted the same way."""
    joins = _batch()
    Rs = [dev(r) for r, _ in joins]
    Ss = [dev(s) for _, s in joins]
    pairs, offs = sj.sj_join_batch(ctx, Rs, Ss, None, opts=sj.make_opts(mode, sort_output=True))
    got = pairs.cpu().numpy()
    for j, (r, s) in enumerate(joins):
        want = oracle.brute(r, s) if len(r) * len(s) < 2e7 else oracle.sweep(r, s)
        np.testing.assert_array_equal(got[offs[j]:offs[j + 1]], want)
    # hot tiles beyond shared memory in one join of the batch
    hot = inputs.zipf_pair(40_000, 40_000, seed=77, lattice=64, r_max_extent=1e-4, s_max_extent=1e-3, rho=0.02)
    mix = [joins[0], hot, joins[1]]
    pairs, offs = sj.sj_join_batch(ctx, [dev(r) for r, _ in mix], [dev(s) for _, s in mix],
                                   [sj.make_grid(k) for k in (16, 64, 16)], opts=sj.make_opts(mode, sort_output=True))
    got = pairs.cpu().numpy()
    for j, (r, s) in enumerate(mix):
        np.testing.assert_array_equal(got[offs[j]:offs[j + 1]], oracle.pbsm(r, s, 16 if j != 1 else 64))


@pytest.mark.parametrize("variant", [{"axis": "adaptive"}, {"dedup": "gbda"}])
@pytest.mark.parametrize("mode", ["two_pass", "one_pass_heur"])
def test_batch_sweep_options(sj, ctx, mode, variant):
    """The adaptive sweep axis and GBDA on a batch (each join's own grid for
    the Eq. 2 buckets): every join's range equals the oracle's pairs, the
    graphs of the option are their own (a plain batch after it is exact too)."""
    joins = _batch()
    joins.append(inputs.aniso_pair(20_000, 30_000, seed=91))
    Rs = [dev(r) for r, _ in joins]
    Ss = [dev(s) for _, s in joins]
    for opts in (sj.make_opts(mode, **variant), sj.make_opts(mode)):
        pairs, offs = sj.sj_join_batch(ctx, Rs, Ss, None, opts=opts)
        got = pairs.cpu().numpy()
        for j, (r, s) in enumerate(joins):
            want = oracle.brute(r, s) if len(r) * len(s) < 2e7 else oracle.sweep(r, s)
            np.testing.assert_array_equal(srt(got[offs[j]:offs[j + 1]]), want)
