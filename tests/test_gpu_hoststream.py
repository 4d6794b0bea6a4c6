"""sj_join_host_many: a sequence of joins from host buffers, each join's
input copy overlapping the previous join (copy stream, two staging buffers).
Every join's pairs must equal the oracle's; overflow of one join leaves the
others intact; staging grows between calls and the context stays usable."""
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


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def srt(a):
    a = np.asarray(a, np.int32).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def _joins():
    out = []
    for k, seed in enumerate((51, 52, 53)):
        R, S = inputs.gis_pair(150_000 * (k + 1), 200_000, seed=seed, median_extent=1e-4)
        out.append((R, S, 300 + 200 * k))
    R, S = inputs.uniform_pair(20_000, 30_000, max_extent=4e-3, seed=54)
    out.append((R, S, 64))
    out.append((np.zeros((0, 4), np.float32), S, 16))          # empty R
    R, S = inputs.degenerate_pair(seed=55)
    out.append((R, S, 8))
    return out


@pytest.mark.parametrize("mode", ["two_pass", "one_pass"])
def test_many_joins_equal_oracle(sj, ctx, mode):
    joins = _joins()
    wants = [oracle.pbsm(R, S, 50) for R, S, _ in joins]
    model = None
    if mode == "one_pass":
        from paper_1908_11740_gb300 import learn
        model, _ = learn.load(ctx, learn.DEFAULT_MODEL)
        sj.sj_set_model(ctx, model)
    try:
        outs = [torch.full((len(w) + 5, 2), -1, dtype=torch.int32).pin_memory() for w in wants]
        counts = sj.sj_join_host_many(ctx, [pinned(R) for R, _, _ in joins], [pinned(S) for _, S, _ in joins],
                                      [sj.make_grid(K) for _, _, K in joins], outs, sj.make_opts(mode))
        for w, o, c in zip(wants, outs, counts):
            assert c == len(w)
            np.testing.assert_array_equal(srt(o[:c].numpy()), w)
            assert (o[c:] == -1).all().item()
    finally:
        if model is not None:
            sj.sj_set_model(ctx, None)
            model.free()


def test_overflow_of_one_join(sj, ctx):
    joins = _joins()[:4]
    wants = [oracle.pbsm(R, S, 50) for R, S, _ in joins]
    caps = [len(w) for w in wants]
    caps[1] -= 1                                               # join 1 does not fit
    outs = [torch.zeros((c, 2), dtype=torch.int32).pin_memory() for c in caps]
    with pytest.raises(sj.SJError) as ei:
        sj.sj_join_host_many(ctx, [pinned(R) for R, _, _ in joins], [pinned(S) for _, S, _ in joins],
                             [sj.make_grid(K) for _, _, K in joins], outs)
    assert ei.value.status == sj.SJ_EOVERFLOW
    assert ei.value.required == [len(w) for w in wants]
    for i in (0, 2, 3):
        np.testing.assert_array_equal(srt(outs[i].numpy()), wants[i])
    assert (outs[1] == 0).all().item()


def test_growth_pageable_and_interleaving(sj, ctx):
    small = _joins()[3]
    R, S = inputs.gis_pair(1_500_000, 2_500_000, seed=56)
    big = (R, S, 1000)
    want_s, want_b = oracle.pbsm(small[0], small[1], 50), oracle.pbsm(R, S, 1000)
    for joins, wants in (([small], [want_s]), ([small, big, small], [want_s, want_b, want_s])):
        # pageable host memory works too (the copies then do not overlap)
        outs = [torch.zeros((len(w), 2), dtype=torch.int32) for w in wants]
        counts = sj.sj_join_host_many(ctx, [torch.from_numpy(j[0]) for j in joins],
                                      [torch.from_numpy(j[1]) for j in joins],
                                      [sj.make_grid(j[2]) for j in joins], outs)
        for w, o, c in zip(wants, outs, counts):
            np.testing.assert_array_equal(srt(o[:c].numpy()), w)
        got = sj.sj_join(ctx, torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda(), sj.make_grid(1000))
        np.testing.assert_array_equal(srt(got.cpu().numpy()), want_b)


def test_invalid_arguments_do_no_work(sj, ctx):
    R, S, K = _joins()[3]
    bad = sj.make_grid(0)
    with pytest.raises(sj.SJError) as ei:
        sj.sj_join_host_many(ctx, [pinned(R), pinned(R)], [pinned(S), pinned(S)], [sj.make_grid(K), bad],
                             [torch.zeros((10, 2), dtype=torch.int32)] * 2)
    assert ei.value.status == sj.SJ_EINVAL
    assert sj.sj_join_host_many(ctx, [], [], [], []) == []
