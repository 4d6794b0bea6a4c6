"""GPU parity of the learned result-count predictor and the one-pass join.

* block features and labels of the CUDA path against oracle/learned.py
  (features: float32 scaling and log1p on both sides, rtol 1e-5; labels:
  exact integer pair counts);
* the MLP forward and the gradient of its loss against the float64 oracle
  evaluated at the same (bf16-rounded) weights: fp32 accumulation in a
  different order bounds the difference, rtol 2e-3 on the loss gradient
  relative to its largest component, 1e-4 relative on outputs;
* training lowers the loss on a fixed set;
* the one-pass join (learned and Eq. 2 sizing, and a model forced to
  under-size so that blocks are re-run) returns exactly the oracle's pairs,
  through the library buffer, the host-buffer entry point and a caller
  buffer.
"""
import numpy as np
import pytest

import oracle
import oracle.learned as L
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


def sorted_pairs(t):
    a = t.cpu().numpy().astype(np.int32)
    return a[np.lexsort((a[:, 1], a[:, 0]))] if len(a) else a.reshape(0, 2)


def test_block_features_and_labels(sj, ctx):
    R, S = inputs.gis_pair(40_000, 60_000, seed=31, median_extent=1e-3)
    K = 200
    X, Y, B = sj.sj_block_features(ctx, dev(R), dev(S), sj.make_grid(K), with_blocks=True)
    G = sj.sj_last_stats(ctx)["block_side"]
    assert G >= 1 and X.shape[0] > 10
    want_f = L.block_features(R, S, K, K, G)
    want_l = L.block_labels(R, S, K, K, G)
    got_b = B.cpu().numpy()
    assert sorted(got_b.tolist()) == sorted(want_f.keys())
    Xc, Yc = X.cpu().numpy(), Y.cpu().numpy()
    for row, b in enumerate(got_b):
        np.testing.assert_allclose(Xc[row], want_f[int(b)], rtol=1e-5, atol=1e-6)
        assert int(round(np.expm1(float(Yc[row])))) == want_l[int(b)]


def test_block_labels_when_tiles_exceed_shared_memory(sj, ctx):
    """Skew-shaped input whose hottest tiles hold more entries than shared
    memory: the features still come from the two-level partition, the labels
    from the single-level path's per-tile counts; both equal the oracle's."""
    R, S = inputs.zipf_pair(200_000, 200_000, seed=35, lattice=256, r_max_extent=2e-3, s_max_extent=4e-3, rho=0.0)
    K = 400
    assert oracle.tile_counts(R, K).max() > 3072
    X, Y, B = sj.sj_block_features(ctx, dev(R), dev(S), sj.make_grid(K), with_blocks=True)
    G = sj.sj_last_stats(ctx)["block_side"]
    want_f = L.block_features(R, S, K, K, G)
    want_l = L.block_labels(R, S, K, K, G)
    got_b = B.cpu().numpy()
    assert sorted(got_b.tolist()) == sorted(want_f.keys())
    Xc, Yc = X.cpu().numpy(), Y.cpu().numpy()
    total = 0
    for row, b in enumerate(got_b):
        np.testing.assert_allclose(Xc[row], want_f[int(b)], rtol=1e-5, atol=1e-6)
        got = int(round(float(np.expm1(np.float64(Yc[row])))))
        assert abs(got - want_l[int(b)]) <= max(1, 1e-6 * want_l[int(b)])   # float32 log1p of large counts
        total += want_l[int(b)]
    assert total == len(oracle.pbsm(R, S, K))


def test_mlp_forward_and_gradient(sj, ctx):
    g = np.random.default_rng(5)
    p = g.normal(0, 0.2, L.PARAMS).astype(np.float32)
    m = sj.Model(ctx, p)
    try:
        _, pinf = m.get_params(inference=True)
        X = g.uniform(0, 6, (3000, L.FEAT)).astype(np.float32)
        Y = g.uniform(0, 5, 3000).astype(np.float32)
        out = m.forward(dev(X)).cpu().numpy()
        want = L.mlp_forward(pinf, X)
        np.testing.assert_allclose(out, want, rtol=1e-4, atol=1e-4 * np.abs(want).max())
        grad, loss = m.grad(dev(X), dev(Y))
        wl, wg = L.mlp_loss_grad(pinf, X, Y)
        assert abs(float(loss.item()) - wl) <= 1e-4 * wl
        gg = grad.cpu().numpy()
        assert np.max(np.abs(gg - wg)) <= 2e-3 * np.max(np.abs(wg))
        # bf16 rounding: the inference weights are the master weights rounded to bf16
        w = np.asarray(p[L.OFF_W1:L.OFF_B1], np.float32)
        bits = w.view(np.uint32)
        rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000).view(np.float32)
        np.testing.assert_array_equal(pinf[L.OFF_W1:L.OFF_B1], rounded)
    finally:
        m.free()


def test_training_lowers_the_loss(sj, ctx):
    from paper_1908_11740_gb300 import learn

    R, S = inputs.gis_pair(300_000, 600_000, seed=33, median_extent=1e-4)
    X, Y = sj.sj_block_features(ctx, dev(R), dev(S), sj.make_grid(600))
    model, hist = learn.train(ctx, X, Y, epochs=40, batch=512, lr=3e-3, verbose=False)
    try:
        assert hist[-1] < hist[0]
        pred = model.forward(X)
        mse = float(((pred - Y) ** 2).mean().item())
        var = float(((Y - Y.mean()) ** 2).mean().item())
        assert mse < 0.6 * var, (mse, var)
    finally:
        model.free()


@pytest.mark.parametrize("kind", ["eq2", "learned", "undersized"])
def test_one_pass_equals_oracle(sj, ctx, kind):
    R, S = inputs.gis_pair(500_000, 800_000, seed=34, median_extent=1e-4)
    g = sj.make_grid(800)
    want = oracle.pbsm(R, S, 800)
    model = None
    try:
        if kind == "eq2":
            opts = sj.make_opts("one_pass_heur", margin=0.1)
        else:
            p = np.zeros(L.PARAMS, np.float32)
            if kind == "learned":
                from paper_1908_11740_gb300 import learn
                X, Y = sj.sj_block_features(ctx, dev(R), dev(S), g)
                model, _ = learn.train(ctx, X, Y, epochs=20, batch=256, verbose=False)
            else:
                p[L.OFF_B3] = 0.0            # predicts 0 pairs everywhere: most blocks re-run
                model = sj.Model(ctx, p)
            sj.sj_set_model(ctx, model)
            opts = sj.make_opts("one_pass", margin=0.0 if kind == "undersized" else 0.25)
        got = sorted_pairs(sj.sj_join(ctx, dev(R), dev(S), g, opts))
        st = sj.sj_last_stats(ctx)
        np.testing.assert_array_equal(got, want)
        assert st["one_pass"] == 1
        if kind == "undersized":
            assert st["refit_items"] > 0
        # the host-buffer entry point and the caller buffer take the same path
        host = sj.sj_join_host(ctx, R, S, g, opts=opts).numpy()
        np.testing.assert_array_equal(sorted_pairs(torch.from_numpy(host)), want)
        buf = torch.empty((len(want) + 3, 2), dtype=torch.int32, device="cuda")
        n = sj.sj_join_into(ctx, dev(R), dev(S), g, buf, opts)
        torch.cuda.synchronize()
        assert n == len(want)
        np.testing.assert_array_equal(sorted_pairs(buf[:n]), want)
    finally:
        sj.sj_set_model(ctx, None)
        if model is not None:
            model.free()


def test_one_pass_without_model_is_rejected(sj, ctx):
    R, S = inputs.uniform_pair(1000, 1000, seed=3)
    with pytest.raises(sj.SJError) as e:
        sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(16), sj.make_opts("one_pass"))
    assert e.value.status == sj.SJ_EINVAL
    # SJ_AUTO without a model is the exact two-pass join
    got = sorted_pairs(sj.sj_join(ctx, dev(R), dev(S), sj.make_grid(16), sj.make_opts("auto")))
    np.testing.assert_array_equal(got, oracle.brute(R, S))
