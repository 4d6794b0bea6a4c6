"""Allocation failure through the C ABI: a context whose allocator refuses
requests beyond a byte budget (a host-side cap, no GPU fault) returns
SJ_ENOMEM from every join entry point that needs more, and the context stays
usable: with its allocator restored, the same joins return the oracle's
pairs."""
import numpy as np
import pytest

import oracle
from paper_1908_11740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sorted(t):
    a = t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def test_capped_allocator_gives_enomem_and_context_survives():
    from paper_1908_11740_gb300 import build, sj

    build.build()
    lib = sj.load()
    ctx = sj.sj_create(0)
    base = ctx.allocator
    used = {}
    budget = [1 << 20]   # 1 MiB

    def alloc(nbytes, user):
        if sum(used.values()) + int(nbytes) > budget[0]:
            return None                  # refused: the library must report SJ_ENOMEM
        p = base._alloc(nbytes, user)
        used[p] = int(nbytes)
        return p

    def free(ptr, user):
        used.pop(int(ptr or 0), None)
        base._free(ptr, user)

    a_cb, f_cb = sj.ALLOC_FN(alloc), sj.FREE_FN(free)
    try:
        R, S = inputs.gis_pair(300_000, 500_000, seed=52, median_extent=2e-4)
        want = oracle.pbsm(R, S, 500)
        dR, dS = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
        g = sj.make_grid(500)
        sj._check(ctx.handle, lib.sj_set_allocator(ctx.handle, a_cb, f_cb, None))
        for call in (lambda: sj.sj_join(ctx, dR, dS, g),
                     lambda: sj.sj_count(ctx, dR, dS, g),
                     lambda: sj.sj_join(ctx, dR, dS, g, sj.make_opts("one_pass_heur"))):
            with pytest.raises(sj.SJError) as e:
                call()
            assert e.value.status == sj.SJ_ENOMEM
        # a larger budget that still holds the join works under the cap
        budget[0] = 4 << 30
        np.testing.assert_array_equal(_sorted(sj.sj_join(ctx, dR, dS, g)), want)
        assert sum(used.values()) <= budget[0]
        # the default allocator back: the context joins as before
        sj._check(ctx.handle, lib.sj_set_allocator(ctx.handle, base.alloc_cb, base.free_cb, None))
        np.testing.assert_array_equal(_sorted(sj.sj_join(ctx, dR, dS, g)), want)
        assert sj.sj_count(ctx, dR, dS, g) == len(want)
    finally:
        lib.sj_set_allocator(ctx.handle, base.alloc_cb, base.free_cb, None)
        sj.sj_destroy(ctx)
