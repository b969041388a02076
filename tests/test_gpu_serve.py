"""Serving loop (continuous batching): requests for several resident catalogs,
with and without the gradient flag and in both precisions, arrive while
others are on the GPU; each result must be what the same request gives when
evaluated alone.  Every hyperpoint of a batch is computed independently (one
block per (event, point), per-point selection partials and combine), so the
stated tolerance is met exactly: the test requires bitwise equality.
Also: cancellation, admission by HBM footprint, latency statistics."""
import numpy as np
import pytest

from synth import catalog as sc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chim():
    from paper_2504_02034_b300 import build
    build.build()
    import paper_2504_02034_b300 as pkg
    return pkg


def _cats():
    a = sc.config_catalog(2, variant=0, n_events=8, n_pe=800, n_inj=20000, gal_median=60)
    b = sc.config_catalog(2, variant=2, n_events=5, n_pe=600, n_inj=15000, gal_median=40,
                          kde_mode=sc.KDE_SINGLE_1D)
    return a, b


def _points(n, seed, xi0):
    return sc.make_hyperpoints(n, seed=seed, Xi0=xi0)


def test_results_alone_equal_results_in_the_mix(chim):
    ca, cb = _cats()
    with chim.Context(0) as ctx:
        ia, ib = ctx.load(ca), ctx.load(cb)
        rng = np.random.default_rng(7)
        reqs = []
        for r in range(24):
            cid = ia if r % 3 else ib
            n = int(np.exp(rng.uniform(0.0, np.log(40))))
            flags = (chim.SERVE_MIXED if rng.random() < 0.7 else 0) | (chim.SERVE_GRAD if rng.random() < 0.3 else 0)
            th = _points(n, 100 + r, 0.6 if cid == ia else 1.8)
            reqs.append((cid, th, flags))
        tickets = []
        for cid, th, flags in reqs:
            tickets.append(chim.chimera_serve_submit(ctx.h, cid, th, flags))
        out = [chim.chimera_serve_poll(ctx.h, t, th.shape[0], grad=bool(f & chim.SERVE_GRAD))
               for t, (_, th, f) in zip(tickets, reqs)]
        st = chim.chimera_serve_stats(ctx.h)
        assert st["completed"] == len(reqs)
        assert st["points"] == sum(th.shape[0] for _, th, _ in reqs)
        assert 0.0 < st["p50_ms"] <= st["p99_ms"]
        # some requests were batched together
        assert st["batches"] < len(reqs)
        for (cid, th, flags), (lnL, g, status) in zip(reqs, out):
            prec = chim.MIXED if flags & chim.SERVE_MIXED else chim.FP64
            if flags & chim.SERVE_GRAD:
                lnL1, g1, st1 = ctx.grad(cid, th, prec)
                assert np.array_equal(g, g1)
            else:
                lnL1, _, st1 = ctx.loglike(cid, th, prec)
            assert np.array_equal(lnL, lnL1)
            assert np.array_equal(status, st1)


def test_cancel_and_unknown_ticket(chim):
    ca, _ = _cats()
    with chim.Context(0) as ctx:
        cid = ctx.load(ca)
        big = _points(256, 11, 0.6)
        # saturate the lanes with slow gradient requests of distinct keys
        busy = [chim.chimera_serve_submit(ctx.h, cid, big, f)
                for f in (chim.SERVE_GRAD, chim.SERVE_GRAD | chim.SERVE_MIXED, chim.SERVE_GRAD,
                          chim.SERVE_GRAD | chim.SERVE_MIXED)]
        victim = chim.chimera_serve_submit(ctx.h, cid, big[:3], 0)
        chim.chimera_serve_cancel(ctx.h, victim)
        with pytest.raises(chim.ChimeraError) as e:
            chim.chimera_serve_poll(ctx.h, victim, 3)
        assert e.value.code == chim.CHIMERA_ERR_CANCELLED
        for t in busy:
            chim.chimera_serve_poll(ctx.h, t, 256, grad=True)
        with pytest.raises(chim.ChimeraError) as e:
            chim.chimera_serve_poll(ctx.h, victim, 3)
        assert e.value.code == chim.CHIMERA_ERR_NOT_FOUND


def test_admission_by_hbm_footprint(chim):
    ca, _ = _cats()
    with chim.Context(0) as probe:
        cid = probe.load(ca)
        info = probe.info(cid)
    prof = 8 * info["n_pixels"] * info["n_z"] * 2
    budget = info["device_bytes"] + prof + 24 * 2 ** 20
    with chim.Context(0, hbm_budget_bytes=budget) as ctx:
        cid = ctx.load(ca)
        small = _points(2, 21, 0.6)
        t = chim.chimera_serve_submit(ctx.h, cid, small, chim.SERVE_MIXED)
        lnL, _, st = chim.chimera_serve_poll(ctx.h, t, 2)
        assert np.all(np.isfinite(lnL))
        big = _points(512, 22, 0.6)
        t = chim.chimera_serve_submit(ctx.h, cid, big, chim.SERVE_MIXED)
        with pytest.raises(chim.ChimeraError) as e:
            chim.chimera_serve_poll(ctx.h, t, 512)
        assert e.value.code == chim.CHIMERA_ERR_ADMISSION
        # the loop keeps serving after a refused request
        t = chim.chimera_serve_submit(ctx.h, cid, small, chim.SERVE_MIXED)
        lnL2, _, _ = chim.chimera_serve_poll(ctx.h, t, 2)
        assert np.array_equal(lnL, lnL2)


def test_cache_of_one_catalog_makes_room_for_another(chim):
    """The per-Om galaxy-profile caches of catalog A fill the budget; a later
    call on catalog B that needs a larger workspace frees A's least recently
    used entries instead of failing, and both catalogs' results stay those of
    a context without a budget."""
    ca, cb = _cats()
    with chim.Context(0) as probe:
        ia, ib = probe.load(ca), probe.load(cb)
        fa, fb = probe.info(ia), probe.info(ib)
        pa = _points(16, 31, 1.0)
        pb = _points(64, 32, 1.0)
        ref_a, _, _ = probe.loglike(ia, pa, chim.MIXED)
        ref_b, _, _ = probe.loglike(ib, pb, chim.MIXED)
    per_entry = 4 * fa["n_pixels"] * fa["n_z"]
    room = 32 * 2 ** 20
    budget = fa["device_bytes"] + fb["device_bytes"] + room
    with chim.Context(0, hbm_budget_bytes=budget) as ctx:
        ia, ib = ctx.load(ca), ctx.load(cb)
        rng = np.random.default_rng(33)
        # more distinct Om values than the room holds profiles of catalog A
        for _ in range(int(2 * room / (16 * per_entry)) + 2):
            t = pa.copy()
            t[:, 1] = 0.2 + 0.2 * rng.random(16)
            lnL, _, _ = ctx.loglike(ia, t, chim.MIXED)
            assert np.all(np.isfinite(lnL))
        lnL_b, _, _ = ctx.loglike(ib, pb, chim.MIXED)
        np.testing.assert_array_equal(lnL_b, ref_b)
        lnL_a, _, _ = ctx.loglike(ia, pa, chim.MIXED)
        np.testing.assert_array_equal(lnL_a, ref_a)
