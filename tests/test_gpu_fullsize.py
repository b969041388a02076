"""Full-size parity for the batched photometric and the differentiation
workloads, in the launch configuration of their sizes, on outputs the oracle
can compute one at a time (sampled events, the selection term) and on
properties that hold at any size.

* Photometric catalog: 300 events x 5000 PE, sigma_z = 0.05(1+z), x3 galaxy
  counts stored as BF16, 512 hyperpoints per launch, mixed.  The oracle reads
  the same BF16-rounded galaxy values.
* Differentiation catalog: 5000 events x 4000 PE, 5e6 injections, 64
  hyperpoints with Om varying, ln L and the 12-component gradient (mixed).
  Sampled events (with their own Om) against the oracle; the gradient is
  additive over disjoint event sets sharing the injections,
  grad(A u B) = grad(A) + grad(B), which checks the full-size adjoint launch
  against two independent half-size launches; the first 50 events with
  all the injections are compared with the oracle's analytic gradient.
Tolerances are those of the mixed path (per event |Delta ln I| <= 1e-4,
|Delta ln xi| <= 3e-6).
"""
import math

import numpy as np
import pytest

from synth import catalog as sc

pytestmark = pytest.mark.gpu

MIX_EV = 1e-4


@pytest.fixture(scope="module")
def chim():
    from paper_2504_02034_b300 import build
    build.build()
    import paper_2504_02034_b300 as pkg
    return pkg


@pytest.fixture(scope="module")
def ctx(chim):
    c = chim.Context(0)
    yield c
    c.close()


def _subset(cat, events):
    """Catalog holding only `events` (same injections, same N_gal,tot)."""
    so, po, go = cat["sample_off"], cat["pix_off"], cat["gal_off"]
    keys = ("dL", "m1_det", "m2_det", "pix_of_sample")
    out = dict(cat)
    sl = [np.arange(so[e], so[e + 1]) for e in events]
    pl = [np.arange(po[e], po[e + 1]) for e in events]
    idx = np.concatenate(sl)
    pidx = np.concatenate(pl)
    for k in keys:
        out[k] = np.ascontiguousarray(cat[k][idx])
    out["sample_off"] = np.concatenate([[0], np.cumsum([len(x) for x in sl])]).astype(np.int64)
    out["pix_off"] = np.concatenate([[0], np.cumsum([len(x) for x in pl])]).astype(np.int64)
    out["sky_S"] = np.ascontiguousarray(cat["sky_S"][pidx])
    gl = [np.arange(go[p], go[p + 1]) for p in pidx]
    gidx = np.concatenate(gl)
    out["gal_off"] = np.concatenate([[0], np.cumsum([len(x) for x in gl])]).astype(np.int64)
    out["gal_z"] = np.ascontiguousarray(cat["gal_z"][gidx])
    out["gal_sigma"] = np.ascontiguousarray(cat["gal_sigma"][gidx])
    out["n_events"] = len(events)
    return out


def test_photometric_bf16_512_points(chim, ctx, orc):
    cat = sc.config_catalog(3)
    assert cat["gal_storage"] == sc.GAL_BF16
    th = sc.config_hyperpoints(3)
    assert th.shape[0] == 512
    cid = ctx.load(cat)
    try:
        terms = ctx.terms(cid, th, chim.MIXED)
        lnL, neff, st = ctx.loglike(cid, th, chim.MIXED)
        oc = orc.Catalog(sc.quantize_galaxies(cat, sc.GAL_BF16))
        # a walker can leave an event with no sample inside its mass range
        # (I_i = 0): ln L = -inf with OUT_OF_SUPPORT, and the oracle agrees
        bad = ~np.isfinite(lnL)
        assert bad.sum() < 0.1 * th.shape[0]
        for h in np.nonzero(bad)[0][:2]:
            assert st[h] & chim.PT_OUT_OF_SUPPORT
            evs0 = np.nonzero(~np.isfinite(terms["lnI"][h]))[0]
            assert evs0.size > 0
            for ev in evs0[:2]:
                assert oc.event_lnI(th[h], int(ev)) == -math.inf, (h, ev)
        # ln L is the sum of its stages, for every admissible point of the launch
        ok = ~bad
        ref_sum = terms["lnI"][ok].sum(axis=1) - cat["n_events"] * np.log(terms["xi"][ok])
        np.testing.assert_allclose(lnL[ok], ref_sum, rtol=0, atol=1e-9 * np.abs(lnL[ok]).max())
        rng = np.random.default_rng(31)
        evs = [0, cat["n_events"] - 1] + [int(e) for e in rng.choice(cat["n_events"], 2, replace=False)]
        hs = [h for h in (0, 255, 511, 100, 300) if ok[h]][:3]
        for h in hs:
            for ev in evs:
                ref = oc.event_lnI(th[h], ev)
                assert abs(terms["lnI"][h, ev] - ref) <= MIX_EV, (h, ev, terms["lnI"][h, ev] - ref)
        for h in hs[:2]:
            xi, _ = oc.selection(th[h])
            assert abs(math.log(terms["xi"][h]) - math.log(xi)) <= 3e-6
    finally:
        ctx.unload(cid)


@pytest.fixture(scope="module")
def c4():
    return sc.config_catalog(4)


def test_differentiation_catalog_sampled_events(chim, ctx, orc, c4):
    cat = c4
    th = sc.config_hyperpoints(4)
    assert th.shape[0] == 64 and len(np.unique(th[:, 1])) > 32  # Om varies
    cid = ctx.load(cat)
    try:
        lnL, g, st = ctx.grad(cid, th, chim.MIXED)
        assert np.all(np.isfinite(g))
        assert np.all(g[~np.isfinite(lnL)] == 0.0)
        terms = ctx.terms(cid, th, chim.MIXED)
        oc = orc.Catalog(cat)
        rng = np.random.default_rng(41)
        evs = [0, cat["n_events"] - 1] + [int(e) for e in rng.choice(cat["n_events"], 2, replace=False)]
        for h in (1, 40):
            for ev in evs:
                ref = oc.event_lnI(th[h], ev)
                assert abs(terms["lnI"][h, ev] - ref) <= MIX_EV, (h, ev, terms["lnI"][h, ev] - ref)
        xi, _ = oc.selection(th[40])
        assert abs(math.log(terms["xi"][40]) - math.log(xi)) <= 3e-6
    finally:
        ctx.unload(cid)


def test_differentiation_subset_gradient_vs_oracle_gradient(chim, ctx, orc, c4):
    """The first 50 events of the differentiation catalog with all its
    injections: ln L and the 12-component gradient of two hyperpoints (Om
    varying) against the oracle's analytic gradient, FP64 and mixed."""
    cat = _subset(c4, list(range(50)))
    th = sc.config_hyperpoints(4)
    oc = orc.Catalog(cat)
    cid = ctx.load(cat)
    try:
        for h in (1, 40):
            t = th[h]
            lo, go, so = oc.grad(t)
            if not math.isfinite(lo):
                continue
            l64, g64, s64 = ctx.grad(cid, t[None, :], chim.FP64)
            lm, gm, sm = ctx.grad(cid, t[None, :], chim.MIXED)
            assert s64[0] == so and sm[0] == so
            assert abs(l64[0] - lo) <= 1e-6 * cat["n_events"] and abs(lm[0] - lo) <= 1e-3
            for k in range(12):
                assert abs(g64[0, k] - go[k]) <= 1e-6 * abs(go[k]) + 1e-6 / abs(t[k]), ("fp64", h, k, g64[0, k], go[k])
                assert abs(gm[0, k] - go[k]) <= 2e-3 * abs(go[k]) + 1e-2 / abs(t[k]), ("mixed", h, k, gm[0, k], go[k])
    finally:
        ctx.unload(cid)


def test_differentiation_gradient_is_additive_over_events(chim, ctx, c4):
    cat = c4
    th = sc.config_hyperpoints(4)[:16]
    ne = cat["n_events"]
    half = ne // 2
    parts = [_subset(cat, list(range(half))), _subset(cat, list(range(half, ne)))]
    cid = ctx.load(cat)
    try:
        lnL, g, _ = ctx.grad(cid, th, chim.MIXED)
    finally:
        ctx.unload(cid)
    gs, ls = [], []
    for part in parts:
        pid = ctx.load(part)
        try:
            l, gp, _ = ctx.grad(pid, th, chim.MIXED)
            gs.append(gp)
            ls.append(l)
        finally:
            ctx.unload(pid)
    # ln L(A u B) = ln L(A) + ln L(B) (each part carries N_obs of its own
    # events); a point with an empty event (ln L = -inf) has gradient 0 and
    # is compared only through its ln L
    ok = np.isfinite(lnL)
    assert ok.sum() >= th.shape[0] // 2
    np.testing.assert_array_equal(np.isfinite(ls[0] + ls[1]), ok)
    np.testing.assert_allclose(lnL[ok], (ls[0] + ls[1])[ok], rtol=1e-12, atol=1e-9 * np.abs(lnL[ok]).max())
    assert np.all(g[~ok] == 0.0)
    gsum = (gs[0] + gs[1])[ok]
    scale = np.abs(g[ok]).max(axis=0) + 1e-12
    # the whole catalog and its halves add their events' FP32 terms in
    # different groupings, so the additivity holds to the FP32 rounding of
    # those sums, ~1e-9 of each component's scale
    assert np.all(np.abs(g[ok] - gsum) <= 1e-8 * scale + 1e-12), np.abs(g[ok] - gsum).max(axis=0)
