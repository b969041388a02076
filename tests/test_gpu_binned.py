"""GPU parity of the binned-KDE option (CHIMERA_MIXED_BINNED) against the
oracle's binned form, its stated error against the unbinned result, and its
argument rules.

Tolerances: those of the mixed path against the binned oracle (per event
|Delta ln I_i| <= 1e-4, ln L within 1e-3 per catalog); against the unbinned
mixed result, the stated binning bound (dz/b)^2 / 8 per event plus the
mixed path's own 2e-4.
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


@pytest.mark.parametrize("kde_mode", [sc.KDE_MANY_1D, sc.KDE_SINGLE_1D])
def test_binned_matches_binned_oracle(chim, ctx, orc, kde_mode):
    cat = sc.config_catalog(2, n_events=6, n_pe=1500, n_inj=20000, gal_median=60, kde_mode=kde_mode)
    th = sc.config_hyperpoints(2, n=3)
    oc = orc.Catalog(cat)
    cid = ctx.load(cat)
    try:
        lnL, neff, st = ctx.loglike(cid, th, chim.MIXED_BINNED)
        terms = ctx.terms(cid, th, chim.MIXED_BINNED)
        for h in range(th.shape[0]):
            ref = oc.loglike(th[h], binned=True)
            assert st[h] == ref["status"]
            assert abs(lnL[h] - ref["lnL"]) <= 1e-3, (h, lnL[h] - ref["lnL"])
            np.testing.assert_allclose(terms["lnI"][h], ref["lnI"], rtol=0, atol=MIX_EV)
    finally:
        ctx.unload(cid)


@pytest.mark.parametrize("kde_mode", [sc.KDE_MANY_1D, sc.KDE_SINGLE_1D])
def test_binned_error_against_unbinned_within_bound(chim, ctx, kde_mode):
    cat = sc.config_catalog(2, n_events=20, n_pe=3000, n_inj=20000, gal_median=80, kde_mode=kde_mode)
    th = sc.config_hyperpoints(2, n=8)
    dz = cat["z_max"] / (cat["n_z"] - 1)
    cid = ctx.load(cat)
    try:
        tb = ctx.terms(cid, th, chim.MIXED_BINNED)
        tm = ctx.terms(cid, th, chim.MIXED)
        np.testing.assert_array_equal(tb["bw"], tm["bw"])  # the samples' bandwidth
        ok = np.isfinite(tm["lnI"])
        np.testing.assert_array_equal(np.isfinite(tb["lnI"]), ok)
        bound = (dz / tm["bw"]) ** 2 / 8 + 2e-4
        assert np.all(np.abs(tb["lnI"] - tm["lnI"])[ok] <= bound[ok])
        np.testing.assert_array_equal(tb["xi"], tm["xi"])  # the selection term is not binned
    finally:
        ctx.unload(cid)


def test_binned_batch_independence_and_rules(chim, ctx):
    cat = sc.config_catalog(2, n_events=5, n_pe=800, n_inj=10000, gal_median=40, kde_mode=sc.KDE_SINGLE_1D)
    th = sc.config_hyperpoints(2, n=4)
    bad = th[0].copy()
    bad[7], bad[8] = 60.0, 50.0  # m_max < m_min: inadmissible
    pts = np.vstack([th, bad])
    cid = ctx.load(cat)
    try:
        lnL, _, st = ctx.loglike(cid, pts, chim.MIXED_BINNED)
        for h in range(th.shape[0]):
            l1, _, _ = ctx.loglike(cid, pts[h:h + 1], chim.MIXED_BINNED)
            assert l1[0] == lnL[h]
        assert lnL[-1] == -math.inf and st[-1] & chim.PT_OUT_OF_SUPPORT
        lnL2, _, _ = ctx.loglike(cid, pts, chim.MIXED_BINNED)
        assert np.array_equal(lnL, lnL2)  # deterministic
        with pytest.raises(chim.ChimeraError) as e:
            ctx.grad(cid, th[:1], chim.MIXED_BINNED)
        assert e.value.code == chim.CHIMERA_ERR_INVALID_ARG
    finally:
        ctx.unload(cid)


def test_binned_full_size_single1d_sampled_events(chim, ctx, orc):
    """The 300-event x 5000 PE catalog in single-1D form, 16 points per launch
    (the launch the bench times for the binned option): sampled events
    against the binned oracle."""
    cat = sc.config_catalog(2, kde_mode=sc.KDE_SINGLE_1D)
    th = sc.config_hyperpoints(2)
    cid = ctx.load(cat)
    try:
        terms = ctx.terms(cid, th, chim.MIXED_BINNED)
        oc = orc.Catalog(cat)
        rng = np.random.default_rng(61)
        evs = [0, cat["n_events"] - 1] + [int(e) for e in rng.choice(cat["n_events"], 2, replace=False)]
        for h in (0, 15):
            for ev in evs:
                ref = oc.event_lnI(th[h], ev, binned=True)
                assert abs(terms["lnI"][h, ev] - ref) <= MIX_EV, (h, ev, terms["lnI"][h, ev] - ref)
    finally:
        ctx.unload(cid)
