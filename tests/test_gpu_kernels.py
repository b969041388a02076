"""GPU parity of the Epanechnikov kernel option (CHIMERA_KERNEL_EPANECHNIKOV
OR'ed into the precision) against the oracle's Epanechnikov form, in FP64,
mixed and binned precision, many-1D and single-1D.

Tolerances: those of each precision (FP64: per event |Delta ln I_i| <= 1e-7,
|Delta ln L| <= 1e-6 N_events; mixed and binned: per event 1e-4, ln L 1e-3).
"""
import math

import numpy as np
import pytest

from synth import catalog as sc

pytestmark = pytest.mark.gpu

EPAN = 1  # oracle kernel shape


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
def test_epanechnikov_matches_oracle(chim, ctx, orc, kde_mode):
    cat = sc.config_catalog(2, n_events=5, n_pe=1200, n_inj=15000, gal_median=50, kde_mode=kde_mode)
    th = sc.config_hyperpoints(2, n=2)
    oc = orc.Catalog(cat, kernel=EPAN)
    cid = ctx.load(cat)
    try:
        for base, binned, ev_tol in ((chim.FP64, False, 1e-7), (chim.MIXED, False, 1e-4),
                                     (chim.MIXED_BINNED, True, 1e-4)):
            prec = base | chim.KERNEL_EPANECHNIKOV
            lnL, _, st = ctx.loglike(cid, th, prec)
            terms = ctx.terms(cid, th, prec)
            for h in range(th.shape[0]):
                ref = oc.loglike(th[h], binned=binned)
                assert st[h] == ref["status"]
                tol = 1e-6 * cat["n_events"] if base == chim.FP64 else 1e-3
                assert abs(lnL[h] - ref["lnL"]) <= tol, (base, h, lnL[h] - ref["lnL"])
                np.testing.assert_allclose(terms["lnI"][h], ref["lnI"], rtol=0, atol=ev_tol)
    finally:
        ctx.unload(cid)


def test_epanechnikov_differs_from_gaussian_and_rules(chim, ctx, orc):
    cat = sc.config_catalog(2, n_events=4, n_pe=800, n_inj=10000, gal_median=40)
    th = sc.config_hyperpoints(2, n=3)
    cid = ctx.load(cat)
    try:
        lg, _, _ = ctx.loglike(cid, th, chim.MIXED)
        le, _, _ = ctx.loglike(cid, th, chim.MIXED | chim.KERNEL_EPANECHNIKOV)
        assert np.all(np.isfinite(le)) and np.all(le != lg)
        # batch independence and determinism
        for h in range(th.shape[0]):
            l1, _, _ = ctx.loglike(cid, th[h:h + 1], chim.MIXED | chim.KERNEL_EPANECHNIKOV)
            assert l1[0] == le[h]
        for prec in (chim.MIXED | chim.KERNEL_EPANECHNIKOV, chim.FP64 | chim.KERNEL_EPANECHNIKOV):
            with pytest.raises(chim.ChimeraError) as e:
                ctx.grad(cid, th[:1], prec)
            assert e.value.code == chim.CHIMERA_ERR_INVALID_ARG
        with pytest.raises(chim.ChimeraError):
            ctx.loglike(cid, th[:1], chim.MIXED | 0x40)  # unknown flag
    finally:
        ctx.unload(cid)
