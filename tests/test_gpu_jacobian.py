"""GPU parity of the per-sample Jacobian placement (CHIMERA_JACOBIAN_PER_SAMPLE
OR'ed into the precision; Eq. jacobian on each PE sample's KDE weight, the
bandwidth from the weights of Eq. gw-kernel, psi alone on the grid) against
the oracle's variant, in FP64, mixed and binned precision, with the Gaussian
and the Epanechnikov kernel, many-1D and single-1D, at a modified-gravity
point (Xi0 != 1, so that the Jacobian's shape depends on the hyperparameters).

Tolerances: those of each precision (FP64: per event |Delta ln I_i| <= 1e-7,
|Delta ln L| <= 1e-6 N_events; mixed and binned: per event 1e-4, ln L 1e-3).
"""
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


@pytest.fixture(scope="module")
def ctx(chim):
    c = chim.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("kde_mode", [sc.KDE_MANY_1D, sc.KDE_SINGLE_1D])
@pytest.mark.parametrize("kernel", [0, 1])
def test_per_sample_jacobian_matches_oracle(chim, ctx, orc, kde_mode, kernel):
    cat = sc.config_catalog(2, n_events=5, n_pe=1200, n_inj=15000, gal_median=50, kde_mode=kde_mode)
    th = sc.config_hyperpoints(2, n=2)
    th[:, 2] = [1.3, 0.8]
    th[:, 3] = 2.0
    oc = orc.Catalog(cat, kernel=kernel, jacobian=orc.JACOBIAN_PER_SAMPLE)
    flag = chim.JACOBIAN_PER_SAMPLE | (chim.KERNEL_EPANECHNIKOV if kernel else 0)
    cid = ctx.load(cat)
    try:
        for base, binned, ev_tol in ((chim.FP64, False, 1e-7), (chim.MIXED, False, 1e-4),
                                     (chim.MIXED_BINNED, True, 1e-4)):
            lnL, _, st = ctx.loglike(cid, th, base | flag)
            terms = ctx.terms(cid, th, base | flag)
            for h in range(th.shape[0]):
                ref = oc.loglike(th[h], binned=binned)
                assert st[h] == ref["status"]
                tol = 1e-6 * cat["n_events"] if base == chim.FP64 else 1e-3
                assert abs(lnL[h] - ref["lnL"]) <= tol, (base, h, lnL[h] - ref["lnL"])
                np.testing.assert_allclose(terms["lnI"][h], ref["lnI"], rtol=0, atol=ev_tol)
    finally:
        ctx.unload(cid)


def test_per_sample_jacobian_differs_and_rules(chim, ctx):
    cat = sc.config_catalog(2, n_events=4, n_pe=800, n_inj=10000, gal_median=40)
    th = sc.config_hyperpoints(2, n=3)
    th[:, 2] = 1.2
    cid = ctx.load(cat)
    try:
        for base in (chim.FP64, chim.MIXED):
            lg, _, _ = ctx.loglike(cid, th, base)
            lp, _, _ = ctx.loglike(cid, th, base | chim.JACOBIAN_PER_SAMPLE)
            assert np.all(np.isfinite(lp)) and np.all(lp != lg)
            for h in range(th.shape[0]):  # batch independence
                l1, _, _ = ctx.loglike(cid, th[h:h + 1], base | chim.JACOBIAN_PER_SAMPLE)
                assert l1[0] == lp[h]
            with pytest.raises(chim.ChimeraError) as e:
                ctx.grad(cid, th[:1], base | chim.JACOBIAN_PER_SAMPLE)
            assert e.value.code == chim.CHIMERA_ERR_INVALID_ARG
        with pytest.raises(chim.ChimeraError):
            ctx.loglike(cid, th[:1], chim.MIXED | 0x40)  # unknown flag
    finally:
        ctx.unload(cid)
