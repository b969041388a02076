"""GPU parity of the "3D" kernel (CHIMERA_KDE_3D catalogs, Sec. 2.3, the
cross-check variant) against the oracle, which evaluates the trivariate
Gaussian directly (the GPU splits it into a sky factor and a conditional
Gaussian in z).  FP64 only: per event |Delta ln I_i| <= 1e-7 and
|Delta ln L| <= 1e-6 N_events, with the Jacobian on the grid and on the
samples; the calls the variant does not take are refused.
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


@pytest.fixture(scope="module")
def cat3():
    return sc.config_catalog(2, n_events=5, n_pe=900, n_inj=12000, gal_median=40, kde_mode=sc.KDE_3D)


@pytest.mark.parametrize("jacobian", [0, 1])
def test_kde3_matches_oracle(chim, ctx, orc, cat3, jacobian):
    th = sc.config_hyperpoints(2, n=3)
    th[1, 1] = 0.33  # a second Om
    th[2, 2] = 1.3   # modified GW propagation
    oc = orc.Catalog(cat3, jacobian=jacobian)
    prec = chim.FP64 | (chim.JACOBIAN_PER_SAMPLE if jacobian else 0)
    cid = ctx.load(cat3)
    try:
        lnL, _, st = ctx.loglike(cid, th, prec)
        terms = ctx.terms(cid, th, prec)
        for h in range(th.shape[0]):
            ref = oc.loglike(th[h])
            assert st[h] == ref["status"]
            assert abs(lnL[h] - ref["lnL"]) <= 1e-6 * cat3["n_events"], (h, lnL[h] - ref["lnL"])
            np.testing.assert_allclose(terms["lnI"][h], ref["lnI"], rtol=0, atol=1e-7)
    finally:
        ctx.unload(cid)


def test_kde3_is_its_own_kernel_and_rules(chim, ctx, cat3):
    th = sc.config_hyperpoints(2, n=2)
    m1 = dict(cat3)
    m1["kde_mode"] = sc.KDE_MANY_1D
    a, b = ctx.load(cat3), ctx.load(m1)
    try:
        l3, _, _ = ctx.loglike(a, th, chim.FP64)
        lm, _, _ = ctx.loglike(b, th, chim.FP64)
        assert np.all(np.isfinite(l3)) and np.all(l3 != lm)
        for prec in (chim.MIXED, chim.MIXED_BINNED, chim.FP64 | chim.KERNEL_EPANECHNIKOV):
            with pytest.raises(chim.ChimeraError) as e:
                ctx.loglike(a, th, prec)
            assert e.value.code == chim.CHIMERA_ERR_INVALID_ARG
        with pytest.raises(chim.ChimeraError) as e:
            ctx.grad(a, th[:1], chim.FP64)
        assert e.value.code == chim.CHIMERA_ERR_INVALID_ARG
        with pytest.raises(chim.ChimeraError) as e:
            chim.chimera_serve_submit(ctx.h, a, th[:1], chim.SERVE_MIXED)
        assert e.value.code == chim.CHIMERA_ERR_INVALID_ARG
        # the catalog stays usable after the refusals
        l3b, _, _ = ctx.loglike(a, th, chim.FP64)
        np.testing.assert_array_equal(l3, l3b)
    finally:
        ctx.unload(a)
        ctx.unload(b)


def test_kde3_degenerate_event(chim, ctx, orc):
    """An event with three PE samples has no positive-definite covariance
    over (z, x, y) in either form: its ln I is -inf on both sides, the other
    events keep their values."""
    cat = sc.config_catalog(2, n_events=3, n_pe=400, n_inj=8000, gal_median=30, kde_mode=sc.KDE_3D)
    so = cat["sample_off"]
    keep = np.ones(int(so[-1]), bool)
    keep[so[0] + 3:so[1]] = False           # event 0 keeps 3 samples
    out = dict(cat)
    counts = np.array([keep[so[e]:so[e + 1]].sum() for e in range(cat["n_events"])])
    out["sample_off"] = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    for k in ("dL", "m1_det", "m2_det", "pix_of_sample", "sky_xy"):
        out[k] = np.ascontiguousarray(cat[k][keep])
    th = sc.config_hyperpoints(2, n=1)
    oc = orc.Catalog(out)
    ref = oc.loglike(th[0])
    cid = ctx.load(out)
    try:
        lnI = ctx.terms(cid, th, chim.FP64)["lnI"][0]
        assert ref["lnI"][0] == -np.inf and lnI[0] == -np.inf
        np.testing.assert_allclose(lnI[1:], ref["lnI"][1:], rtol=0, atol=1e-7)
        lnL, _, st = ctx.loglike(cid, th, chim.FP64)
        assert lnL[0] == -np.inf and ref["lnL"] == -np.inf
        assert st[0] == ref["status"], (st[0], ref["status"])
    finally:
        ctx.unload(cid)
