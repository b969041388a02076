"""The batched mixed-path galaxy profiles (up to PROF_MB = 16 new Om values per
pass, the Om-independent Gaussians shared by the columns; Eq. p-cat as a
contraction over galaxies) against the one-Om launches and the oracle.

The batched kernels repeat the one-Om arithmetic per column in the same
order, so ln L and every ln I_i must be bit-identical between a call that
brings 19 new Om values at once (batches of 16 and 3) and calls that bring
them one by one; and both must match the oracle at the mixed tolerance
(per event 1e-4, ln L 1e-3).  Covers many-1D and single-1D, F32 and BF16
galaxy storage, sparse and dense pixels, and an incomplete catalog.
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


def _points(n, seed):
    th = sc.config_hyperpoints(2, n=n)
    th[:, 1] = 0.27 + 0.06 * np.random.default_rng(seed).random(n)
    return th


CASES = [
    ("many1d-f32", dict(kde_mode=sc.KDE_MANY_1D), False),
    ("single1d-f32", dict(kde_mode=sc.KDE_SINGLE_1D), False),
    ("many1d-bf16", dict(kde_mode=sc.KDE_MANY_1D, gal_storage=sc.GAL_BF16), False),
    ("many1d-incomplete", dict(kde_mode=sc.KDE_MANY_1D), True),
]


@pytest.mark.parametrize("name,kw,incomplete", CASES, ids=[c[0] for c in CASES])
def test_batched_profiles_equal_one_om_and_oracle(chim, ctx, orc, name, kw, incomplete):
    cat = sc.config_catalog(2, n_events=6, n_pe=900, n_inj=12000, gal_median=1500, **kw)
    if incomplete:
        cat = sc.add_completeness(cat, seed=31, f_R=0.7)
    assert np.diff(cat["gal_off"]).max() > 1024  # dense pixels take the dense kernels
    a, b = ctx.load(cat), ctx.load(cat)
    try:
        for k, prec in enumerate((chim.MIXED, chim.MIXED_BINNED)):
            th = _points(19, seed=100 * k + len(name))  # new Om values for each precision
            lb, _, sb = ctx.loglike(b, th, prec)            # 19 new Om: batches of 16 and 3
            tb = ctx.terms(b, th, prec)["lnI"]
            la = np.empty_like(lb)
            ta = np.empty_like(tb)
            for h in range(th.shape[0]):                     # one new Om per call
                la[h] = ctx.loglike(a, th[h:h + 1], prec)[0][0]
                ta[h] = ctx.terms(a, th[h:h + 1], prec)["lnI"][0]
            np.testing.assert_array_equal(lb, la)
            np.testing.assert_array_equal(tb, ta)
        # 16-bit storage: the oracle reads the stored (decoded) galaxy values
        oc = orc.Catalog(sc.quantize_galaxies(cat, cat["gal_storage"]) if cat.get("gal_storage", 0) else cat)
        for h in (0, 5, 18):
            ref = oc.loglike(th[h], binned=True)
            assert abs(lb[h] - ref["lnL"]) <= 1e-3, (h, lb[h] - ref["lnL"])
            np.testing.assert_allclose(tb[h], ref["lnI"], rtol=0, atol=1e-4)
    finally:
        ctx.unload(a)
        ctx.unload(b)


def test_batched_profiles_mixed_forward_vs_oracle(chim, ctx, orc):
    cat = sc.config_catalog(2, n_events=5, n_pe=1200, n_inj=15000, gal_median=80)
    th = _points(10, seed=77)
    oc = orc.Catalog(cat)
    cid = ctx.load(cat)
    try:
        lnL, _, st = ctx.loglike(cid, th, chim.MIXED)
        terms = ctx.terms(cid, th, chim.MIXED)["lnI"]
        for h in range(th.shape[0]):
            ref = oc.loglike(th[h])
            assert st[h] == ref["status"]
            assert abs(lnL[h] - ref["lnL"]) <= 1e-3
            np.testing.assert_allclose(terms[h], ref["lnI"], rtol=0, atol=1e-4)
    finally:
        ctx.unload(cid)


@pytest.mark.parametrize("kde_mode,incomplete", [(sc.KDE_MANY_1D, False), (sc.KDE_SINGLE_1D, False),
                                                 (sc.KDE_MANY_1D, True)])
def test_batched_gradient_profiles_equal_one_om(chim, ctx, kde_mode, incomplete):
    """The gradient's dG/dOm profiles and dD/dOm tables, batched over new Om
    values, against one new Om per call: bit-identical ln L and gradient."""
    cat = sc.config_catalog(2, n_events=5, n_pe=700, n_inj=10000, gal_median=1500, kde_mode=kde_mode)
    if incomplete:
        cat = sc.add_completeness(cat, seed=41, f_R=0.8)
    th = _points(19, seed=5 + kde_mode + 2 * incomplete)  # batches of 16 and 3
    a, b = ctx.load(cat), ctx.load(cat)
    try:
        lb, gb, _ = ctx.grad(b, th, chim.MIXED)
        for h in range(th.shape[0]):
            la, ga, _ = ctx.grad(a, th[h:h + 1], chim.MIXED)
            assert la[0] == lb[h], h
            np.testing.assert_array_equal(ga[0], gb[h])
        assert np.all(np.isfinite(gb))
    finally:
        ctx.unload(a)
        ctx.unload(b)
