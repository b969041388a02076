"""GPU parity of the incomplete-catalog option (Eqs. p-gal, p-miss, f-R)
against the oracle: forward ln L and per-event ln I in FP64, mixed and binned
precision, many-1D and single-1D; the FP64 adjoint (whose dG/dOm now holds
the Om derivative of V_c(z_max) in the missing-galaxy term) against the
oracle's finite differences, and the mixed adjoint against the FP64 one.

Tolerances: those of each precision (FP64: per event |Delta ln I_i| <= 1e-7,
|Delta ln L| <= 1e-6 N_events; mixed and binned: per event 1e-4, ln L 1e-3);
gradients as in the complete case (FP64 vs finite differences 2e-5 relative
+ 1e-4/|theta_k|, mixed vs FP64 2e-3 relative + 1e-2/|theta_k|).
"""
import numpy as np
import pytest

from synth import catalog as sc

from _edges import edge_free
from test_gpu_grad import _check_fd

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


def _drop_pixel_galaxies(cat, pixels):
    """Copy of `cat` whose listed pixels hold no catalog galaxy."""
    out = dict(cat)
    go = cat["gal_off"]
    keep = np.ones(cat["gal_z"].size, bool)
    for p in pixels:
        keep[go[p]:go[p + 1]] = False
    counts = np.diff(go)
    counts[list(pixels)] = 0
    out["gal_off"] = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    out["gal_z"] = np.ascontiguousarray(cat["gal_z"][keep])
    out["gal_sigma"] = np.ascontiguousarray(cat["gal_sigma"][keep])
    return out


@pytest.mark.parametrize("kde_mode", [sc.KDE_MANY_1D, sc.KDE_SINGLE_1D])
def test_incomplete_forward_matches_oracle(chim, ctx, orc, kde_mode):
    cat = sc.config_catalog(2, n_events=5, n_pe=1200, n_inj=15000, gal_median=50, kde_mode=kde_mode)
    ic = sc.add_completeness(_drop_pixel_galaxies(cat, [0, int(cat["pix_off"][2])]), seed=21, f_R=0.6)
    th = sc.config_hyperpoints(2, n=2)
    th[1, 1] = 0.34  # a second Om: a second profile
    oc = orc.Catalog(ic)
    cid = ctx.load(ic)
    try:
        for prec, binned, ev_tol in ((chim.FP64, False, 1e-7), (chim.MIXED, False, 1e-4),
                                     (chim.MIXED_BINNED, True, 1e-4)):
            lnL, _, st = ctx.loglike(cid, th, prec)
            terms = ctx.terms(cid, th, prec)
            for h in range(th.shape[0]):
                ref = oc.loglike(th[h], binned=binned)
                assert st[h] == ref["status"]
                tol = 1e-6 * cat["n_events"] if prec == chim.FP64 else 1e-3
                assert abs(lnL[h] - ref["lnL"]) <= tol, (prec, h, lnL[h] - ref["lnL"])
                np.testing.assert_allclose(terms["lnI"][h], ref["lnI"], rtol=0, atol=ev_tol)
    finally:
        ctx.unload(cid)


def test_complete_limit_is_bit_identical(chim, ctx):
    cat = sc.config_catalog(2, n_events=4, n_pe=800, n_inj=10000, gal_median=40)
    full = sc.add_completeness(cat, seed=3)
    full["completeness"] = np.ones_like(full["completeness"])
    full["f_R"] = 1.0
    th = sc.config_hyperpoints(2, n=3)
    a, b = ctx.load(cat), ctx.load(full)
    try:
        for prec in (chim.FP64, chim.MIXED):
            la, _, _ = ctx.loglike(a, th, prec)
            lb, _, _ = ctx.loglike(b, th, prec)
            np.testing.assert_array_equal(la, lb)
            _, ga, _ = ctx.grad(a, th[:1], prec)
            _, gb, _ = ctx.grad(b, th[:1], prec)
            np.testing.assert_array_equal(ga, gb)
    finally:
        ctx.unload(a)
        ctx.unload(b)


def test_incomplete_adjoint_matches_oracle_fd(chim, ctx, orc):
    cat = sc.config_catalog(2, n_events=5, n_pe=600, n_inj=20000, gal_median=60)
    t = sc.config_hyperpoints(2, n=1)[0].copy()
    t[1] = 0.32
    ic = sc.add_completeness(edge_free(cat, t), seed=5, f_R=0.5)
    oc = orc.Catalog(ic)
    gfd = oc.grad_fd(t, rel_step=1e-4)
    cid = ctx.load(ic)
    try:
        lnL, g, st = ctx.grad(cid, t[None, :], chim.FP64)
        assert abs(lnL[0] - oc.loglike(t)["lnL"]) <= 1e-6 * cat["n_events"]
        _check_fd(g[0], gfd, t, 2e-5, 1e-4, "fp64-incomplete")
        _, go, _ = oc.grad(t)
        _check_fd(g[0], go, t, 1e-6, 1e-6, "fp64-vs-oracle-grad-incomplete")
        _, gm, _ = ctx.grad(cid, t[None, :], chim.MIXED)
        _check_fd(gm[0], go, t, 2e-3, 1e-2, "mixed-vs-oracle-grad-incomplete")
        _check_fd(gm[0], g[0], t, 2e-3, 1e-2, "mixed-vs-fp64-incomplete")
    finally:
        ctx.unload(cid)


def test_incomplete_descriptor_rules(chim, ctx):
    cat = sc.config_catalog(2, n_events=2, n_pe=300, n_inj=2000, gal_median=20)
    ic = sc.add_completeness(cat, seed=4)
    for key, val in (("f_R", 1.5), ("f_R", -0.1)):
        bad = dict(ic)
        bad[key] = val
        with pytest.raises(chim.ChimeraError) as e:
            ctx.load(bad)
        assert e.value.code == chim.CHIMERA_ERR_INVALID_ARG
    bad = dict(ic)
    bad["completeness"] = ic["completeness"].copy()
    bad["completeness"][0, 3] = 1.2
    with pytest.raises(chim.ChimeraError):
        ctx.load(bad)
    bad = dict(ic)
    bad["pix_area"] = ic["pix_area"].copy()
    bad["pix_area"][1] = 0.0
    with pytest.raises(chim.ChimeraError):
        ctx.load(bad)


def test_empty_catalog_limit_matches_oracle(chim, ctx, orc):
    """f_R = 0 and P_compl = 0 everywhere: the galaxy term is the homogeneous
    prior alone (the catalog's galaxies drop out), in FP64 and mixed."""
    cat = sc.config_catalog(2, n_events=4, n_pe=800, n_inj=10000, gal_median=40)
    ic = sc.add_completeness(cat, seed=9)
    ic["completeness"] = np.zeros_like(ic["completeness"])
    ic["f_R"] = 0.0
    th = sc.config_hyperpoints(2, n=2)
    th[1, 1] = 0.33
    oc = orc.Catalog(ic)
    cid = ctx.load(ic)
    try:
        for prec, ev_tol in ((chim.FP64, 1e-7), (chim.MIXED, 1e-4)):
            terms = ctx.terms(cid, th, prec)
            for h in range(th.shape[0]):
                np.testing.assert_allclose(terms["lnI"][h], oc.loglike(th[h])["lnI"], rtol=0, atol=ev_tol)
    finally:
        ctx.unload(cid)
