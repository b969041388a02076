"""GPU adjoint (chimera_grad) against the oracle's gradient: the analytic one
(orc_grad, the hand-derived FP64 chain) and the central finite differences of
the oracle's ln L.

The adjoint returns the almost-everywhere derivative: samples or injections
that cross a mass edge (m_min, m_max) or the selection's z_max under a
finite-difference step make jumps that no derivative contains.  The test
catalogs therefore drop every PE sample and injection whose source-frame
masses or redshift lie within a 1 % margin of those edges at the test point
(a step of 1e-4 relative moves them by ~1e-4 relative), so the oracle's
finite differences measure the derivative itself.

Tolerance: the central difference with relative step h = 1e-4 has truncation
error ~ h^2 |d^3 lnL| ~ 1e-8 relative; the KDE support and window edges of
the oracle add jumps of at most exp(-18) of an event integral per grid point
that crosses them, i.e. <= ~1e-8 / (2 h theta_k) in the derivative.  We
require |g_gpu - g_fd| <= 2e-5 |g_fd| + 1e-4 / |theta_k| (FP64 path).  The
mixed path follows its own computed ln L (FP32 z and weights, FP32 KDE and
profile); its gradient must match the FP64 adjoint to 2e-3 relative plus
1e-2 / |theta_k|.  Against the analytic oracle gradient (both FP64, both the
almost-everywhere derivative): the FP64 adjoint within 1e-6 relative +
1e-6 / |theta_k| (the GPU's windows and interpolated distance tables against
the oracle's full grid and adaptive quadrature), the mixed adjoint within the
mixed tolerance above.
"""
import math

import numpy as np
import pytest

from synth import catalog as sc
from _edges import edge_free

pytestmark = pytest.mark.gpu

C_KMS = 299792.458


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


def _check_fd(g, gfd, th, rtol, atol_scale, what):
    for k in range(12):
        tol = rtol * abs(gfd[k]) + atol_scale / abs(th[k])
        assert abs(g[k] - gfd[k]) <= tol, (what, k, g[k], gfd[k], tol)


def _catalog_many1d():
    cat = sc.config_catalog(2, n_events=5, n_pe=600, n_inj=20000, gal_median=60)
    th = sc.config_hyperpoints(2, n=2)
    return cat, th


@pytest.mark.parametrize("xi0", [1.0, 1.6])
def test_fp64_adjoint_matches_oracle_fd_many1d(chim, ctx, orc, xi0):
    cat, th = _catalog_many1d()
    t = th[0].copy()
    t[2] = xi0
    cat = edge_free(cat, t)
    oc = orc.Catalog(cat)
    gfd = oc.grad_fd(t, rel_step=1e-4)
    cid = ctx.load(cat)
    try:
        lnL, g, st = ctx.grad(cid, t[None, :], chim.FP64)
        ref = oc.loglike(t)
        assert abs(lnL[0] - ref["lnL"]) <= 1e-6 * cat["n_events"]
        _check_fd(g[0], gfd, t, 2e-5, 1e-4, "fp64-many1d")
        lo, go, so = oc.grad(t)
        _check_fd(g[0], go, t, 1e-6, 1e-6, "fp64-vs-oracle-grad")
        # mixed adjoint against the oracle's gradient and the FP64 adjoint
        lnLm, gm, stm = ctx.grad(cid, t[None, :], chim.MIXED)
        _check_fd(gm[0], go, t, 2e-3, 1e-2, "mixed-vs-oracle-grad")
        _check_fd(gm[0], g[0], t, 2e-3, 1e-2, "mixed-vs-fp64")
    finally:
        ctx.unload(cid)


def test_fp64_adjoint_matches_oracle_fd_single1d(chim, ctx, orc):
    cat = sc.config_catalog(2, n_events=4, n_pe=500, n_inj=8000, gal_median=40,
                            kde_mode=sc.KDE_SINGLE_1D)
    t = sc.config_hyperpoints(2, n=1)[0].copy()
    t[1] = 0.33       # an Om away from the fiducial one
    t[9] = 2.2
    cat = edge_free(cat, t)
    oc = orc.Catalog(cat)
    gfd = oc.grad_fd(t, rel_step=1e-4)
    cid = ctx.load(cat)
    try:
        lnL, g, st = ctx.grad(cid, t[None, :], chim.FP64)
        _check_fd(g[0], gfd, t, 2e-5, 1e-4, "fp64-single1d")
        lo, go, so = oc.grad(t)
        _check_fd(g[0], go, t, 1e-6, 1e-6, "fp64-vs-oracle-grad-single1d")
        lnLm, gm, stm = ctx.grad(cid, t[None, :], chim.MIXED)
        _check_fd(gm[0], go, t, 2e-3, 1e-2, "mixed-vs-oracle-grad-single1d")
        _check_fd(gm[0], g[0], t, 2e-3, 1e-2, "mixed-vs-fp64-single1d")
    finally:
        ctx.unload(cid)


def test_adjoint_batch_independence_and_inadmissible(chim, ctx):
    cat, th = _catalog_many1d()
    cat = edge_free(cat, th[0])
    pts = np.stack([th[0], th[1], th[0]])
    pts[1, 1] = 0.32
    bad = th[0].copy()
    bad[7], bad[8] = 60.0, 50.0                # m_max < m_min: inadmissible
    pts = np.vstack([pts, bad])
    cid = ctx.load(cat)
    try:
        for prec in (chim.FP64, chim.MIXED):
            lnL, g, st = ctx.grad(cid, pts, prec)
            lnL1, g1, _ = ctx.grad(cid, pts[:1], prec)
            assert np.array_equal(g[0], g1[0]) and np.array_equal(g[0], g[2])
            assert lnL[3] == -math.inf and np.all(g[3] == 0.0)
            assert st[3] & chim.PT_OUT_OF_SUPPORT
            lnLf, _, _ = ctx.loglike(cid, pts, prec)
            assert np.array_equal(lnL, lnLf)
            # determinism
            _, g2, _ = ctx.grad(cid, pts, prec)
            assert np.array_equal(g, g2)
    finally:
        ctx.unload(cid)


def test_autograd_function(chim, ctx):
    import torch
    cat, th = _catalog_many1d()
    cat = edge_free(cat, th[0])
    cid = ctx.load(cat)
    try:
        t = torch.tensor(th[:2], dtype=torch.float64, requires_grad=True)
        lnL = chim.ChimeraLogLike.apply(t, ctx, cid, chim.FP64)
        (lnL * torch.tensor([1.0, -2.0], dtype=torch.float64)).sum().backward()
        _, g, _ = ctx.grad(cid, th[:2], chim.FP64)
        np.testing.assert_array_equal(t.grad.numpy(), np.stack([g[0], -2.0 * g[1]]))
    finally:
        ctx.unload(cid)
