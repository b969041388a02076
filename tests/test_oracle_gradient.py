"""Pins of the oracle's analytic gradient (orc_grad) and of its per-sample
reweighting (samples_h), independent of the code under test.

* d D_c / d Om against closed forms: Einstein-de Sitter (Om = 1),
  D_c' = (c/H0)[(1+z)^(-1/2) - (1+z)^(-7/2)/7 - 6/7], and de Sitter (Om = 0),
  D_c' = -(c/H0)[((1+z)^4 - 1)/4 - z]/2.
* The 12-component gradient against central differences of the oracle's
  ln L (relative step 1e-4) on catalogs from which samples and injections
  near a mass edge or z_max are removed (the almost-everywhere derivative):
  a dropped term, a wrong sign or a missing chain link in any stage (distance
  inversion, mass model, Scott bandwidth, KDE, galaxy term, grid factor,
  selection) shows up as an O(1) relative error in some component.
* The reweighting of every PE sample (Sec. 2.1, Eq. gw-kernel): z_j by
  inverting an independent d_L^gw built on the hypergeometric closed form of
  the flat-LCDM distance, source-frame masses m_det / (1+z_j) and
  w_j = p(m1) p(m2|m1) from the separately pinned mass functions.
"""
import math

import mpmath as mp
import numpy as np
import pytest
from scipy.optimize import brentq

from _edges import edge_free
from synth import catalog as sc

C = 299792.458


@pytest.mark.parametrize("z", [1e-4, 0.01, 0.5, 1.5, 4.0, 9.5])
def test_dDc_dOm_closed_forms(orc, z):
    a = 1.0 + z
    eds = C / 70.0 * (a ** -0.5 - a ** -3.5 / 7.0 - 6.0 / 7.0)
    assert orc.dDc_dOm(z, 70.0, 1.0) == pytest.approx(eds, rel=1e-12, abs=1e-12 * C / 70.0)
    des = -C / 70.0 * 0.5 * ((a ** 4 - 1.0) / 4.0 - z)
    assert orc.dDc_dOm(z, 70.0, 0.0) == pytest.approx(des, rel=1e-12, abs=1e-12 * C / 70.0)


def _grad_case(mode, xi0, incomplete=False, seed_shift=0):
    cat = sc.config_catalog(2, n_events=4, n_pe=400, n_inj=20000, gal_median=40, kde_mode=mode)
    th = sc.config_hyperpoints(2, n=1 + seed_shift)[seed_shift].copy()
    th[2] = xi0
    cat = edge_free(cat, th)
    if incomplete:
        cat = sc.add_completeness(cat, seed=5, f_R=0.5)
    return cat, th


@pytest.mark.parametrize("mode,xi0,incomplete", [(1, 1.0, False), (1, 1.6, False), (0, 0.7, False),
                                                  (1, 1.3, True)])
def test_analytic_gradient_matches_central_differences(orc, mode, xi0, incomplete):
    cat, th = _grad_case(mode, xi0, incomplete)
    oc = orc.Catalog(cat)
    lnL, g, st = oc.grad(th)
    ref = oc.loglike(th)
    assert st == ref["status"] and lnL == pytest.approx(ref["lnL"], rel=1e-13, abs=0)
    fd = oc.grad_fd(th, rel_step=1e-4)
    # truncation of the central difference ~h^2 relative; the KDE support
    # edges of the oracle move grid points in and out of a support, jumps of
    # e^-18 of an event integral, i.e. <= ~1e-8 / (2 h |theta_k|)
    for k in range(12):
        tol = 2e-6 * abs(fd[k]) + 1e-4 / abs(th[k])
        assert abs(g[k] - fd[k]) <= tol, (k, g[k], fd[k])


def test_gradient_of_inadmissible_point_is_zero(orc):
    cat, th = _grad_case(1, 1.0)
    t = th.copy()
    t[7], t[8] = 60.0, 50.0
    lnL, g, st = orc.Catalog(cat).grad(t)
    assert lnL == -math.inf and st & orc.OUT_OF_SUPPORT and np.all(g == 0.0)


def _dc_hyp2f1(z, H0, Om):
    # int_0^z dz'/E = (1-Om)^(-1/2) [F(1+z) - F(1)], F(x) = x 2F1(1/3, 1/2; 4/3; -a x^3),
    # a = Om/(1-Om)
    mp.mp.dps = 30
    a = mp.mpf(Om) / (1 - mp.mpf(Om))
    F = lambda x: x * mp.hyp2f1(mp.mpf(1) / 3, mp.mpf(1) / 2, mp.mpf(4) / 3, -a * x ** 3)
    return float((F(1 + mp.mpf(z)) - F(mp.mpf(1))) / mp.sqrt(1 - mp.mpf(Om)) * C / H0)


@pytest.mark.parametrize("xi0,n", [(1.0, 1.91), (1.7, 2.5)])
def test_sample_reweighting_independent(orc, xi0, n):
    cat = sc.config_catalog(1, n_events=2, n_pe=40)
    th = sc.config_hyperpoints(1)[0].copy()
    th[2], th[3] = xi0, n
    oc = orc.Catalog(cat)
    so = cat["sample_off"]

    def dgw(z):  # Eq. dL-mg on the hypergeometric distance
        return (1.0 + z) * _dc_hyp2f1(z, th[0], th[1]) * (xi0 + (1.0 - xi0) * (1.0 + z) ** -n)

    for ev in range(cat["n_events"]):
        z, w, v = oc.samples(th, ev)
        for q in range(0, int(so[ev + 1] - so[ev]), 7):
            j = so[ev] + q
            d = cat["dL"][j]
            zr = brentq(lambda x: dgw(x) - d, 0.0, 10.0, xtol=1e-15, rtol=1e-15)
            assert v[q]
            assert z[q] == pytest.approx(zr, rel=1e-12, abs=1e-14)
            m1, m2 = cat["m1_det"][j] / (1.0 + zr), cat["m2_det"][j] / (1.0 + zr)
            wr = orc.p_m1(m1, th, cat["lambda_g"]) * orc.p_m2(m2, m1, th, cat["beta"])
            assert w[q] == pytest.approx(wr, rel=1e-10, abs=1e-300)
