"""Pins of the oracle's likelihood assembly (Eqs. hyperlike, like-integrals,
gw-kernel-*, p-cat, bias) against identities that do not reuse its code:
unit KDE normalisation, the Gaussian product identity, an analytic
selection term for injections drawn from the population itself, invariance
of ln L under constant rescalings of p_pop, many-1D = single-1D at one
pixel, and brute-force continuous quadrature on a tiny catalog."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import _catalogs as tc


def _event(rng, z0, n, t, rel=0.03, npix=1, gal=None, sig=0.02, dgw=None):
    dgw = dgw or (lambda z: None)
    d0 = dgw(z0)
    dL = d0 * (1 + rel * rng.standard_normal(n))
    m1 = (30 + 3 * rng.standard_normal(n)) * (1 + z0)
    m2 = (24 + 3 * rng.standard_normal(n)) * (1 + z0)
    m1, m2 = np.maximum(m1, m2), np.minimum(m1, m2)
    pix = rng.integers(0, npix, n)
    counts = np.bincount(pix, minlength=npix)
    S = counts / (n * 1e-4)
    if gal is None:
        gal = [[z0 + 0.01 * (k - 1), z0 + 0.03] for k in range(npix)]
    return dict(dL=dL, m1d=m1, m2d=m2, pix=pix, S=S, gal_z=gal,
                gal_sigma=[[sig] * len(g) for g in gal])


def test_kde_unit_normalisation(orc):
    rng = np.random.default_rng(1)
    t = tc.theta()
    ev = _event(rng, 0.5, 300, t, dgw=lambda z: orc.dL_gw(z, t))
    cat = orc.Catalog(tc.build([ev], n_z=4001, kde_mode=0))
    K = cat.kde(t, 0)
    z, w, v = cat.samples(t, 0)
    dz = 1.5 / 4000
    wts = np.full(4001, dz); wts[0] = wts[-1] = dz / 2
    assert np.sum(wts * K) == pytest.approx(np.sum(w) / 300, rel=1e-10)
    assert v.all() and (w > 0).all()


def test_gaussian_product_identity(orc):
    """F := 1 and dV/dz := 1 (hooks): then I = sum_k S_k (1/N_k)(1/N_gal)
    sum_{j in k} w_j sum_{g in k} N(z_g; z_j, sqrt(b^2 + s_g^2)) / Z_g."""
    rng = np.random.default_rng(2)
    t = tc.theta(Xi0=1.4)
    ev = _event(rng, 0.6, 200, t, npix=2, sig=0.01, dgw=lambda z: orc.dL_gw(z, t))
    n_z = 20001
    for mode in (0, 1):
        cat = orc.Catalog(tc.build([ev], n_z=n_z, kde_mode=mode))
        hk = orc.hooks(flags=3)
        z, w, v = cat.samples(t, 0)
        b = cat.bandwidth(t, 0)
        ntot = sum(len(g) for g in ev["gal_z"])
        expect = 0.0
        for k in range(2):
            sel = ev["pix"] == k
            Nk = sel.sum() if mode == 1 else 200
            zz = z if mode == 0 else z[sel]
            ww = w if mode == 0 else w[sel]
            for zg, sg in zip(ev["gal_z"][k], ev["gal_sigma"][k]):
                s = math.sqrt(b * b + sg * sg)
                dens = np.exp(-0.5 * ((zg - zz) / s) ** 2) / (math.sqrt(2 * math.pi) * s)
                expect += ev["S"][k] / Nk / ntot * np.sum(ww * dens)
        got = math.exp(cat.event_lnI(t, 0, hk))
        assert got == pytest.approx(expect, rel=1e-9)


def test_many_equals_single_at_one_pixel(orc):
    from synth import catalog as sc
    cat = sc.config_catalog(1)
    t = tc.theta()
    a = orc.Catalog(cat, kde_mode=1).loglike(t)
    b = orc.Catalog(cat, kde_mode=0).loglike(t)
    assert a["lnL"] == pytest.approx(b["lnL"], rel=1e-13, abs=1e-11)
    np.testing.assert_allclose(a["lnI"], b["lnI"], rtol=1e-13)


@pytest.fixture(scope="module")
def small_c2():
    from synth import catalog as sc
    return sc.config_catalog(2, variant=1, n_events=4, n_pe=300, n_inj=4000, n_z=400, gal_median=60)


@pytest.mark.parametrize("scale", [dict(psi_scale=3.7), dict(mass_scale=0.21),
                                   dict(psi_scale=1e-3, mass_scale=40.0)])
def test_ln_l_invariant_under_ppop_rescaling(orc, small_c2, scale):
    """A constant factor in p_pop cancels between prod I_i and xi^N_obs
    (Eq. hyperlike); psi is only defined up to a constant (Sec. 3.1)."""
    cat = orc.Catalog(small_c2)
    t = tc.theta(H0=72.0, Xi0=1.2)
    ref = cat.loglike(t)
    got = cat.loglike(t, orc.hooks(**scale))
    assert got["lnL"] == pytest.approx(ref["lnL"], abs=1e-9)
    assert got["lnI"] != pytest.approx(ref["lnI"], rel=1e-3)


def _self_drawn_injections(orc, t, n, rng):
    """Injections whose stored draw density is p_pop itself (detector frame):
    pi_inj = q(z) p(m1,m2) / [(1+z)^2 J], q = psi p_z / ((1+z) C).  Then every
    s_j equals C = int_0^zmax psi p_z / (1+z) dz, whatever (z_j, m_j) are."""
    H0, zmax = t[0], 1.5
    pz = lambda z: tc.eds_dvdz(z, H0) / tc.eds_vc(zmax, H0)
    Cn = quad(lambda z: orc.psi(z, t) * pz(z) / (1 + z), 0, zmax, epsrel=1e-13, epsabs=0)[0]
    z = rng.uniform(0.02, 1.45, n)
    m1 = rng.uniform(8, 90, n)
    m2 = t[7] + rng.uniform(0.05, 0.95, n) * (m1 - t[7])
    d = np.array([tc.eds_dgw(x, t) for x in z])
    lp = []
    for x, a, b in zip(z, m1, m2):
        pm = orc.p_m1(a, t, 0.039) * orc.p_m2(b, a, t, 1.1)
        q = orc.psi(x, t) * pz(x) / ((1 + x) * Cn)
        lp.append(math.log(q * pm / ((1 + x) ** 2 * tc.eds_J(x, t))))
    return dict(dL=d, m1d=m1 * (1 + z), m2d=m2 * (1 + z), log_pi=np.array(lp)), Cn


@pytest.mark.parametrize("xi0,n", [(1.0, 1.91), (1.8, 2.7), (0.6, 1.91)])
def test_selection_analytic(orc, xi0, n):
    rng = np.random.default_rng(3)
    t = tc.theta(Om=1.0, Xi0=xi0, n=n, H0=68.0)
    inj, Cn = _self_drawn_injections(orc, t, 400, rng)
    ev = _event(rng, 0.5, 50, t, dgw=lambda z: tc.eds_dgw(z, t))
    ndet = 400
    for ntot in (ndet, 3 * ndet):
        cat = orc.Catalog(tc.build([ev], n_z=256, inj=inj, n_inj_total=ntot))
        xi, neff, s = cat.selection(t, want_s=True)
        np.testing.assert_allclose(s, Cn, rtol=1e-11)
        assert xi == pytest.approx(Cn * ndet / ntot, rel=1e-11)
        if ntot > ndet:
            assert neff == pytest.approx(ndet / (1 - ndet / ntot), rel=1e-6)


def test_brute_force_continuous_quadrature(orc):
    """Tiny catalog, EdS background: the oracle's grid sum at N_z = 20001
    against scipy quad of the continuous Eq. like-integrals with continuous
    galaxy normalisation.  The difference is the grid's discretisation error."""
    rng = np.random.default_rng(4)
    t = tc.theta(Om=1.0, Xi0=1.8, n=2.7, H0=66.0)
    dg = lambda z: tc.eds_dgw(z, t)
    evs = [_event(rng, 0.45, 40, t, npix=2, sig=0.02, dgw=dg,
                  gal=[[0.40, 0.47, 0.52], [0.43, 0.49, 0.61]]),
           _event(rng, 0.8, 40, t, npix=1, sig=0.02, dgw=dg, gal=[[0.74, 0.8, 0.83]])]
    zmax = 1.5
    H0 = t[0]
    for mode in (0, 1):
        raw = tc.build(evs, n_z=20001, kde_mode=mode)
        cat = orc.Catalog(raw)
        ntot = raw["n_gal_total"]
        F = lambda z: orc.psi(z, t) / ((1 + z) ** 3 * tc.eds_J(z, t))
        for i, ev in enumerate(evs):
            z, w, v = cat.samples(t, i)
            b = cat.bandwidth(t, i)
            phi = lambda x, zz, ww: np.sum(ww * np.exp(-0.5 * ((x - zz) / b) ** 2)) / (math.sqrt(2 * math.pi) * b)
            I = 0.0
            for k in range(len(ev["S"])):
                sel = ev["pix"] == k if mode == 1 else np.ones(len(z), bool)
                Nk = int(sel.sum())
                gz, gs = ev["gal_z"][k], ev["gal_sigma"][k]
                Zg = [quad(lambda x: math.exp(-0.5 * ((x - a) / s) ** 2) / (math.sqrt(2 * math.pi) * s)
                           * tc.eds_dvdz(x, H0), 0, zmax, points=[a], epsrel=1e-12)[0]
                      for a, s in zip(gz, gs)]
                G = lambda x: tc.eds_dvdz(x, H0) / ntot * sum(
                    math.exp(-0.5 * ((x - a) / s) ** 2) / (math.sqrt(2 * math.pi) * s) / Zg[m]
                    for m, (a, s) in enumerate(zip(gz, gs)))
                zz, ww = (z[sel], w[sel]) if mode == 1 else (z, w)
                integrand = lambda x: phi(x, zz, ww) / Nk * F(x) * G(x)
                # each KDE lives on the grid segment that holds its samples,
                # widened by 6 bandwidths (Sec. 2.3)
                lo, hi = max(0.0, zz.min() - 6 * b), min(zmax, zz.max() + 6 * b)
                pts = [a for a in gz if lo < a < hi]
                I += ev["S"][k] * quad(integrand, lo, hi, points=pts or None, limit=400, epsrel=1e-12)[0]
            got = cat.event_lnI(t, i)
            assert got == pytest.approx(math.log(I), abs=1e-8)


def test_samples_beyond_table_get_zero_weight(orc):
    rng = np.random.default_rng(5)
    t = tc.theta()
    ev = _event(rng, 0.5, 20, t, dgw=lambda z: orc.dL_gw(z, t))
    ev["dL"][3] = orc.dL_gw(10.0, t) * 1.5
    cat = orc.Catalog(tc.build([ev], n_z=256))
    z, w, v = cat.samples(t, 0)
    assert not v[3] and w[3] == 0.0 and v.sum() == 19


def test_status_codes(orc, small_c2):
    cat = orc.Catalog(small_c2)
    r = cat.loglike(tc.theta(m_min=60.0, m_max=50.0))
    assert r["lnL"] == -math.inf and r["status"] == orc.OUT_OF_SUPPORT
    r = cat.loglike(tc.theta(Xi0=0.01, n=40.0))
    assert r["lnL"] == -math.inf and r["status"] == orc.NONMONOTONE
    # no sample survives the mass cut: I_i = 0 -> -inf, never NaN
    r = cat.loglike(tc.theta(m_min=150.0, m_max=190.0))
    assert r["lnL"] == -math.inf and r["status"] & orc.OUT_OF_SUPPORT
    r = cat.loglike(tc.theta())
    assert math.isfinite(r["lnL"])
    few = dict(small_c2)
    for k in ("inj_dL", "inj_m1d", "inj_m2d", "inj_log_pi"):
        few[k] = small_c2[k][:3]
    r = orc.Catalog(few).loglike(tc.theta())
    assert r["status"] & orc.NEFF_LOW


def test_bandwidth_rule(orc, small_c2):
    """Scott's rule with the weighted effective sample size (reading R2)."""
    cat = orc.Catalog(small_c2)
    t = tc.theta()
    for ev in range(small_c2["n_events"]):
        z, w, v = cat.samples(t, ev)
        W1 = w.sum()
        mean = (w * z).sum() / W1
        var = (w * (z - mean) ** 2).sum() / W1
        neff = W1 ** 2 / (w ** 2).sum()
        assert cat.bandwidth(t, ev) == pytest.approx(math.sqrt(var) * neff ** -0.2, rel=1e-12)
