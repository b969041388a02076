"""Pins of the oracle's incomplete-catalog option (Eqs. p-gal, p-miss, f-R:
p_gal = f_R p_cat + (1 - f_R) p_miss, the missing galaxies homogeneous in
comoving volume).  Reading: the completeness of each pixel on the grid, the
pixel's solid angle and f_R are inputs; the pixel's galaxy mass is
f_R G_cat + (dOmega/4 pi)(1 - P_compl) dV_c/dz / V_c(z_max).

What fixes it independently of its own code:
  * a fully complete catalog (P_compl = 1, f_R = 1) is the complete one;
  * with P_compl = 1 the missing term vanishes, so any f_R only scales the
    catalog term;
  * with nothing in the catalog (f_R = 0, P_compl = 0) the pixel holds the
    homogeneous prior alone, whose redshift integral is the pixel's share of
    the sky, dOmega / 4 pi (dV_c/dz integrates to V_c(z_max)).
"""
import numpy as np

from synth import catalog as sc


def _cats():
    cat = sc.config_catalog(2, n_events=3, n_pe=600, n_inj=2000, gal_median=40)
    return cat, sc.add_completeness(cat, seed=8)


def test_complete_limit_is_the_complete_catalog(orc):
    cat, ic = _cats()
    full = dict(ic)
    full["completeness"] = np.ones_like(ic["completeness"])
    full["f_R"] = 1.0
    th = sc.config_hyperpoints(2, n=1)[0]
    oc, of = orc.Catalog(cat), orc.Catalog(full)
    for ev in range(cat["n_events"]):
        np.testing.assert_array_equal(of.galaxy_profile(th, ev, 0), oc.galaxy_profile(th, ev, 0))
        assert of.event_lnI(th, ev) == oc.event_lnI(th, ev)
    half = dict(full)
    half["f_R"] = 0.5
    oh = orc.Catalog(half)
    np.testing.assert_allclose(oh.galaxy_profile(th, 1, 0), 0.5 * oc.galaxy_profile(th, 1, 0), rtol=1e-15)


def test_empty_catalog_pixel_mass_is_its_sky_fraction(orc):
    _, ic = _cats()
    empty = dict(ic)
    empty["completeness"] = np.zeros_like(ic["completeness"])
    empty["f_R"] = 0.0
    oe = orc.Catalog(empty)
    th = sc.config_hyperpoints(2, n=1)[0]
    n_z, z_max = ic["n_z"], ic["z_max"]
    tw = np.full(n_z, z_max / (n_z - 1))
    tw[0] = tw[-1] = 0.5 * tw[0]
    po = ic["pix_off"]
    for ev in range(ic["n_events"]):
        for k in range(int(po[ev + 1] - po[ev])):
            G = oe.galaxy_profile(th, ev, k)
            share = ic["pix_area"][po[ev] + k] / (4.0 * np.pi)
            assert abs((tw * G).sum() - share) <= 1e-5 * share, (ev, k)


def test_incompleteness_changes_the_event_integral(orc):
    cat, ic = _cats()
    th = sc.config_hyperpoints(2, n=1)[0]
    oc, oi = orc.Catalog(cat), orc.Catalog(ic)
    d = [oi.event_lnI(th, ev) - oc.event_lnI(th, ev) for ev in range(cat["n_events"])]
    assert all(np.isfinite(d)) and max(abs(x) for x in d) > 1e-3
