"""Pins of the oracle's "3D" kernel (Sec. 2.3, the cross-check variant):
a weighted Gaussian KDE over (z, x, y), (x, y) a flat local sky chart of the
event, Scott's rule in three dimensions (n_eff^(-1/7) times the weighted
covariance), evaluated at (z_a, pixel centre) on the grid portion holding the
samples.

What fixes it independently of its own code:
  * scipy.stats.gaussian_kde with the same weights and Scott's rule (the
    library routine the reading names) gives the same density, times the
    mean weight (sum w / N), at every grid point of the support;
  * the KDE vanishes outside the samples' range +- 6 sqrt(H_zz);
  * the 3D and many-1D kernels estimate the same event integral (they agree
    within the kernels' smoothing: Sec. 2.3 and the paper's appendix report
    the three KDE variants consistent).
"""
import numpy as np
from scipy.stats import gaussian_kde

import oracle
from synth import catalog as sc


def _setup():
    cat = sc.config_catalog(2, n_events=3, n_pe=600, n_inj=2000, gal_median=30, kde_mode=sc.KDE_3D)
    th = sc.config_hyperpoints(2, n=1)[0]
    return cat, th


def test_matches_scipy_weighted_gaussian_kde():
    cat, th = _setup()
    oc = oracle.Catalog(cat)
    so, po = cat["sample_off"], cat["pix_off"]
    za = np.linspace(0.0, cat["z_max"], cat["n_z"])
    for ev in range(cat["n_events"]):
        z, w, v = oc.samples(th, ev)
        xy = cat["sky_xy"][so[ev]:so[ev + 1]]
        kde = gaussian_kde(np.vstack([z[v], xy[v, 0], xy[v, 1]]), weights=w[v], bw_method="scott")
        H = oc.kde3_bandwidth(th, ev)
        np.testing.assert_allclose(H, kde.covariance, rtol=1e-10, atol=0.0)
        scale = w[v].sum() / z.size
        zlo = z[v].min() - 6.0 * np.sqrt(H[0, 0])
        zhi = z[v].max() + 6.0 * np.sqrt(H[0, 0])
        inside = (za >= zlo) & (za <= zhi)
        for k in range(min(4, int(po[ev + 1] - po[ev]))):
            K = oc.kde3(th, ev, k)
            P = cat["pix_xy"][po[ev] + k]
            pts = np.vstack([za[inside], np.full(inside.sum(), P[0]), np.full(inside.sum(), P[1])])
            ref = scale * kde(pts)
            np.testing.assert_allclose(K[inside], ref, rtol=1e-9, atol=1e-12 * ref.max())
            assert np.all(K[~inside] == 0.0)


def test_3d_and_many1d_event_integrals_agree():
    """With the many-1D sky factor of Eq. gw-kernel-many1d (the 2-D KDE of the
    samples' sky positions at each pixel centre, scipy's Scott rule), the 3D
    and many-1D kernels estimate the same integral: they differ only through
    the kernels' smoothing (0.16 at most in ln I_i on this catalog)."""
    cat = sc.config_catalog(2, n_events=6, n_pe=1500, n_inj=2000, gal_median=30, kde_mode=sc.KDE_3D)
    th = sc.config_hyperpoints(2, n=1)[0]
    so, po = cat["sample_off"], cat["pix_off"]
    m1 = dict(cat)
    S = cat["sky_S"].copy()
    for ev in range(cat["n_events"]):
        xy = cat["sky_xy"][so[ev]:so[ev + 1]]
        S[po[ev]:po[ev + 1]] = gaussian_kde(xy.T)(cat["pix_xy"][po[ev]:po[ev + 1]].T)
    m1["sky_S"] = S
    o3 = oracle.Catalog(cat)
    om = oracle.Catalog(m1, kde_mode=sc.KDE_MANY_1D)
    d = np.array([o3.event_lnI(th, ev) - om.event_lnI(th, ev) for ev in range(cat["n_events"])])
    assert np.all(np.isfinite(d)) and np.any(d != 0.0)
    assert np.all(np.abs(d) < 0.25), d
