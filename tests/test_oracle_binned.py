"""Pins of the oracle's binned-KDE option (the paper bins the weighted PE
samples of each pixel or event, Sec. 2.3; reading: linear binning onto the
grid lattice z_n = n dz, then the KDE of the nodes with the samples'
bandwidth and support).

What fixes the binned oracle independently of its own code:
  * linear binning splits a sample between the two bracketing nodes in
    proportion to its distance from the other one, so it keeps the total
    weight and the weighted mean exactly (brute force on a small set);
  * samples that sit on nodes are their own bins: the binned KDE equals the
    unbinned one;
  * a Gaussian KDE whose windows lie inside the grid sums, by the trapezoid
    rule, to sum(w)/N for both forms (the Gaussian's Riemann sum at b >> dz);
  * the binned KDE converges to the unbinned one at second order in dz
    (halving dz divides the error by ~4);
  * per event, |ln I_binned - ln I| <= (dz/b)^2 / 8, the stated error bound.
"""
import numpy as np
import pytest

from synth import catalog as sc


def test_linear_bins_split_and_conservation(orc):
    dz = 0.01
    cb, lost = orc.linear_bins([2.25 * dz], [2.0], dz, 0, 6)
    assert lost == 0
    np.testing.assert_allclose(cb, [0, 0, 1.5, 0.5, 0, 0], rtol=0, atol=1e-15)
    rng = np.random.default_rng(5)
    z = rng.uniform(0.1, 0.9, 4000)
    w = rng.gamma(2.0, 1.0, 4000)
    b0, nb = 5, 92
    cb, lost = orc.linear_bins(z, w, dz, b0, nb)
    assert lost == 0
    zn = (b0 + np.arange(nb)) * dz
    assert abs(cb.sum() - w.sum()) <= 1e-12 * w.sum()
    assert abs((cb * zn).sum() - (w * z).sum()) <= 1e-12 * (w * z).sum()
    assert np.all(cb >= 0.0)
    # nodes outside the kept range are counted, not silently added
    _, lost = orc.linear_bins([0.5 * dz, 50.5 * dz], [1.0, 1.0], dz, 10, 20)
    assert lost == 4
    # zero-weight samples and missing redshifts contribute nothing
    cb, lost = orc.linear_bins([3.5 * dz, np.inf], [0.0, 1.0], dz, 0, 6)
    assert lost == 0 and np.all(cb == 0.0)


def test_samples_on_nodes_bin_to_themselves(orc):
    n_z, z_max = 301, 1.5
    nodes = z_max * np.arange(n_z) / (n_z - 1)
    rng = np.random.default_rng(6)
    idx = rng.integers(60, 240, 500)
    z = nodes[idx]
    w = rng.uniform(0.2, 2.0, 500)
    b = 0.03
    K = orc.kde_arrays(z, w, b, n_z, z_max)
    Kb = orc.kde_arrays(z, w, b, n_z, z_max, binned=True)
    assert K.max() > 0.0
    np.testing.assert_allclose(Kb, K, rtol=1e-12, atol=1e-12 * K.max())


def test_binned_and_unbinned_kde_integrate_to_the_mean_weight(orc):
    n_z, z_max = 1000, 1.5
    dz = z_max / (n_z - 1)
    rng = np.random.default_rng(7)
    z = rng.normal(0.7, 0.05, 3000)
    w = rng.uniform(0.0, 1.0, 3000)
    b = 0.012
    for binned in (False, True):
        K = orc.kde_arrays(z, w, b, n_z, z_max, binned=binned)
        tw = np.full(n_z, dz)
        tw[0] = tw[-1] = 0.5 * dz
        assert abs((tw * K).sum() - w.mean()) <= 1e-8 * w.mean(), binned


def test_binned_kde_converges_at_second_order(orc):
    z_max, b = 1.5, 0.02
    rng = np.random.default_rng(8)
    z = rng.normal(0.6, 0.06, 2000)
    w = rng.uniform(0.1, 1.0, 2000)
    errs = []
    for n_z in (301, 601, 1201):
        K = orc.kde_arrays(z, w, b, n_z, z_max)
        Kb = orc.kde_arrays(z, w, b, n_z, z_max, binned=True)
        errs.append(np.abs(Kb - K).max() / K.max())
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.0 <= e0 / e1 <= 5.0, errs
    # and the size matches the variance the binning adds, <= dz^2/4 per sample
    dz = z_max / 300
    assert errs[0] <= 0.5 * (dz / b) ** 2


@pytest.mark.parametrize("kde_mode", [sc.KDE_MANY_1D, sc.KDE_SINGLE_1D])
def test_event_error_within_the_stated_bound(orc, kde_mode):
    cat = sc.config_catalog(2, n_events=5, n_pe=1500, n_inj=2000, gal_median=50, kde_mode=kde_mode)
    oc = orc.Catalog(cat)
    dz = cat["z_max"] / (cat["n_z"] - 1)
    for th in sc.config_hyperpoints(2, n=2):
        for ev in range(cat["n_events"]):
            b = oc.bandwidth(th, ev)
            d = oc.event_lnI(th, ev, binned=True) - oc.event_lnI(th, ev)
            assert abs(d) <= (dz / b) ** 2 / 8, (ev, d, dz / b)
