"""Pins of the oracle's per-sample Jacobian variant (Eq. jacobian inside
Eq. like-integrals; reading: the KDE weight of PE sample j becomes
w_j / [(1+z_j)^3 |d d_L^gw/dz (z_j)|], the bandwidth keeps Scott's rule of the
weights w_j of Eq. gw-kernel, and the grid factor keeps psi(z) alone).

What fixes it independently of its own code:
  * the per-pixel KDE integrates (trapezoid rule) to the pixel's mean
    per-sample weight (1/N_k) sum_j w_j / Jac(z_j), and its first moment to
    (1/N_k) sum_j w_j z_j / Jac(z_j): the factor sits on each sample at its
    own redshift (a factor taken at the grid point, or a wrong sample,
    breaks both), with Jac from the oracle's d_L^gw derivative;
  * the grid-placement KDE of the same pixel keeps the mass (1/N_k) sum w_j;
  * the grid factors of the two placements differ by exactly the Jacobian;
  * the two placements give nearby event integrals (to first order in b).
"""
import numpy as np

import oracle
from synth import catalog as sc


def _trap(n_z, z_max):
    dz = z_max / (n_z - 1)
    tw = np.full(n_z, dz)
    tw[0] = tw[-1] = 0.5 * dz
    return tw, np.linspace(0.0, z_max, n_z)


def _setup(kde_mode=sc.KDE_MANY_1D):
    cat = sc.config_catalog(2, n_events=3, n_pe=2000, n_inj=2000, gal_median=30, kde_mode=kde_mode)
    th = sc.config_hyperpoints(2, n=1)[0].copy()
    th[2], th[3] = 1.4, 2.0  # modified GW propagation: a Jacobian that varies across the samples
    return cat, th


def test_per_sample_kde_mass_and_mean():
    cat, th = _setup()
    og = oracle.Catalog(cat, jacobian=oracle.JACOBIAN_GRID)
    op = oracle.Catalog(cat, jacobian=oracle.JACOBIAN_PER_SAMPLE)
    tw, za = _trap(cat["n_z"], cat["z_max"])
    so, po = cat["sample_off"], cat["pix_off"]
    checked = 0
    for ev in range(cat["n_events"]):
        z, w, v = og.samples(th, ev)
        pix = cat["pix_of_sample"][so[ev]:so[ev + 1]]
        assert og.bandwidth(th, ev) == op.bandwidth(th, ev)
        jac = np.array([(1.0 + zj) ** 3 * abs(oracle.J(zj, th)) if ok else 1.0 for zj, ok in zip(z, v)])
        for k in range(int(po[ev + 1] - po[ev])):
            sel = pix == k
            n_k = int(sel.sum())
            if n_k < 20:
                continue
            Kp = op.kde(th, ev, k)
            Kg = og.kde(th, ev, k)
            wk, zk, vk = w[sel], z[sel], v[sel]
            mass_p = np.sum(np.where(vk, wk / jac[sel], 0.0)) / n_k
            mean_p = np.sum(np.where(vk, wk * zk / jac[sel], 0.0)) / n_k
            mass_g = np.sum(np.where(vk, wk, 0.0)) / n_k
            assert abs((tw * Kp).sum() - mass_p) <= 1e-6 * mass_p, (ev, k)
            assert abs((tw * Kp * za).sum() - mean_p) <= 1e-6 * mean_p, (ev, k)
            assert abs((tw * Kg).sum() - mass_g) <= 1e-6 * mass_g, (ev, k)
            checked += 1
    assert checked >= 3


def test_single1d_event_kde_mass():
    cat, th = _setup(sc.KDE_SINGLE_1D)
    op = oracle.Catalog(cat, jacobian=oracle.JACOBIAN_PER_SAMPLE)
    tw, _ = _trap(cat["n_z"], cat["z_max"])
    for ev in range(cat["n_events"]):
        z, w, v = op.samples(th, ev)
        jac = np.array([(1.0 + zj) ** 3 * abs(oracle.J(zj, th)) if ok else 1.0 for zj, ok in zip(z, v)])
        K = op.kde(th, ev, -1)
        mass = np.sum(np.where(v, w / jac, 0.0)) / z.size
        assert abs((tw * K).sum() - mass) <= 1e-6 * mass, ev


def test_grid_factors_differ_by_the_jacobian():
    cat, th = _setup()
    Fg = oracle.Catalog(cat).grid_factor(th)
    Fp = oracle.Catalog(cat, jacobian=oracle.JACOBIAN_PER_SAMPLE).grid_factor(th)
    _, za = _trap(cat["n_z"], cat["z_max"])
    jac = np.array([(1.0 + z) ** 3 * abs(oracle.J(z, th)) for z in za])
    np.testing.assert_allclose(Fg * jac, Fp, rtol=1e-13, atol=0.0)
    np.testing.assert_allclose(Fp, [oracle.psi(z, th) for z in za], rtol=1e-13, atol=0.0)


def test_placements_agree_to_first_order_in_b():
    """Moving 1/Jac from z_a to z_j changes the integrand by ~ (z_a - z_j)
    d(1/Jac)/dz inside the kernel, and the galaxy term, sharper than the
    kernel, does not cancel the odd part: |Delta ln I| <= 2 b max|d ln Jac/dz|."""
    cat, th = _setup()
    og = oracle.Catalog(cat)
    op = oracle.Catalog(cat, jacobian=oracle.JACOBIAN_PER_SAMPLE)
    d = np.array([op.event_lnI(th, ev) - og.event_lnI(th, ev) for ev in range(cat["n_events"])])
    assert np.all(np.isfinite(d)) and np.any(d != 0.0)
    for ev in range(cat["n_events"]):
        z, _, v = og.samples(th, ev)
        zz = np.linspace(z[v].min(), z[v].max(), 64)
        lj = lambda x: 3.0 * np.log1p(x) + np.log(abs(oracle.J(x, th)))
        slope = max(abs(lj(x + 1e-5) - lj(x - 1e-5)) / 2e-5 for x in zz)
        b = og.bandwidth(th, ev)
        assert abs(d[ev]) <= 2.0 * b * slope, (ev, d[ev], b, slope)
