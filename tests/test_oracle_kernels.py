"""Pins of the oracle's Epanechnikov kernel option (Sec. 2.3 offers Gaussian
and Epanechnikov 1-D kernels; reading: (3/4)(1 - u^2) on |u| <= 1 with
width h = sqrt(5) b, whose variance equals the Gaussian's b^2).

What fixes it independently of its own code:
  * compact support: a sample contributes nothing beyond h of itself, and
    something everywhere inside;
  * unit mass: the KDE sums (trapezoid rule) to the mean weight, as the
    Gaussian one does;
  * the kernel's variance is b^2 for both shapes: the KDE's variance is the
    weighted sample variance plus b^2, whichever the kernel;
  * the binned form of the Epanechnikov KDE equals the unbinned one for
    samples on grid nodes (as for the Gaussian).
"""
import numpy as np

E = 1  # oracle.EPANECHNIKOV


def _trap(n_z, z_max):
    dz = z_max / (n_z - 1)
    tw = np.full(n_z, dz)
    tw[0] = tw[-1] = 0.5 * dz
    return tw, np.linspace(0.0, z_max, n_z)


def test_compact_support(orc):
    n_z, z_max, b = 3001, 1.5, 0.02
    h = np.sqrt(5.0) * b
    z0 = 0.7003
    K = orc.kde_arrays([z0], [1.0], b, n_z, z_max, kernel=E)
    _, za = _trap(n_z, z_max)
    d = np.abs(za - z0)
    assert np.all(K[d > h * (1 + 1e-12)] == 0.0)
    assert np.all(K[d < h * (1 - 1e-9)] > 0.0)
    # the Gaussian of the same b reaches beyond h
    Kg = orc.kde_arrays([z0], [1.0], b, n_z, z_max)
    assert np.any(Kg[d > 1.2 * h] > 0.0)


def test_unit_mass_and_variance(orc):
    n_z, z_max = 20001, 1.5
    tw, za = _trap(n_z, z_max)
    rng = np.random.default_rng(11)
    z = rng.normal(0.7, 0.04, 400)
    w = rng.uniform(0.1, 1.0, 400)
    b = 0.015
    mean_w = np.average(z, weights=w)
    var_w = np.average((z - mean_w) ** 2, weights=w)
    for kernel in (0, E):
        K = orc.kde_arrays(z, w, b, n_z, z_max, kernel=kernel)
        mass = (tw * K).sum()
        assert abs(mass - w.mean()) <= 1e-6 * w.mean(), kernel
        m1 = (tw * K * za).sum() / mass
        var = (tw * K * (za - m1) ** 2).sum() / mass
        assert abs(m1 - mean_w) <= 1e-8, kernel
        assert abs(var - (var_w + b * b)) <= 1e-5 * (var_w + b * b), (kernel, var, var_w + b * b)


def test_binned_epanechnikov_on_nodes(orc):
    n_z, z_max = 301, 1.5
    nodes = z_max * np.arange(n_z) / (n_z - 1)
    rng = np.random.default_rng(12)
    z = nodes[rng.integers(80, 220, 300)]
    w = rng.uniform(0.2, 2.0, 300)
    K = orc.kde_arrays(z, w, 0.03, n_z, z_max, kernel=E)
    Kb = orc.kde_arrays(z, w, 0.03, n_z, z_max, binned=True, kernel=E)
    assert K.max() > 0.0
    np.testing.assert_allclose(Kb, K, rtol=1e-12, atol=1e-12 * K.max())
