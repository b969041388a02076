"""Pins of the oracle's population model (Sec. 3.1): normalisation of the
mass densities by independent quadrature, support edges, and the
Madau-Dickinson peak position, which follows from the shape alone."""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import minimize_scalar

FID = np.array([70.0, 0.3, 1.0, 1.91, 3.4, 34.0, 3.6, 5.0, 100.0, 2.7, 3.0, 2.0])


def th(alpha=3.4, mu=34.0, sg=3.6, mmin=5.0, mmax=100.0, gamma=2.7, kappa=3.0, zp=2.0):
    t = FID.copy()
    t[4:12] = [alpha, mu, sg, mmin, mmax, gamma, kappa, zp]
    return t


@pytest.mark.parametrize("kw", [dict(), dict(alpha=1.0), dict(alpha=1.5, mu=10.0),
                                dict(alpha=8.0, mmin=2.5, mmax=60.0), dict(mu=120.0, sg=5.0),
                                dict(mu=3.0, sg=0.4, mmin=4.0)])
@pytest.mark.parametrize("lam", [0.0, 0.039, 0.9])
def test_primary_mass_normalised(orc, kw, lam):
    t = th(**kw)
    pts = [min(max(t[5], t[7]), t[8])]
    val = quad(lambda m: orc.p_m1(m, t, lam), t[7], t[8], points=pts, limit=200,
               epsabs=0, epsrel=1e-12)[0]
    assert val == pytest.approx(1.0, rel=1e-9)


def test_primary_mass_support(orc):
    t = th()
    assert orc.p_m1(4.999, t, 0.039) == 0.0
    assert orc.p_m1(100.001, t, 0.039) == 0.0
    assert orc.p_m1(5.0, t, 0.039) > 0.0
    # pure power law away from the peak has slope -alpha
    r = orc.p_m1(80.0, t, 0.0) / orc.p_m1(40.0, t, 0.0)
    assert r == pytest.approx(2.0 ** -3.4, rel=1e-13)


@pytest.mark.parametrize("beta", [1.1, 0.0, -1.0, -3.0, 6.0])
@pytest.mark.parametrize("m1", [5.5, 20.0, 95.0])
def test_secondary_mass_normalised(orc, beta, m1):
    t = th()
    val = quad(lambda m: orc.p_m2(m, m1, t, beta), t[7], m1, epsabs=0, epsrel=1e-12)[0]
    assert val == pytest.approx(1.0, rel=1e-9)
    assert orc.p_m2(m1 * 1.0001, m1, t, beta) == 0.0
    assert orc.p_m2(t[7] * 0.999, m1, t, beta) == 0.0
    assert orc.p_m2(t[7], t[7] * 0.99, t, beta) == 0.0  # m1 below m_min


@pytest.mark.parametrize("gamma,kappa,zp", [(2.7, 3.0, 2.0), (1.0, 5.0, 1.0), (5.0, 2.0, 3.0)])
def test_madau_dickinson_peak(orc, gamma, kappa, zp):
    # d psi/dz = 0 where gamma (1 + x) = (gamma + kappa) x, x = ((1+z)/(1+z_p))^(gamma+kappa)
    t = th(gamma=gamma, kappa=kappa, zp=zp)
    z_star = (1 + zp) * (gamma / kappa) ** (1.0 / (gamma + kappa)) - 1
    res = minimize_scalar(lambda z: -orc.psi(z, t), bounds=(0.0, 8.0), method="bounded",
                          options=dict(xatol=1e-10))
    assert res.x == pytest.approx(z_star, abs=1e-6)
    # low-z slope d ln psi / d ln(1+z) -> gamma when (1+z)/(1+z_p) -> 0
    t2 = th(gamma=gamma, kappa=kappa, zp=1e6)
    e = 1e-6
    slope = (np.log(orc.psi(e, t2)) - np.log(orc.psi(0.0, t2))) / np.log1p(e)
    assert slope == pytest.approx(gamma, rel=1e-5)
