"""Pins of the oracle's cosmology (Eqs. dL-em, dL-mg, jacobian) against
closed forms, a hypergeometric identity, a printed number of the paper and
its own inverse, independent of the oracle's quadrature."""
import math
import os

import mpmath as mp
import numpy as np
import pytest
from scipy.integrate import quad

C = 299792.458
FID = np.array([70.0, 0.3, 1.0, 1.91, 3.4, 34.0, 3.6, 5.0, 100.0, 2.7, 3.0, 2.0])
ZS = [1e-4, 0.01, 0.3, 1.0, 1.5, 3.0, 9.5]


def th(**kw):
    t = FID.copy()
    names = ["H0", "Om", "Xi0", "n", "alpha", "mu_g", "sigma_g", "m_min", "m_max", "gamma", "kappa", "z_p"]
    for k, v in kw.items():
        t[names.index(k)] = v
    return t


@pytest.mark.parametrize("z", ZS)
def test_einstein_de_sitter_closed_form(orc, z):
    # Om = 1: d_L = (2c/H0)(1+z)(1 - (1+z)^(-1/2))
    for H0 in (50.0, 70.0, 140.0):
        # 1 - (1+z)^(-1/2) written without cancellation: z / (s (1 + s)), s = sqrt(1+z)
        s = math.sqrt(1 + z)
        exact = 2 * C / H0 * (1 + z) * z / (s * (1 + s))
        assert orc.dL_em(z, H0, 1.0) == pytest.approx(exact, rel=1e-13, abs=0)


@pytest.mark.parametrize("z", ZS)
def test_de_sitter_closed_form(orc, z):
    # Om = 0: E = 1, d_L = (1+z) c z / H0
    exact = (1 + z) * C * z / 70.0
    assert orc.dL_em(z, 70.0, 0.0) == pytest.approx(exact, rel=1e-13, abs=0)


def _dc_hyp2f1(z, H0, Om):
    # int_0^z dz'/sqrt(Om(1+z')^3 + 1 - Om)
    #   = (1-Om)^(-1/2) [F(1+z) - F(1)],  F(x) = x 2F1(1/3, 1/2; 4/3; -a x^3),
    # a = Om/(1-Om): the textbook identity int dx (1 + a x^3)^(-1/2).
    mp.mp.dps = 40
    a = mp.mpf(Om) / (1 - mp.mpf(Om))
    F = lambda x: x * mp.hyp2f1(mp.mpf(1) / 3, mp.mpf(1) / 2, mp.mpf(4) / 3, -a * x ** 3)
    val = (F(1 + mp.mpf(z)) - F(mp.mpf(1))) / mp.sqrt(1 - mp.mpf(Om))
    return float(val * C / H0)


@pytest.mark.parametrize("Om", [0.05, 0.25, 0.3, 0.7, 0.95])
@pytest.mark.parametrize("z", [0.01, 0.5, 1.5, 4.0, 10.0])
def test_flat_lcdm_hypergeometric(orc, Om, z):
    assert orc.Dc(z, 70.0, Om) == pytest.approx(_dc_hyp2f1(z, 70.0, Om), rel=1e-13, abs=0)


def test_xi0_one_reduces_to_em(orc):
    for n in (1.0, 1.91, 5.0):
        t = th(Xi0=1.0, n=n)
        for z in ZS:
            assert orc.dL_gw(z, t) == orc.dL_em(z, 70.0, 0.3)
    for xi0 in (0.1, 0.6, 1.8, 7.0):
        assert orc.Xi(0.0, xi0, 2.7) == pytest.approx(1.0, abs=1e-15)
        # high-z limit of Eq. dL-mg
        assert orc.Xi(1e8, xi0, 2.7) == pytest.approx(xi0, rel=1e-12)


@pytest.mark.parametrize("xi0,n", [(0.6, 1.91), (1.0, 1.91), (1.8, 1.91), (0.1, 5.0), (3.0, 1.0)])
def test_round_trip(orc, xi0, n):
    t = th(Xi0=xi0, n=n, H0=67.0)
    for z in np.linspace(1e-3, 9.9, 37):
        d = orc.dL_gw(z, t)
        z2 = orc.z_of_dL(d, t)
        assert abs(z2 - z) < 1e-12 * (1 + z)


def test_inversion_out_of_range(orc):
    t = th()
    assert orc.z_of_dL(orc.dL_gw(10.0, t) * 1.0001, t) is None
    assert orc.z_of_dL(-5.0, t) is None
    assert orc.z_of_dL(0.0, t) is None


@pytest.mark.parametrize("xi0,n,Om", [(0.6, 1.91, 0.3), (1.8, 2.7, 0.25), (0.1, 5.0, 0.3)])
def test_jacobian_matches_central_difference(orc, xi0, n, Om):
    t = th(Xi0=xi0, n=n, Om=Om)
    for z in (0.05, 0.4, 1.2, 3.0):
        h = 1e-5
        fd = (orc.dL_gw(z + h, t) - orc.dL_gw(z - h, t)) / (2 * h)
        assert orc.J(z, t) == pytest.approx(fd, rel=1e-8)


def test_volume_element(orc):
    # EdS: D_c = (2c/H0)(1 - (1+z)^(-1/2)), dD_c/dz = (c/H0)(1+z)^(-3/2)
    for z in (0.1, 0.9, 2.5):
        Dc = 2 * C / 70 * (1 - (1 + z) ** -0.5)
        dDc = C / 70 * (1 + z) ** -1.5
        assert orc.dVc_dz(z, 70.0, 1.0) == pytest.approx(4 * math.pi * Dc ** 2 * dDc, rel=1e-13)
        assert orc.Vc(z, 70.0, 1.0) == pytest.approx(4 * math.pi / 3 * Dc ** 3, rel=1e-13)
    # dV/dz is the derivative of V (flat LCDM)
    for z in (0.3, 1.1):
        h = 1e-5
        fd = (orc.Vc(z + h, 70.0, 0.3) - orc.Vc(z - h, 70.0, 0.3)) / (2 * h)
        assert orc.dVc_dz(z, 70.0, 0.3) == pytest.approx(fd, rel=1e-8)


def _golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    vals = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


def test_paper_event_rate(orc):
    """Sec. 3.3 prints dN/dt ~ 1.4e4 per year for the fiducial model; the
    oracle's psi and dV_c/dz must reproduce it to the two printed digits."""
    g = _golden("rate_sec3_3.txt")
    t = th(H0=g["H0"], Om=g["Om"], gamma=g["gamma"], kappa=g["kappa"], z_p=g["z_p"])
    R0 = g["R0_per_Gpc3_yr"] * 1e-9  # per Mpc^3
    psi0 = orc.psi(0.0, t)
    for norm in (1.0, psi0):  # psi is only defined up to a constant; either reading
        val = R0 * quad(lambda z: orc.psi(z, t) / norm / (1 + z) * orc.dVc_dz(z, g["H0"], g["Om"]),
                        0.0, g["z_upper"], epsrel=1e-10)[0]
        lead = float(f"{val:.{int(g['printed_sig_digits']) - 1}e}")
        assert lead == g["printed_rate_per_yr"], val


def test_monotonicity_guard(orc):
    assert orc.monotone(th()) == 1
    assert orc.monotone(th(Xi0=0.1, n=5.0)) == 1
    # a violently decreasing Xi makes d_L^gw fall with z somewhere
    assert orc.monotone(th(Xi0=0.01, n=40.0)) == 0


def test_theta_admissibility(orc):
    assert orc.check_theta(th()) == 0
    for bad in (dict(H0=-1.0), dict(Om=1.2), dict(Xi0=0.0), dict(sigma_g=0.0),
                dict(m_min=50.0, m_max=40.0), dict(z_p=-1.5), dict(H0=float("nan"))):
        assert orc.check_theta(th(**bad)) == 1
