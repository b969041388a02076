"""Small hand-built catalogs for the oracle pins (test helpers only)."""
import math

import numpy as np

C = 299792.458
FID = np.array([70.0, 0.3, 1.0, 1.91, 3.4, 34.0, 3.6, 5.0, 100.0, 2.7, 3.0, 2.0])


def theta(**kw):
    names = ["H0", "Om", "Xi0", "n", "alpha", "mu_g", "sigma_g", "m_min", "m_max", "gamma", "kappa", "z_p"]
    t = FID.copy()
    for k, v in kw.items():
        t[names.index(k)] = v
    return t


def build(events, *, n_z, z_max=1.5, inj=None, n_inj_total=None, lambda_g=0.039, beta=1.1,
          kde_mode=1, n_gal_total=None):
    """events: list of dict(dL, m1d, m2d, pix (per-sample pixel index),
    S (per-pixel), gal_z (list per pixel), gal_sigma (list per pixel))."""
    so = [0]
    dL, m1, m2, pix = [], [], [], []
    pix_off = [0]
    S = []
    gal_off = [0]
    gz, gs = [], []
    for e in events:
        n = len(e["dL"])
        so.append(so[-1] + n)
        dL += list(e["dL"]); m1 += list(e["m1d"]); m2 += list(e["m2d"]); pix += list(e["pix"])
        npix = len(e["S"])
        pix_off.append(pix_off[-1] + npix)
        S += list(e["S"])
        for k in range(npix):
            gal_off.append(gal_off[-1] + len(e["gal_z"][k]))
            gz += list(e["gal_z"][k]); gs += list(e["gal_sigma"][k])
    if inj is None:
        inj = dict(dL=[1000.0], m1d=[30.0], m2d=[25.0], log_pi=[0.0])
    ntot = len(inj["dL"]) if n_inj_total is None else n_inj_total
    return dict(
        n_events=len(events), sample_off=np.array(so, np.int64),
        dL=np.array(dL), m1_det=np.array(m1), m2_det=np.array(m2),
        pix_of_sample=np.array(pix, np.int32), pix_off=np.array(pix_off, np.int64),
        sky_S=np.array(S), gal_off=np.array(gal_off, np.int64),
        gal_z=np.array(gz), gal_sigma=np.array(gs),
        n_gal_total=float(len(gz) if n_gal_total is None else n_gal_total),
        z_max=z_max, n_z=n_z, n_inj_total=int(ntot),
        inj_dL=np.array(inj["dL"], float), inj_m1d=np.array(inj["m1d"], float),
        inj_m2d=np.array(inj["m2d"], float), inj_log_pi=np.array(inj["log_pi"], float),
        lambda_g=lambda_g, beta=beta, kde_mode=kde_mode, gal_storage=0,
    )


# ---- Einstein-de Sitter closed forms (Om = 1) used by the brute-force pins
def eds_dc(z, H0):
    s = math.sqrt(1 + z)
    return 2 * C / H0 * z / (s * (1 + s))


def eds_ddc(z, H0):
    return C / H0 * (1 + z) ** -1.5


def eds_xi(z, xi0, n):
    return xi0 + (1 - xi0) * (1 + z) ** -n


def eds_dgw(z, t):
    return (1 + z) * eds_dc(z, t[0]) * eds_xi(z, t[2], t[3])


def eds_J(z, t):
    H0, xi0, n = t[0], t[2], t[3]
    dc, ddc = eds_dc(z, H0), eds_ddc(z, H0)
    xi = eds_xi(z, xi0, n)
    dxi = -n * (1 - xi0) * (1 + z) ** (-n - 1)
    return dc * xi + (1 + z) * ddc * xi + (1 + z) * dc * dxi


def eds_dvdz(z, H0):
    return 4 * math.pi * eds_dc(z, H0) ** 2 * eds_ddc(z, H0)


def eds_vc(z, H0):
    return 4 * math.pi / 3 * eds_dc(z, H0) ** 3
