"""Edge-free copies of catalogs for derivative checks (test helper).

The likelihood's derivative with respect to a parameter is the
almost-everywhere one: PE samples or injections whose source-frame masses
cross m_min / m_max, or injections crossing z_max, under a finite-difference
step make jumps that no derivative contains.  These copies drop every sample
and injection within a relative margin of those edges at the test point, so
that central differences measure the derivative itself.
"""
import numpy as np

C_KMS = 299792.458


def _z_of_dgw(d, th, zmax=12.0, npts=400001):
    """Generous numerical inverse of Eq. dL-mg (trapezoid table), used only to
    decide which samples sit near an edge."""
    H0, Om, Xi0, n = th[:4]
    z = np.linspace(0.0, zmax, npts)
    inv_e = 1.0 / np.sqrt(Om * (1.0 + z) ** 3 + 1.0 - Om)
    dc = np.concatenate([[0.0], np.cumsum(0.5 * (inv_e[1:] + inv_e[:-1]) * np.diff(z))]) * C_KMS / H0
    dgw = (1.0 + z) * dc * (Xi0 + (1.0 - Xi0) / (1.0 + z) ** n)
    return np.interp(d, dgw, z)


def edge_free(cat, th, margin=0.01):
    """Copy of `cat` without the samples / injections near a mass or z_max edge."""
    mmin, mmax = th[7], th[8]

    def near(m1d, m2d, dL):
        a = 1.0 + _z_of_dgw(dL, th)
        m1, m2 = m1d / a, m2d / a
        bad = np.zeros(m1.shape, bool)
        for m in (m1, m2):
            for e in (mmin, mmax):
                bad |= np.abs(m / e - 1.0) < margin
        return bad, a - 1.0

    out = dict(cat)
    bad, _ = near(cat["m1_det"], cat["m2_det"], cat["dL"])
    so = cat["sample_off"]
    keep = ~bad
    # keep at least two samples per event
    for e in range(cat["n_events"]):
        assert keep[so[e]:so[e + 1]].sum() >= 2
    counts = np.array([keep[so[e]:so[e + 1]].sum() for e in range(cat["n_events"])])
    out["sample_off"] = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    for k in ("dL", "m1_det", "m2_det", "pix_of_sample"):
        out[k] = np.ascontiguousarray(cat[k][keep])
    ibad, zi = near(cat["inj_m1d"], cat["inj_m2d"], cat["inj_dL"])
    ibad |= np.abs(zi / cat["z_max"] - 1.0) < margin
    for k in ("inj_dL", "inj_m1d", "inj_m2d", "inj_log_pi"):
        out[k] = np.ascontiguousarray(cat[k][~ibad])
    return out
