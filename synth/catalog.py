"""Seeded synthetic O5-like catalogs (inputs only; see package docstring).

Recipe (the shapes of Sec. 3 of the paper, made synthetic):

* parent population: redshift from psi(z) dV_c/dz / (1+z) on [0, 1.5]
  (Madau-Dickinson psi, Sec. 3.1), primary mass from the power law + Gaussian
  peak truncated to [m_min, m_max], secondary mass from m2^beta on
  [m_min, m1] (Sec. 3.1, Table 1 shapes with the fiducials below);
* detection: a deterministic S/N proxy
  rho = 200 (Mc_det / 30 Msun)^(5/6) (1 Gpc / d_L), detected when rho > 20;
* PE samples: observed = truth (1 + s eps0), samples = observed (1 + s eps_j)
  with s = 10 % for d_L and 5 % for the detector-frame masses (a stand-in for
  the Fisher-matrix PE of Sec. 3.2);
* sky: tangent-plane Gaussian localisation, equal-area square pixels sized so
  that an event covers about N_pix pixels (log-uniform integer in [1, 64]),
  sky factor S_ik = (N_ik / N_s) / Delta Omega_pix (histogram estimate);
* galaxies: lognormal counts per event (median 2e3, sigma_ln 1.19, clipped to
  [1, 5e4]), uniform in comoving volume over the event's redshift range,
  spread over its pixels in proportion to S_ik, host galaxy included;
  sigma_z = 1e-3 (spectroscopic) or 0.05 (1+z) (photometric, Sec. 4);
* injections: d_L ~ d_L^2 on [10, 2e4] Mpc, m1_det log-uniform on [3, 400],
  m2_det uniform on [3, m1_det], with the closed-form draw density stored as
  ln pi_inj; only detected injections are kept, N_inj counts all draws.

The distance-redshift relation used to *place* synthetic events is a private
fine-table integral below; it feeds only the data, never an expected value.
"""
import math

import numpy as np

C_KMS = 299792.458

PARAM_NAMES = ("H0", "Om", "Xi0", "n", "alpha", "mu_g", "sigma_g",
               "m_min", "m_max", "gamma", "kappa", "z_p")

FIDUCIAL = dict(H0=70.0, Om=0.3, Xi0=1.0, n=1.91, alpha=3.4, mu_g=34.0,
                sigma_g=3.6, m_min=5.0, m_max=100.0, gamma=2.7, kappa=3.0,
                z_p=2.0)
LAMBDA_G = 0.039
BETA = 1.1

# Walker box: Table 1 priors where the paper gives them; Om and m_min are
# fixed or absent there, so a plausible range is used for the walker ball.
PRIOR_BOX = dict(H0=(10.0, 200.0), Om=(0.1, 0.5), Xi0=(0.1, 10.0),
                 n=(1.0, 5.0), alpha=(1.5, 12.0), mu_g=(2.0, 50.0),
                 sigma_g=(0.4, 10.0), m_min=(2.0, 10.0), m_max=(50.0, 200.0),
                 gamma=(0.0, 12.0), kappa=(0.0, 6.0), z_p=(0.0, 4.0))

SEED_BASE = 2504020340

KDE_SINGLE_1D = 0
KDE_MANY_1D = 1
KDE_3D = 2  # the "3D" kernel over (z, sky), a cross-check variant
GAL_F32 = 0
GAL_F16 = 1
GAL_BF16 = 2


class _TruthDistance:
    """Private d_L^GW(z) on a fine trapezoid table, used to place events."""

    def __init__(self, H0, Om, Xi0, n, zmax=12.0, npts=240001):
        z = np.linspace(0.0, zmax, npts)
        inv_e = 1.0 / np.sqrt(Om * (1.0 + z) ** 3 + 1.0 - Om)
        seg = 0.5 * (inv_e[1:] + inv_e[:-1]) * np.diff(z)
        dc = np.concatenate([[0.0], np.cumsum(seg)]) * (C_KMS / H0)
        xi = Xi0 + (1.0 - Xi0) / (1.0 + z) ** n
        self.z = z
        self.dc = dc
        self.dgw = (1.0 + z) * dc * xi
        self.inv_e = inv_e

    def dgw_of_z(self, zz):
        return np.interp(zz, self.z, self.dgw)

    def z_of_dgw(self, d):
        return np.interp(d, self.dgw, self.z)

    def z_of_vc(self, vc):
        return np.interp(vc, self.dc ** 3, self.z)

    def vc_of_z(self, zz):
        return np.interp(zz, self.z, self.dc) ** 3


def _inverse_cdf_sampler(x, pdf):
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(x))])
    cdf /= cdf[-1]
    return lambda u: np.interp(u, cdf, x)


def _draw_parent(rng, n, truth, fid, zmax=1.5):
    zg = np.linspace(0.0, zmax, 20001)
    ibase = np.interp(zg, truth.z, truth.dc) ** 2 * np.interp(zg, truth.z, truth.inv_e)
    psi = (1.0 + zg) ** fid["gamma"] / (1.0 + ((1.0 + zg) / (1.0 + fid["z_p"])) ** (fid["gamma"] + fid["kappa"]))
    zs = _inverse_cdf_sampler(zg, psi * ibase / (1.0 + zg))(rng.random(n))

    mg = np.linspace(fid["m_min"], fid["m_max"], 40001)
    a = fid["alpha"]
    pl = mg ** (-a)
    pl /= np.trapezoid(pl, mg)
    g = np.exp(-0.5 * ((mg - fid["mu_g"]) / fid["sigma_g"]) ** 2)
    g /= np.trapezoid(g, mg)
    m1 = _inverse_cdf_sampler(mg, (1 - LAMBDA_G) * pl + LAMBDA_G * g)(rng.random(n))
    b1 = BETA + 1.0
    lo = fid["m_min"] ** b1
    m2 = (lo + rng.random(n) * (m1 ** b1 - lo)) ** (1.0 / b1)
    return zs, m1, m2


def _snr(m1d, m2d, dl):
    mc = (m1d * m2d) ** 0.6 / (m1d + m2d) ** 0.2
    return 200.0 * (mc / 30.0) ** (5.0 / 6.0) * (1000.0 / dl)


def _positive_scatter(rng, center, rel, size):
    out = center * (1.0 + rel * rng.standard_normal(size))
    bad = out <= 0
    while np.any(bad):
        out[bad] = center * (1.0 + rel * rng.standard_normal(int(bad.sum())))
        bad = out <= 0
    return out


def make_catalog(*, n_events, n_pe, n_inj, n_z, Xi0, photo=False,
                 gal_median=2000.0, gal_factor=1.0, gal_fixed=None,
                 n_pix_max=64, single_pixel=False, z_max=1.5, seed=0,
                 kde_mode=KDE_MANY_1D, gal_storage=GAL_F32, sigma_spec=1e-3,
                 n_parent_batch=5000):
    """Build one synthetic catalog as a dict of numpy arrays.

    Layout (all CSR offsets int64, values float64):
      sample_off[n_events+1]; dL, m1_det, m2_det, ra, dec per sample;
      pix_of_sample (int32, index within the event's pixel list);
      pix_off[n_events+1] into the flat pixel list; sky_S per pixel [sr^-1];
      gal_off[n_pix_total+1]; gal_z, gal_sigma per galaxy;
      inj_dL, inj_m1d, inj_m2d, inj_log_pi per detected injection.
    """
    rng = np.random.default_rng(seed)
    fid = dict(FIDUCIAL)
    fid["Xi0"] = Xi0
    truth = _TruthDistance(fid["H0"], fid["Om"], Xi0, fid["n"])

    # ---- detected events: first n_events detections in seed order
    ev_z, ev_m1, ev_m2 = [], [], []
    got = 0
    while got < n_events:
        zs, m1, m2 = _draw_parent(rng, n_parent_batch, truth, fid, z_max)
        dl = truth.dgw_of_z(zs)
        det = _snr(m1 * (1 + zs), m2 * (1 + zs), dl) > 20.0
        idx = np.nonzero(det)[0][: n_events - got]
        ev_z.append(zs[idx]); ev_m1.append(m1[idx]); ev_m2.append(m2[idx])
        got += idx.size
    ev_z = np.concatenate(ev_z); ev_m1 = np.concatenate(ev_m1); ev_m2 = np.concatenate(ev_m2)
    ev_dl = truth.dgw_of_z(ev_z)

    sample_off = np.arange(n_events + 1, dtype=np.int64) * n_pe
    dL = np.empty(n_events * n_pe); m1d = np.empty_like(dL); m2d = np.empty_like(dL)
    ra = np.empty_like(dL); dec = np.empty_like(dL)
    pix_of_sample = np.empty(n_events * n_pe, dtype=np.int32)
    pix_off = [0]
    sky_S = []
    sky_xy = np.empty((n_events * n_pe, 2))  # flat local sky chart per event [rad]
    pix_xy = []                               # pixel centres in the same chart
    gal_off = [0]
    gal_z = []
    gal_sigma = []
    sig_sky = 0.01
    zgrid_fine = truth.z
    for i in range(n_events):
        sl = slice(i * n_pe, (i + 1) * n_pe)
        od = _positive_scatter(rng, ev_dl[i], 0.10, 1)[0]
        om1 = _positive_scatter(rng, ev_m1[i] * (1 + ev_z[i]), 0.05, 1)[0]
        om2 = _positive_scatter(rng, ev_m2[i] * (1 + ev_z[i]), 0.05, 1)[0]
        d = _positive_scatter(rng, od, 0.10, n_pe)
        a1 = _positive_scatter(rng, om1, 0.05, n_pe)
        a2 = _positive_scatter(rng, om2, 0.05, n_pe)
        sw = a2 > a1
        a1[sw], a2[sw] = a2[sw], a1[sw]
        dL[sl] = d; m1d[sl] = a1; m2d[sl] = a2

        # sky localisation in a tangent plane about the observed centre
        ra0 = rng.uniform(0, 2 * np.pi)
        dec0 = np.arcsin(rng.uniform(-1, 1))
        true_off = -sig_sky * rng.standard_normal(2)
        x = sig_sky * rng.standard_normal(n_pe)
        y = sig_sky * rng.standard_normal(n_pe)
        ra[sl] = ra0 + x / max(np.cos(dec0), 1e-3)
        dec[sl] = dec0 + y
        if single_pixel:
            side = 40.0 * sig_sky
            pix = np.zeros(n_pe, dtype=np.int64)
            keys = np.array([0])
            counts = np.array([n_pe])
            host_key = 0
        else:
            target = int(np.clip(np.floor(np.exp(rng.uniform(0, np.log(n_pix_max + 1)))), 1, n_pix_max))
            side = sig_sky * math.sqrt(40.0 / target)
            while True:  # grow the pixels until the occupied set is within n_pix_max
                ix = np.floor(x / side + 0.5).astype(np.int64)
                iy = np.floor(y / side + 0.5).astype(np.int64)
                code = (ix + 4096) * 8192 + (iy + 4096)
                keys, pix, counts = np.unique(code, return_inverse=True, return_counts=True)
                if keys.size <= n_pix_max:
                    break
                side *= 1.1
            hx = int(np.floor(true_off[0] / side + 0.5)); hy = int(np.floor(true_off[1] / side + 0.5))
            hcode = (hx + 4096) * 8192 + (hy + 4096)
            hit = np.nonzero(keys == hcode)[0]
            host_key = int(hit[0]) if hit.size else int(np.argmax(counts))
        npix = keys.size
        pix_of_sample[sl] = pix.astype(np.int32)
        sky_xy[sl, 0], sky_xy[sl, 1] = x, y
        if single_pixel:
            pix_xy.append((0.0, 0.0))
        else:
            pix_xy.extend(zip(((keys // 8192) - 4096) * side, ((keys % 8192) - 4096) * side))
        S = counts / (n_pe * side * side)
        sky_S.extend(S.tolist())
        pix_off.append(pix_off[-1] + npix)

        # galaxies, uniform in comoving volume over the event's z range
        if gal_fixed is not None:
            ng = int(gal_fixed)
        else:
            ng = int(np.clip(round(gal_median * np.exp(1.19 * rng.standard_normal())), 1, 50000))
            ng = max(1, int(round(ng * gal_factor)))
        zs_ev = np.interp(d, truth.dgw, zgrid_fine)
        lo, hi = np.quantile(zs_ev, [0.0005, 0.9995])
        mid, half = 0.5 * (lo + hi), 0.75 * (hi - lo)
        zlo, zhi = max(0.0, mid - half), min(z_max, mid + half)
        if zhi <= zlo:
            zlo, zhi = max(0.0, z_max - 0.05), z_max
        v0, v1 = truth.vc_of_z(zlo), truth.vc_of_z(zhi)
        gz = truth.z_of_vc(v0 + rng.random(ng) * (v1 - v0))
        gp = rng.choice(npix, size=ng, p=counts / counts.sum())
        # host galaxy: the true redshift, in the pixel holding the true position
        gz = np.concatenate([gz, [ev_z[i]]])
        gp = np.concatenate([gp, [host_key]])
        order = np.argsort(gp, kind="stable")
        gz, gp = gz[order], gp[order]
        per_pix = np.bincount(gp, minlength=npix)
        for k in range(npix):
            gal_off.append(gal_off[-1] + int(per_pix[k]))
        gal_z.extend(gz.tolist())
        sig = 0.05 * (1.0 + gz) if photo else np.full(gz.shape, sigma_spec)
        gal_sigma.extend(sig.tolist())

    # ---- injections (detected only)
    inj = {"dL": [], "m1d": [], "m2d": [], "lp": []}
    dlo, dhi, mlo, mhi = 10.0, 2.0e4, 3.0, 400.0
    left = int(n_inj)
    while left > 0:
        k = min(left, 1_000_000)
        di = (dlo ** 3 + rng.random(k) * (dhi ** 3 - dlo ** 3)) ** (1.0 / 3.0)
        a1 = mlo * np.exp(rng.random(k) * np.log(mhi / mlo))
        a2 = mlo + rng.random(k) * (a1 - mlo)
        det = _snr(a1, a2, di) > 20.0
        lp = (np.log(3.0 * di ** 2 / (dhi ** 3 - dlo ** 3))
              - np.log(a1 * np.log(mhi / mlo)) - np.log(a1 - mlo))
        inj["dL"].append(di[det]); inj["m1d"].append(a1[det]); inj["m2d"].append(a2[det]); inj["lp"].append(lp[det])
        left -= k

    gal_z = np.asarray(gal_z, dtype=np.float64)
    return dict(
        n_events=int(n_events),
        sample_off=sample_off,
        dL=dL, m1_det=m1d, m2_det=m2d, ra=ra, dec=dec,
        pix_of_sample=pix_of_sample,
        sky_xy=sky_xy, pix_xy=np.asarray(pix_xy, dtype=np.float64).reshape(-1, 2),
        pix_off=np.asarray(pix_off, dtype=np.int64),
        sky_S=np.asarray(sky_S, dtype=np.float64),
        gal_off=np.asarray(gal_off, dtype=np.int64),
        gal_z=gal_z,
        gal_sigma=np.asarray(gal_sigma, dtype=np.float64),
        n_gal_total=float(gal_z.size),
        z_max=float(z_max), n_z=int(n_z),
        n_inj_total=int(n_inj),
        inj_dL=np.concatenate(inj["dL"]), inj_m1d=np.concatenate(inj["m1d"]),
        inj_m2d=np.concatenate(inj["m2d"]), inj_log_pi=np.concatenate(inj["lp"]),
        lambda_g=LAMBDA_G, beta=BETA,
        kde_mode=int(kde_mode), gal_storage=int(gal_storage),
        truth=dict(z=ev_z, m1=ev_m1, m2=ev_m2, dL=ev_dl, Xi0=Xi0),
    )


def add_completeness(cat, *, seed, f_R=0.75, width=0.05, zc_range=(0.3, 1.0)):
    """An incomplete-catalog version of `cat` (Eqs. p-gal, p-miss, f-R): each
    pixel gets its solid angle (side^2 of the tangent-plane square, recovered
    from its sample count and sky factor: S_k = (N_k / N_s) / Delta Omega_k)
    and a completeness that falls from 1 to 0 around a pixel redshift z_c
    (logistic of width `width`, z_c uniform in zc_range) on the grid; f_R is
    the catalog's full-sky completeness fraction, an input."""
    rng = np.random.default_rng(seed)
    out = dict(cat)
    so, po = cat["sample_off"], cat["pix_off"]
    area = np.empty(cat["sky_S"].size)
    for e in range(cat["n_events"]):
        ns = int(so[e + 1] - so[e])
        cnt = np.bincount(cat["pix_of_sample"][so[e]:so[e + 1]], minlength=int(po[e + 1] - po[e]))
        area[po[e]:po[e + 1]] = cnt / (ns * cat["sky_S"][po[e]:po[e + 1]])
    za = cat["z_max"] * np.arange(cat["n_z"]) / (cat["n_z"] - 1)
    zc = rng.uniform(zc_range[0], zc_range[1], area.size)
    out["pix_area"] = area
    out["completeness"] = np.ascontiguousarray(1.0 / (1.0 + np.exp((za[None, :] - zc[:, None]) / width)))
    out["f_R"] = float(f_R)
    return out


def make_hyperpoints(n, *, seed, Xi0=1.0, vary_Om=False, width=0.01):
    """Walker hyperpoints: a Gaussian ball (width x prior range) about the
    fiducial, clipped to the walker box; Om held at 0.3 unless vary_Om."""
    rng = np.random.default_rng(seed)
    fid = dict(FIDUCIAL)
    fid["Xi0"] = Xi0
    th = np.empty((n, len(PARAM_NAMES)))
    for k, name in enumerate(PARAM_NAMES):
        lo, hi = PRIOR_BOX[name]
        th[:, k] = np.clip(fid[name] + width * (hi - lo) * rng.standard_normal(n), lo, hi)
    if not vary_Om:
        th[:, 1] = fid["Om"]
    if n > 0:
        th[0] = [fid[p] for p in PARAM_NAMES] if not vary_Om else th[0]
    return th


# Configurations (sizes of the five benchmark configurations).
_CONFIGS = {
    1: dict(n_events=10, n_pe=1000, n_inj=10_000, n_z=256, Xi0=1.0, single_pixel=True,
            gal_fixed=200, n_points=1),
    2: dict(n_events=300, n_pe=5000, n_inj=2_000_000, n_z=1000, Xi0=1.0, n_points=16),
    3: dict(n_events=300, n_pe=5000, n_inj=2_000_000, n_z=1000, Xi0=1.0, photo=True,
            gal_factor=3.0, gal_storage=GAL_BF16, n_points=512),
    4: dict(n_events=5000, n_pe=4000, n_inj=5_000_000, n_z=1000, Xi0=1.0, n_points=64,
            vary_Om=True),
}
XI0_VARIANTS = (0.6, 1.0, 1.8)


def config_catalog(config, variant=1, **override):
    """Catalog for a numbered configuration; `variant` picks Xi0 from
    (0.6, 1, 1.8) for configurations 2 and 3; keyword overrides shrink sizes."""
    spec = dict(_CONFIGS[config])
    spec.pop("n_points")
    vary_om = spec.pop("vary_Om", False)
    del vary_om
    if config in (2, 3):
        spec["Xi0"] = XI0_VARIANTS[variant]
    spec.update(override)
    seed = SEED_BASE + 10 * config + variant
    return make_catalog(seed=seed, **spec)


def config_hyperpoints(config, variant=1, n=None):
    spec = _CONFIGS[config]
    n = spec["n_points"] if n is None else n
    xi0 = XI0_VARIANTS[variant] if config in (2, 3) else spec["Xi0"]
    return make_hyperpoints(n, seed=SEED_BASE + 10 * config + variant + 5,
                            Xi0=xi0, vary_Om=spec.get("vary_Om", False))


def quantize_galaxies(cat, storage):
    """Return a copy of `cat` whose galaxy z and sigma are rounded the way the
    device stores them: z as a 16-bit offset from the pixel's smallest z,
    sigma as a 16-bit float (FP16 or BF16).  Feeding the copy to the oracle
    isolates kernel error from storage rounding."""
    import torch  # only for the bf16 rounding primitive

    out = dict(cat)
    if storage == GAL_F32:
        out["gal_z"] = cat["gal_z"].astype(np.float32).astype(np.float64)
        out["gal_sigma"] = cat["gal_sigma"].astype(np.float32).astype(np.float64)
        return out
    dt = torch.float16 if storage == GAL_F16 else torch.bfloat16
    gz = cat["gal_z"].copy()
    gs = cat["gal_sigma"].copy()
    off = cat["gal_off"]
    for p in range(off.size - 1):
        a, b = int(off[p]), int(off[p + 1])
        if b <= a:
            continue
        ref = np.float32(gz[a:b].min())  # the device keeps the pixel's smallest z as reference
        d = torch.tensor((gz[a:b].astype(np.float32) - ref), dtype=torch.float32).to(dt).to(torch.float32).numpy()
        gz[a:b] = (np.float32(ref) + d.astype(np.float32)).astype(np.float64)
        gs[a:b] = torch.tensor(gs[a:b].astype(np.float32)).to(dt).to(torch.float32).numpy().astype(np.float64)
    out["gal_z"] = gz
    out["gal_sigma"] = gs
    return out
