"""The seeded synthetic inputs both sides of every parity test read: their CSR
layout, value ranges and determinism, the photometric redshift errors, the
16-bit galaxy storage rounding and the walker hyperpoints, on small
catalogs of the benchmark configurations' shapes."""
import numpy as np
import pytest

from synth import catalog as sc


@pytest.fixture(scope="module")
def spec_cat():
    return sc.config_catalog(2, n_events=12, n_pe=800, n_inj=40_000, gal_median=150)


@pytest.fixture(scope="module")
def photo_cat():
    return sc.config_catalog(3, n_events=6, n_pe=600, n_inj=20_000, gal_median=100)


def _check_layout(cat):
    ne = cat["n_events"]
    so, po, go = cat["sample_off"], cat["pix_off"], cat["gal_off"]
    assert so.dtype == np.int64 and po.dtype == np.int64 and go.dtype == np.int64
    assert so.size == ne + 1 and so[0] == 0 and np.all(np.diff(so) > 0) and so[-1] == cat["dL"].size
    assert po.size == ne + 1 and po[0] == 0 and np.all(np.diff(po) >= 1)
    assert po[-1] == cat["sky_S"].size and go.size == po[-1] + 1
    assert go[0] == 0 and np.all(np.diff(go) >= 0) and go[-1] == cat["gal_z"].size == cat["gal_sigma"].size
    assert cat["n_gal_total"] == cat["gal_z"].size
    for key in ("m1_det", "m2_det", "pix_of_sample"):
        assert cat[key].size == cat["dL"].size
    # pixel indices are local to the event and every pixel holds a sample
    for i in range(ne):
        pix = cat["pix_of_sample"][so[i]:so[i + 1]]
        npix = po[i + 1] - po[i]
        assert pix.min() == 0 and pix.max() == npix - 1
        assert np.unique(pix).size == npix
    n = cat["inj_dL"].size
    assert 0 < n <= cat["n_inj_total"]
    for key in ("inj_m1d", "inj_m2d", "inj_log_pi"):
        assert cat[key].size == n


def _check_values(cat):
    assert np.all(cat["dL"] > 0) and np.all(np.isfinite(cat["dL"]))
    assert np.all(cat["m2_det"] > 0) and np.all(cat["m1_det"] >= cat["m2_det"])
    assert np.all(cat["sky_S"] > 0)
    assert np.all(cat["gal_sigma"] > 0)
    assert np.all((cat["gal_z"] >= 0) & (cat["gal_z"] <= cat["z_max"]))
    assert np.all(cat["inj_m1d"] >= cat["inj_m2d"]) and np.all(np.isfinite(cat["inj_log_pi"]))
    # injections are drawn with d_L in [10, 2e4] Mpc
    assert np.all((cat["inj_dL"] >= 10.0) & (cat["inj_dL"] <= 2.0e4))


def test_spectroscopic_layout_and_values(spec_cat):
    _check_layout(spec_cat)
    _check_values(spec_cat)
    assert np.all(spec_cat["gal_sigma"] == 1e-3)
    assert spec_cat["pix_off"][-1] > spec_cat["n_events"]  # several pixels per event somewhere


def test_photometric_layout_and_values(photo_cat):
    _check_layout(photo_cat)
    _check_values(photo_cat)
    np.testing.assert_allclose(photo_cat["gal_sigma"], 0.05 * (1.0 + photo_cat["gal_z"]), rtol=1e-15)
    assert photo_cat["gal_storage"] == sc.GAL_BF16


def test_single_pixel_configuration():
    cat = sc.config_catalog(1)
    _check_layout(cat)
    assert np.all(np.diff(cat["pix_off"]) == 1)
    assert np.all(cat["pix_of_sample"] == 0)


def test_seeded_and_deterministic(spec_cat):
    again = sc.config_catalog(2, n_events=12, n_pe=800, n_inj=40_000, gal_median=150)
    for key, v in spec_cat.items():
        if isinstance(v, np.ndarray):
            assert np.array_equal(v, again[key]), key
    other = sc.config_catalog(2, variant=0, n_events=12, n_pe=800, n_inj=40_000, gal_median=150)
    assert not np.array_equal(other["dL"], spec_cat["dL"])  # another Xi0 variant, another seed


def test_injection_density_normalised():
    """ln pi_inj of the injection draw (d_L^3 uniform on [10, 2e4] Mpc, m1
    log-uniform on [3, 400], m2 uniform on [3, m1]) integrates to one over
    its support, by quadrature of the catalog's own formula."""
    from scipy import integrate
    dlo, dhi, mlo, mhi = 10.0, 2.0e4, 3.0, 400.0

    def lp(d, a1):
        return (np.log(3.0 * d ** 2 / (dhi ** 3 - dlo ** 3)) - np.log(a1 * np.log(mhi / mlo))
                - np.log(a1 - mlo))
    # the density does not depend on m2: its integral over m2 in [3, m1] is (m1 - 3) times it
    d_part, _ = integrate.quad(lambda d: np.exp(lp(d, 10.0) - lp(1000.0, 10.0)), dlo, dhi)
    m_part, _ = integrate.quad(lambda a1: (a1 - mlo) * np.exp(lp(1000.0, a1)), mlo, mhi, limit=200)
    assert d_part * m_part == pytest.approx(1.0, rel=1e-7)
    # and the catalog's values are that formula at its draws
    cat = sc.config_catalog(1)
    np.testing.assert_allclose(cat["inj_log_pi"], lp(cat["inj_dL"], cat["inj_m1d"]), rtol=0, atol=1e-12)


@pytest.mark.parametrize("storage,bits", [(sc.GAL_F16, 11), (sc.GAL_BF16, 8)])
def test_sixteen_bit_storage_rounding(photo_cat, storage, bits):
    q = sc.quantize_galaxies(photo_cat, storage)
    s, sq = photo_cat["gal_sigma"], q["gal_sigma"]
    assert np.all(np.abs(sq - s) <= s * 2.0 ** -bits * 1.0001)
    # z is stored as an offset from the pixel's smallest z: the error scales
    # with the offset, and the pixel's smallest z is exact (to float)
    go = photo_cat["gal_off"]
    for p in range(go.size - 1):
        a, b = int(go[p]), int(go[p + 1])
        if b <= a:
            continue
        z, zq = photo_cat["gal_z"][a:b], q["gal_z"][a:b]
        off = z - z.min()
        assert np.all(np.abs(zq - z) <= off * 2.0 ** -bits * 1.0001 + 2e-7 * (1 + z))
    again = sc.quantize_galaxies(q, storage)
    np.testing.assert_array_equal(again["gal_sigma"], sq)  # rounding is idempotent


def test_hyperpoints():
    th = sc.config_hyperpoints(2)
    assert th.shape == (16, 12)
    assert np.all(th[:, 1] == sc.FIDUCIAL["Om"])
    for k, name in enumerate(sc.PARAM_NAMES):
        lo, hi = sc.PRIOR_BOX[name]
        assert np.all((th[:, k] >= lo) & (th[:, k] <= hi)), name
    assert np.array_equal(th[0], [sc.FIDUCIAL[p] if p != "Xi0" else 1.0 for p in sc.PARAM_NAMES])
    th4 = sc.config_hyperpoints(4)
    assert th4.shape == (64, 12) and np.unique(th4[:, 1]).size == 64  # Om varies per point
    assert np.array_equal(sc.config_hyperpoints(4), th4)
