"""Galaxy profiles on the tensor cores (the Om-varying photometric galaxy term).

For a catalog whose galaxies are all photometric (sigma_z = 0.05(1+z), each at
least 0.02 and 8 grid steps wide), the mixed path builds the galaxy term of
Eq. p-cat for up to 256 Om values per pass as two tcgen05 contractions: the
Om-independent Gaussians N(z_a; z_g, sigma_g) in FP16 against the
Om-dependent columns (w_a dV_c/dz and 1/Z_g) split into two FP16 terms, with
FP32 accumulation.  Checked here:

* the catalog reports the tensor-core path; CHIMERA_PROFILE_FP32=1 at load
  keeps the FP32 CUDA-core kernels for the same catalog;
* per event, ln I_i for hyperpoints with distinct Om against the FP32 kernels
  (|Delta ln I_i| <= 1e-4, the mixed path's per-event tolerance; the FP16
  rounding of the Gaussians dominates, ~1.5e-5 on average), and per point ln L
  against the FP64 oracle on the BF16-rounded galaxies (<= 1e-3, the mixed
  path's per-catalog tolerance);
* a profile is a function of its Om alone: a point's ln L computed alone
  equals, bit for bit, the same point's ln L in a batch of 300 distinct Om
  values (two passes of 256 and 44 columns);
* at full size (300 events, x3 galaxies, BF16), 64 distinct Om values against
  the FP32 kernels.
"""
import math
import os

import numpy as np
import pytest

from synth import catalog as sc

pytestmark = pytest.mark.gpu

TOL_EV = 1e-4


@pytest.fixture(scope="module")
def chim():
    from paper_2504_02034_b300 import build
    build.build()
    import paper_2504_02034_b300 as pkg
    return pkg


@pytest.fixture(scope="module")
def ctx(chim):
    c = chim.Context(0)
    yield c
    c.close()


def _load_fp32(ctx, cat):
    os.environ["CHIMERA_PROFILE_FP32"] = "1"
    try:
        return ctx.load(cat)
    finally:
        del os.environ["CHIMERA_PROFILE_FP32"]


def _points(n, lo=0.26, hi=0.34, seed=7):
    th = sc.config_hyperpoints(3, n=n)
    th[:, 1] = np.linspace(lo, hi, n)
    np.random.default_rng(seed).shuffle(th[:, 1])
    return th


def _compare_events(tag, a, b):
    fa, fb = np.isfinite(a), np.isfinite(b)
    np.testing.assert_array_equal(fa, fb)
    sd = a[fa] - b[fa]
    d = np.abs(sd)
    print("MEASURED %s max|dlnI|=%.3e mean|dlnI|=%.3e mean(dlnI)=%.3e" % (tag, d.max(), d.mean(), sd.mean()))
    assert d.max() <= TOL_EV, (tag, d.max())


def test_small_photometric_catalog(chim, ctx, orc):
    cat = sc.config_catalog(3, n_events=12, n_pe=1000, n_inj=20000)
    th = _points(24)
    cid = ctx.load(cat)
    fid = _load_fp32(ctx, cat)
    try:
        assert ctx.info(cid)["profile_path"] == chim.PROFILE_TENSOR_CORES
        assert ctx.info(fid)["profile_path"] == chim.PROFILE_CUDA_CORES
        t_tc = ctx.terms(cid, th, chim.MIXED)
        t_fp = ctx.terms(fid, th, chim.MIXED)
        lnL, _, st = ctx.loglike(cid, th, chim.MIXED)
    finally:
        ctx.unload(cid)
        ctx.unload(fid)
    _compare_events("tc_vs_fp32_small", t_tc["lnI"], t_fp["lnI"])
    oc = orc.Catalog(sc.quantize_galaxies(cat, sc.GAL_BF16))
    for h in (0, 11, 23):
        ref = oc.loglike(th[h])
        assert st[h] == ref["status"]
        if math.isfinite(ref["lnL"]):
            d = lnL[h] - ref["lnL"]
            print("MEASURED tc_small[h=%d] dlnL vs oracle %.3e" % (h, d))
            assert abs(d) <= 1e-3, (h, d)
        else:
            assert lnL[h] == -math.inf


def test_profile_depends_on_its_om_alone(chim, ctx):
    cat = sc.config_catalog(3, n_events=8, n_pe=800, n_inj=10000)
    th = _points(300, lo=0.2, hi=0.4, seed=11)
    cid = ctx.load(cat)
    try:
        lnL_batch, _, _ = ctx.loglike(cid, th, chim.MIXED)
    finally:
        ctx.unload(cid)
    for h in (0, 150, 255, 256, 299):
        cid = ctx.load(cat)  # a fresh profile cache
        try:
            lnL1, _, _ = ctx.loglike(cid, th[h:h + 1], chim.MIXED)
        finally:
            ctx.unload(cid)
        assert lnL1[0] == lnL_batch[h] or (math.isinf(lnL1[0]) and math.isinf(lnL_batch[h])), \
            (h, lnL1[0], lnL_batch[h])


def _galaxy_ms(chim, ctx, cid, th):
    """ln L of points with new Om values; the profile stage's time (ms)."""
    chim.chimera_set_trace(ctx.h, True)
    try:
        ctx.loglike(cid, th, chim.MIXED)
        return chim.chimera_stage_ms(ctx.h)["galaxy"]
    finally:
        chim.chimera_set_trace(ctx.h, False)


def test_full_photometric_catalog_64_om(chim, ctx):
    cat = sc.config_catalog(3)
    th = _points(64)
    cid = ctx.load(cat)
    try:
        assert ctx.info(cid)["profile_path"] == chim.PROFILE_TENSOR_CORES
        t_tc = ctx.terms(cid, th, chim.MIXED)
        ms_tc = _galaxy_ms(chim, ctx, cid, _points(128, lo=0.2, hi=0.25))
    finally:
        ctx.unload(cid)
    fid = _load_fp32(ctx, cat)
    try:
        t_fp = ctx.terms(fid, th, chim.MIXED)
        ms_fp = _galaxy_ms(chim, ctx, fid, _points(128, lo=0.2, hi=0.25))
    finally:
        ctx.unload(fid)
    print("MEASURED profiles of 128 new Om, full photometric catalog: tensor cores %.2f ms, FP32 kernels %.2f ms"
          % (ms_tc, ms_fp))
    _compare_events("tc_vs_fp32_full", t_tc["lnI"], t_fp["lnI"])
    ok = np.all(np.isfinite(t_tc["lnI"]), axis=1)
    d = np.abs(t_tc["lnI"][ok].sum(axis=1) - t_fp["lnI"][ok].sum(axis=1))
    print("MEASURED tc_vs_fp32_full max|d sum lnI|=%.3e" % d.max())
    assert d.max() <= 1e-3


@pytest.mark.parametrize("kde_mode,storage", [(sc.KDE_SINGLE_1D, sc.GAL_F16), (sc.KDE_MANY_1D, sc.GAL_F32)],
                         ids=["single1d-f16", "many1d-f32"])
def test_other_storage_and_kde_modes(chim, ctx, kde_mode, storage):
    """The tensor-core profiles under the single-1D KDE (the sky-summed
    profile is formed after them) and with F16 / F32 galaxy storage, against
    the FP32 kernels of the same catalog; one pixel of an event emptied of
    its galaxies keeps a zero profile."""
    cat = sc.config_catalog(3, n_events=10, n_pe=800, n_inj=10000, kde_mode=kde_mode, gal_storage=storage)
    # empty the galaxies of one pixel (its profile rows must come out zero)
    go = cat["gal_off"].copy()
    p = int(np.argmax(np.diff(go)))
    keep = np.ones(go[-1], bool)
    keep[go[p]:go[p + 1]] = False
    cat = dict(cat)
    cat["gal_z"], cat["gal_sigma"] = cat["gal_z"][keep], cat["gal_sigma"][keep]
    cat["gal_off"] = np.concatenate([[0], np.cumsum(np.diff(go) * (np.arange(len(go) - 1) != p))]).astype(np.int64)
    th = _points(20, seed=5)
    cid = ctx.load(cat)
    fid = _load_fp32(ctx, cat)
    try:
        assert ctx.info(cid)["profile_path"] == chim.PROFILE_TENSOR_CORES
        t_tc = ctx.terms(cid, th, chim.MIXED)
        t_fp = ctx.terms(fid, th, chim.MIXED)
    finally:
        ctx.unload(cid)
        ctx.unload(fid)
    _compare_events("tc_vs_fp32_%d_%d" % (kde_mode, storage), t_tc["lnI"], t_fp["lnI"])


def test_odd_grid_and_extreme_om(chim, ctx):
    """A grid of 777 points (not a multiple of 4: scalar profile stores, a
    partial last 256-point tile, K chunks past the grid's end) and Om values
    at the ends of the admissible range (dV_c/dz far from the fiducial's),
    against the FP32 kernels."""
    cat = sc.config_catalog(3, n_events=8, n_pe=700, n_inj=8000, n_z=777)
    th = sc.config_hyperpoints(3, n=6)
    th[:, 1] = [0.02, 0.1, 0.3, 0.5, 0.8, 0.98]
    cid = ctx.load(cat)
    fid = _load_fp32(ctx, cat)
    try:
        assert ctx.info(cid)["profile_path"] == chim.PROFILE_TENSOR_CORES
        t_tc = ctx.terms(cid, th, chim.MIXED)
        t_fp = ctx.terms(fid, th, chim.MIXED)
    finally:
        ctx.unload(cid)
        ctx.unload(fid)
    _compare_events("tc_vs_fp32_nz777_om_ends", t_tc["lnI"], t_fp["lnI"])
