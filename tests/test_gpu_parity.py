"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded synthetic catalogs.

Tolerances (the accuracy contract of the two paths):
  FP64 path : |Delta ln L| <= 1e-6 * N_events, per event |Delta ln I_i| <= 1e-7
  mixed path: |Delta ln L| <= 1e-3 absolute per catalog,
              per event |Delta ln I_i| <= 1e-4, |Delta ln xi| <= 3e-6
"""
import math

import numpy as np
import pytest

import _catalogs as tc

pytestmark = pytest.mark.gpu

FP64_EV = 1e-7
MIX_EV = 1e-4


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


def _compare(chim, ctx, orc, cat, thetas, precisions=(0, 1), nthreads=0):
    oc = orc.Catalog(cat)
    cid = ctx.load(cat)
    try:
        ref = [oc.loglike(t, nthreads=nthreads) for t in thetas]
        for prec in precisions:
            lnL, neff, st = ctx.loglike(cid, thetas, prec)
            terms = ctx.terms(cid, thetas, prec)
            ne = cat["n_events"]
            for h, r in enumerate(ref):
                assert st[h] == r["status"], (prec, h, st[h], r["status"])
                if not math.isfinite(r["lnL"]):
                    assert lnL[h] == -math.inf
                    continue
                tol = 1e-6 * ne if prec == 0 else 1e-3
                assert abs(lnL[h] - r["lnL"]) <= tol, (prec, h, lnL[h] - r["lnL"])
                etol = FP64_EV if prec == 0 else MIX_EV
                np.testing.assert_allclose(terms["lnI"][h], r["lnI"], rtol=0, atol=etol)
                xtol = 1e-10 if prec == 0 else 3e-6
                assert abs(math.log(terms["xi"][h]) - math.log(r["xi"])) <= xtol
                assert neff[h] == pytest.approx(r["neff"], rel=1e-8 if prec == 0 else 1e-4)
    finally:
        ctx.unload(cid)


def test_config1_tiny_catalog(chim, ctx, orc):
    from synth import catalog as sc
    cat = sc.config_catalog(1)
    th = np.vstack([sc.config_hyperpoints(1), sc.make_hyperpoints(3, seed=7)])
    _compare(chim, ctx, orc, cat, th)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("xi0_variant", [0, 2])
def test_scaled_o5_catalog(chim, ctx, orc, mode, xi0_variant):
    """Configuration 2 shapes at reduced size: 1-64 pixels, lognormal galaxy
    counts, 1000-point grid, ragged sample counts."""
    from synth import catalog as sc
    cat = sc.config_catalog(2, variant=xi0_variant, n_events=12, n_pe=1500, n_inj=30000,
                            gal_median=200, kde_mode=mode)
    th = sc.config_hyperpoints(2, variant=xi0_variant, n=3)
    _compare(chim, ctx, orc, cat, th)


@pytest.mark.parametrize("n_z", [999, 1001, 998])
def test_grid_not_multiple_of_four(chim, ctx, orc, n_z):
    """Grids whose length is not a multiple of 4: the profile rows are not
    16-byte aligned, so the mixed event kernel stages its paired Horner
    tables element by element instead of as float4 (both layouts must give
    the oracle's ln I)."""
    from synth import catalog as sc
    cat = sc.config_catalog(2, n_events=10, n_pe=1500, n_inj=20000, gal_median=200, n_z=n_z)
    th = sc.config_hyperpoints(2, n=3)
    _compare(chim, ctx, orc, cat, th)


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_photometric_16bit_storage(chim, ctx, orc, storage):
    """Photo-z galaxies (sigma = 0.05(1+z)) stored as F32 / F16 / BF16: the
    mixed path against the oracle fed the same stored values."""
    from synth import catalog as sc
    cat = sc.config_catalog(3, n_events=6, n_pe=1200, n_inj=20000, gal_median=150,
                            gal_storage=storage)
    th = sc.config_hyperpoints(3, n=2)
    oc_cat = sc.quantize_galaxies(cat, storage)
    oc = orc.Catalog(oc_cat)
    cid = ctx.load(cat)
    try:
        lnL, neff, st = ctx.loglike(cid, th, 1)
        for h in range(th.shape[0]):
            r = oc.loglike(th[h])
            assert abs(lnL[h] - r["lnL"]) <= 1e-3
    finally:
        ctx.unload(cid)


def _edge_catalog(orc, n_z=400):
    rng = np.random.default_rng(11)
    t = tc.theta()
    dg = lambda z: orc.dL_gw(z, t)
    evs = []
    # ragged sample counts, including 1 and around the warp/group sizes
    for n, z0, rel in [(1, 0.4, 0.05), (31, 0.5, 0.05), (33, 0.6, 0.08), (65, 0.3, 0.1),
                       (129, 1.2, 0.12), (700, 0.05, 0.02), (500, 1.45, 0.1)]:
        d0 = dg(z0)
        dL = d0 * np.abs(1 + rel * rng.standard_normal(n))
        m1 = (30 + 4 * rng.standard_normal(n)) * (1 + z0)
        m2 = (22 + 4 * rng.standard_normal(n)) * (1 + z0)
        m1, m2 = np.maximum(m1, m2), np.minimum(m1, m2)
        npix = 3 if n > 3 else 1
        pix = rng.integers(0, npix, n)
        S = np.bincount(pix, minlength=npix) / (n * 1e-4)
        gal = [list(z0 + 0.02 * rng.standard_normal(5)) for _ in range(npix)]
        if npix > 1:
            gal[1] = []  # a pixel without galaxies
        evs.append(dict(dL=dL, m1d=m1, m2d=m2, pix=pix, S=S, gal_z=gal,
                        gal_sigma=[[1e-3] * len(g) for g in gal]))
    evs[3]["dL"][5] = dg(10.0) * 3.0  # one sample beyond d_L^gw(10)
    inj_n = 3000
    di = (10 ** 3 + rng.random(inj_n) * (2e4 ** 3 - 1e3)) ** (1 / 3)
    a1 = 3 * np.exp(rng.random(inj_n) * np.log(400 / 3))
    a2 = 3 + rng.random(inj_n) * (a1 - 3)
    lp = np.log(3 * di ** 2 / (2e4 ** 3 - 1e3)) - np.log(a1 * np.log(400 / 3)) - np.log(a1 - 3)
    inj = dict(dL=di, m1d=a1, m2d=a2, log_pi=lp)
    return tc.build(evs, n_z=n_z, inj=inj, n_inj_total=10000)


def test_edge_cases(chim, ctx, orc):
    cat = _edge_catalog(orc)
    th = np.vstack([tc.theta(), tc.theta(Xi0=1.7, H0=64.0),
                    tc.theta(m_min=50.0, m_max=40.0),      # inadmissible
                    tc.theta(Xi0=0.01, n=40.0),             # non-monotone d_L^gw
                    tc.theta(m_min=150.0, m_max=190.0)])    # no sample survives
    _compare(chim, ctx, orc, cat, th)
    cat1 = dict(cat)
    cat1["kde_mode"] = 0
    _compare(chim, ctx, orc, cat1, th[:2])


def test_no_detected_injections(chim, ctx, orc):
    cat = _edge_catalog(orc)
    for k in ("inj_dL", "inj_m1d", "inj_m2d", "inj_log_pi"):
        cat[k] = cat[k][:0]
    cid = ctx.load(cat)
    try:
        lnL, neff, st = ctx.loglike(cid, tc.theta(), 1)
        assert lnL[0] == -math.inf and st[0] & chim.PT_OUT_OF_SUPPORT
    finally:
        ctx.unload(cid)


def test_batch_independence_and_determinism(chim, ctx):
    from synth import catalog as sc
    cat = sc.config_catalog(2, n_events=10, n_pe=1000, n_inj=20000, gal_median=100)
    th = sc.config_hyperpoints(2, n=6)
    cid = ctx.load(cat)
    try:
        for prec in (0, 1):
            full, _, _ = ctx.loglike(cid, th, prec)
            again, _, _ = ctx.loglike(cid, th, prec)
            assert np.array_equal(full, again)
            for h in (0, 3, 5):
                alone, _, _ = ctx.loglike(cid, th[h:h + 1], prec)
                assert alone[0] == full[h]
            sub, _, _ = ctx.loglike(cid, th[[5, 1, 3]], prec)
            assert np.array_equal(sub, full[[5, 1, 3]])
    finally:
        ctx.unload(cid)


def test_device_pointer_entry(chim, ctx):
    import torch
    from synth import catalog as sc
    cat = sc.config_catalog(1)
    th = sc.make_hyperpoints(4, seed=3)
    cid = ctx.load(cat)
    try:
        host, neff_h, st_h = ctx.loglike(cid, th, 1)
        tt = torch.tensor(th, device="cuda:0", dtype=torch.float64)
        out = torch.empty(4, device="cuda:0", dtype=torch.float64)
        neff = torch.empty_like(out)
        st = torch.empty(4, device="cuda:0", dtype=torch.int32)
        chim.chimera_loglike_device(ctx.h, cid, tt, 1, out, neff, st)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), host)
        assert np.array_equal(st.cpu().numpy(), st_h)
    finally:
        ctx.unload(cid)


@pytest.fixture(scope="module")
def full_c2(chim, ctx):
    from synth import catalog as sc
    cat = sc.config_catalog(2)
    cid = ctx.load(cat)
    yield cat, cid
    ctx.unload(cid)


def test_full_size_o5_sampled_events(chim, ctx, orc, full_c2):
    """Configuration 2 at full size (300 events x 5000 PE, 2e6 injections) in
    the launch the benchmark times (16 hyperpoints, mixed): sampled events
    and the selection term against the oracle, one at a time."""
    from synth import catalog as sc
    cat, cid = full_c2
    th = sc.config_hyperpoints(2)
    terms = ctx.terms(cid, th, 1)
    oc = orc.Catalog(cat)
    rng = np.random.default_rng(5)
    evs = [0, cat["n_events"] - 1] + list(rng.choice(cat["n_events"], 2, replace=False))
    for h in (0, 7):
        for ev in evs:
            ref = oc.event_lnI(th[h], int(ev))
            assert abs(terms["lnI"][h, ev] - ref) <= MIX_EV, (h, ev)
    xi, neff = oc.selection(th[0])
    assert abs(math.log(terms["xi"][0]) - math.log(xi)) <= 3e-6
    # FP64 single point at full size
    t64 = ctx.terms(cid, th[:1], 0)
    for ev in evs:
        assert abs(t64["lnI"][0, ev] - oc.event_lnI(th[0], int(ev))) <= FP64_EV
