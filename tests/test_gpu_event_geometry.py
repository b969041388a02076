"""The mixed event kernel's two block geometries (10 warps with three blocks
per SM, 16 warps with two; chosen per catalog at load by the shared memory
its largest event needs, then by timing both on the first mixed call): the
same events give the same ln I bit for bit under either, and an event too
large for three blocks per SM matches the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


def _append(a, b):
    """Catalog a with b's events added after its own (a's injections and
    galaxy count, so a's events keep their ln I)."""
    out = dict(a)
    ns_a, np_a, ng_a = a["sample_off"][-1], a["pix_off"][-1], a["gal_off"][-1]
    out["n_events"] = a["n_events"] + b["n_events"]
    out["sample_off"] = np.concatenate([a["sample_off"], b["sample_off"][1:] + ns_a])
    out["pix_off"] = np.concatenate([a["pix_off"], b["pix_off"][1:] + np_a])
    out["gal_off"] = np.concatenate([a["gal_off"], b["gal_off"][1:] + ng_a])
    for k in ("dL", "m1_det", "m2_det", "pix_of_sample", "ra", "dec", "sky_xy", "sky_S", "pix_xy",
              "gal_z", "gal_sigma"):
        if k in a and k in b:
            out[k] = np.concatenate([a[k], b[k]])
    return out


def test_geometries_agree_and_large_event_matches_oracle(chim, ctx, orc):
    from synth import catalog as sc
    small = sc.config_catalog(2, n_events=6, n_pe=1500, n_inj=20000, gal_median=200)
    large = sc.config_catalog(2, variant=2, n_events=1, n_pe=9000, n_inj=2000, gal_median=200)
    both = _append(small, large)
    th = sc.config_hyperpoints(2, n=3)
    ids = ctx.load(small), ctx.load(both)
    try:
        assert ctx.info(ids[0])["event_kernel_warps"] == 10
        assert ctx.info(ids[1])["event_kernel_warps"] == 16
        ta = ctx.terms(ids[0], th, chim.MIXED)
        tb = ctx.terms(ids[1], th, chim.MIXED)
        # the first mixed call timed both geometries and kept one of them;
        # later calls give the same values
        for cid, t in zip(ids, (ta, tb)):
            assert ctx.info(cid)["event_kernel_warps"] in (10, 16)
            again = ctx.terms(cid, th, chim.MIXED)
            assert np.array_equal(again["lnI"], t["lnI"]) and np.array_equal(again["bw"], t["bw"])
        ne = small["n_events"]
        assert np.array_equal(ta["lnI"], tb["lnI"][:, :ne])
        assert np.array_equal(ta["bw"], tb["bw"][:, :ne])
        oc = orc.Catalog(both)
        for h in range(th.shape[0]):
            ref = oc.event_lnI(th[h], ne)
            assert abs(tb["lnI"][h, ne] - ref) <= 1e-4, (h, tb["lnI"][h, ne], ref)
    finally:
        for i in ids:
            ctx.unload(i)
