"""The no-allocation selection entry point (chimera_selection_static), for
callers that may not allocate device memory (a memory pool that owns the
device, another framework's allocator, loops that must not let cudaMalloc or
cudaFree synchronise the device).  Through the C ABI, on consecutive calls
that reuse its fixed device array, it must give the oracle's selection term
and the catalog path's, and it must leave the device's free memory and
torch's allocator untouched.  Kept in a file of its own that pytest collects
last."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pkg():
    from paper_2504_02034_b300 import build
    build.build()
    import paper_2504_02034_b300 as pkg
    return pkg


def _inj(cat, dev):
    import torch
    return {k: torch.tensor(cat[key], device=dev, dtype=torch.float64)
            for k, key in (("dL", "inj_dL"), ("m1d", "inj_m1d"), ("m2d", "inj_m2d"), ("log_pi", "inj_log_pi"))}


def _call(pkg, th, inj, cat, dev):
    import torch
    xi = torch.full((th.shape[0],), float("nan"), device=dev, dtype=torch.float64)
    neff = torch.full_like(xi, float("nan"))
    pkg.chimera_selection_static(th, inj, cat["n_inj_total"], cat["lambda_g"], cat["beta"],
                                 cat["z_max"], xi, neff)
    torch.cuda.synchronize()
    return xi.cpu().numpy(), neff.cpu().numpy()


def test_static_selection_matches_oracle_and_catalog_path(orc):
    import torch
    pkg = _pkg()
    from synth import catalog as sc

    cat = sc.config_catalog(2, n_events=4, n_pe=300, n_inj=200000, gal_median=50)
    th = sc.config_hyperpoints(2, n=5)
    th[3, 1] = 0.31                     # a second Om
    th[4, 7], th[4, 8] = 60.0, 50.0     # an inadmissible point
    with pkg.Context(0) as ctx:
        cid = ctx.load(cat)
        ref = ctx.terms(cid, th, pkg.FP64)
    oc = orc.Catalog(cat)
    oref = [oc.selection(t) if orc.check_theta(t) == 0 else (0.0, 0.0) for t in th]
    dev = torch.device("cuda", 0)
    inj = _inj(cat, dev)
    for call in range(2):
        xi_h, neff_h = _call(pkg, th, inj, cat, dev)
        for h in range(th.shape[0]):
            if oref[h][0] == 0.0:
                assert ref["xi"][h] == 0.0 and xi_h[h] == 0.0 and neff_h[h] == 0.0, (call, h)
                continue
            # FP64 path tolerances of the parity tests, against the oracle
            assert abs(math.log(xi_h[h]) - math.log(oref[h][0])) <= 1e-10, (call, h)
            assert neff_h[h] == pytest.approx(oref[h][1], rel=1e-8), (call, h)
            # and against the catalog path (inverse table over the injections
            # alone here, so ~1e-10 rather than bit for bit)
            assert abs(math.log(xi_h[h]) - math.log(ref["xi"][h])) <= 1e-10, (call, h)
    assert oref[4][0] == 0.0


def test_static_selection_allocates_nothing_64_distinct_om():
    """64 points with 64 distinct Om fill the array's table regions; after a
    first call (lazy module loading may take device memory once), further
    calls change neither the device's free memory nor torch's allocator."""
    import torch
    pkg = _pkg()
    from synth import catalog as sc

    cat = sc.config_catalog(2, n_events=3, n_pe=200, n_inj=100000, gal_median=20)
    th = sc.config_hyperpoints(2, n=64)
    th[:, 1] = np.linspace(0.22, 0.38, 64)
    assert len(np.unique(th[:, 1])) == 64
    with pkg.Context(0) as ctx:
        cid = ctx.load(cat)
        ref = ctx.terms(cid, th, pkg.FP64)
    dev = torch.device("cuda", 0)
    inj = _inj(cat, dev)
    _call(pkg, th, inj, cat, dev)
    xi_o = torch.empty(64, device=dev, dtype=torch.float64)
    ne_o = torch.empty_like(xi_o)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    res0 = torch.cuda.memory_reserved(dev)
    outs = []
    for _ in range(2):
        pkg.chimera_selection_static(th, inj, cat["n_inj_total"], cat["lambda_g"], cat["beta"],
                                     cat["z_max"], xi_o, ne_o)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info(dev)[0] == free0
        assert torch.cuda.memory_reserved(dev) == res0
        outs.append(xi_o.cpu().numpy().copy())
    assert np.array_equal(outs[0], outs[1])
    ok = ref["xi"] > 0
    assert ok.all()
    np.testing.assert_allclose(np.log(outs[1]), np.log(ref["xi"]), rtol=0, atol=1e-10)


def test_static_selection_rejects_oversize_and_bad_distances():
    import torch
    pkg = _pkg()
    dev = torch.device("cuda", 0)
    z = torch.ones(4, device=dev, dtype=torch.float64)
    fid = np.array([70.0, 0.3, 1.0, 1.91, 3.4, 34.0, 3.6, 5.0, 100.0, 2.7, 3.0, 2.0])
    th = np.tile(fid, (65, 1))
    out = torch.zeros(65, device=dev, dtype=torch.float64)
    with pytest.raises(pkg.ChimeraError) as e:
        pkg.chimera_selection_static(th, dict(dL=z, m1d=z, m2d=z, log_pi=z), 10, 0.039, 1.1, 1.5, out, out)
    assert e.value.code == pkg.CHIMERA_ERR_UNSUPPORTED
    # no positive distance: the inverse table would have no range
    zero = torch.zeros(4, device=dev, dtype=torch.float64)
    with pytest.raises(pkg.ChimeraError) as e:
        pkg.chimera_selection_static(th[:2], dict(dL=zero, m1d=z, m2d=z, log_pi=z), 10, 0.039, 1.1, 1.5,
                                     out, out)
    assert e.value.code == pkg.CHIMERA_ERR_INVALID_ARG
    # mismatched lengths are refused before the call
    with pytest.raises(ValueError):
        pkg.chimera_selection_static(th[:2], dict(dL=z, m1d=z[:3], m2d=z, log_pi=z), 10, 0.039, 1.1, 1.5,
                                     out, out)
