"""The no-allocation selection entry point (chimera_selection_static), for
callers that may not allocate device memory (a memory pool that owns the
device, another framework's allocator, loops that must not let cudaMalloc or
cudaFree synchronise the device).  It must give the same selection term as
the catalog path, through the C ABI, on consecutive calls that reuse its
fixed device array.  Kept in a file of its own that pytest collects last."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_selection_matches_catalog_path():
    import torch

    from paper_2504_02034_b300 import build
    build.build()
    import paper_2504_02034_b300 as pkg
    from synth import catalog as sc

    cat = sc.config_catalog(2, n_events=4, n_pe=300, n_inj=200000, gal_median=50)
    th = sc.config_hyperpoints(2, n=5)
    th[3, 1] = 0.31                     # a second Om
    th[4, 7], th[4, 8] = 60.0, 50.0     # an inadmissible point
    with pkg.Context(0) as ctx:
        cid = ctx.load(cat)
        ref = ctx.terms(cid, th, pkg.FP64)
    dev = torch.device("cuda", 0)
    inj = {k: torch.tensor(cat[key], device=dev, dtype=torch.float64)
           for k, key in (("dL", "inj_dL"), ("m1d", "inj_m1d"), ("m2d", "inj_m2d"), ("log_pi", "inj_log_pi"))}
    for call in range(2):
        xi = torch.full((th.shape[0],), float("nan"), device=dev, dtype=torch.float64)
        neff = torch.full_like(xi, float("nan"))
        pkg.chimera_selection_static(th, inj, cat["n_inj_total"], cat["lambda_g"], cat["beta"],
                                     cat["z_max"], xi, neff)
        torch.cuda.synchronize()
        xi_h, neff_h = xi.cpu().numpy(), neff.cpu().numpy()
        for h in range(th.shape[0]):
            if ref["xi"][h] == 0.0:
                assert xi_h[h] == 0.0 and neff_h[h] == 0.0, (call, h)
                continue
            # FP64 path tolerances of the parity tests
            assert abs(math.log(xi_h[h]) - math.log(ref["xi"][h])) <= 1e-10, (call, h)
            assert neff_h[h] == pytest.approx(ref["neff"][h], rel=1e-8), (call, h)
    assert ref["xi"][4] == 0.0


def test_static_selection_rejects_oversize():
    import torch

    from paper_2504_02034_b300 import build
    build.build()
    import paper_2504_02034_b300 as pkg
    dev = torch.device("cuda", 0)
    z = torch.ones(4, device=dev, dtype=torch.float64)
    th = np.tile(np.array([70.0, 0.3, 1.0, 1.91, 3.4, 34.0, 3.6, 5.0, 100.0, 2.7, 3.0, 2.0]), (65, 1))
    out = torch.zeros(65, device=dev, dtype=torch.float64)
    with pytest.raises(pkg.ChimeraError) as e:
        pkg.chimera_selection_static(th, dict(dL=z, m1d=z, m2d=z, log_pi=z), 10, 0.039, 1.1, 1.5, out, out)
    assert e.value.code == pkg.CHIMERA_ERR_UNSUPPORTED
