"""Host-side failure paths, tested without a GPU fault: an allocation that
fails (CHIMERA_FAULT_ALLOC makes the N-th budgeted device allocation after
the variable is set fail) during a catalog load and during a likelihood
call's workspace set-up, after which the same context keeps working; and the
serving poll's timeout on a request that is still on the GPU."""
import math
import os

import numpy as np
import pytest

from synth import catalog as sc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chim():
    from paper_2504_02034_b300 import build
    build.build()
    import paper_2504_02034_b300 as pkg
    return pkg


def _with_fault(n):
    class _F:
        def __enter__(self):
            os.environ["CHIMERA_FAULT_ALLOC"] = str(n)

        def __exit__(self, *a):
            os.environ.pop("CHIMERA_FAULT_ALLOC", None)
    return _F()


def test_allocation_failure_during_load_and_call_leaves_context_usable(chim):
    cat = sc.config_catalog(2, n_events=4, n_pe=400, n_inj=8000, gal_median=30)
    th = sc.config_hyperpoints(2, n=3)
    with chim.Context(0) as ctx:
        for n in (1, 3):
            with _with_fault(n):
                with pytest.raises(chim.ChimeraError) as e:
                    ctx.load(cat)
            assert e.value.code == chim.CHIMERA_ERR_CUDA and "injected" in str(e.value)
        cid = ctx.load(cat)
        # the first call sizes the workspace: make one of its allocations fail
        with _with_fault(2):
            with pytest.raises(chim.ChimeraError) as e:
                ctx.loglike(cid, th, chim.MIXED)
        assert e.value.code == chim.CHIMERA_ERR_CUDA
        lnL, neff, st = ctx.loglike(cid, th, chim.MIXED)
        lnL64, _, _ = ctx.loglike(cid, th, chim.FP64)
        ctx.unload(cid)
    # the same results as a context that never saw a failure
    with chim.Context(0) as ctx2:
        c2 = ctx2.load(cat)
        ref, _, _ = ctx2.loglike(c2, th, chim.MIXED)
        ref64, _, _ = ctx2.loglike(c2, th, chim.FP64)
    np.testing.assert_array_equal(lnL, ref)
    np.testing.assert_array_equal(lnL64, ref64)
    assert np.all(np.isfinite(lnL))


def test_serve_poll_times_out_while_pending_then_completes(chim):
    cat = sc.config_catalog(2, n_events=120, n_pe=3000, n_inj=200000, gal_median=300)
    th = sc.make_hyperpoints(256, seed=77, Xi0=1.0)
    with chim.Context(0) as ctx:
        cid = ctx.load(cat)
        ticket = chim.chimera_serve_submit(ctx.h, cid, th, chim.SERVE_MIXED | chim.SERVE_GRAD)
        # a 256-point gradient request over 120 events takes tens of ms on
        # the GPU: a poll that does not wait finds it pending
        assert chim.chimera_serve_poll(ctx.h, ticket, th.shape[0], timeout_us=0, grad=True) is None
        out = chim.chimera_serve_poll(ctx.h, ticket, th.shape[0], timeout_us=-1, grad=True)
        assert out is not None
        lnL, g, st = out
        ref, gref, _ = ctx.grad(cid, th, chim.MIXED)
        np.testing.assert_array_equal(lnL, ref)
        np.testing.assert_array_equal(g, gref)
        # the ticket is forgotten after its successful poll
        with pytest.raises(chim.ChimeraError) as e:
            chim.chimera_serve_poll(ctx.h, ticket, th.shape[0], timeout_us=0, grad=True)
        assert e.value.code == chim.CHIMERA_ERR_NOT_FOUND
        ctx.unload(cid)


def test_results_reproducible_between_interleaved_calls(chim):
    """ln L and the mixed gradient of a batch are the same bit for bit when
    calls on another catalog run in between (the reweighting kernel sorts
    its deferred FP64 samples, whose list fills in atomic order, before
    adding their moments, so the bandwidths do not depend on timing)."""
    a = sc.config_catalog(2, n_events=40, n_pe=3000, n_inj=100000, gal_median=300)
    b = sc.config_catalog(2, variant=2, n_events=60, n_pe=2500, n_inj=80000, gal_median=300)
    th = sc.make_hyperpoints(16, seed=5, Xi0=1.0)
    thb = sc.make_hyperpoints(16, seed=6, Xi0=1.8)
    with chim.Context(0) as ctx:
        ia, ib = ctx.load(a), ctx.load(b)
        lnL0, g0, st0 = ctx.grad(ia, th, chim.MIXED)
        terms0 = ctx.terms(ia, th, chim.MIXED)
        for _ in range(3):
            ctx.grad(ib, thb, chim.MIXED)
            ctx.loglike(ib, thb[:7], chim.MIXED)
            lnL, g, st = ctx.grad(ia, th, chim.MIXED)
            terms = ctx.terms(ia, th, chim.MIXED)
            np.testing.assert_array_equal(lnL, lnL0)
            np.testing.assert_array_equal(g, g0)
            np.testing.assert_array_equal(st, st0)
            np.testing.assert_array_equal(terms["bw"], terms0["bw"])
            np.testing.assert_array_equal(terms["lnI"], terms0["lnI"])
