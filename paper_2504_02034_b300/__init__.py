"""Python binding of libchimera, the B300 (sm_103a) standard-siren likelihood
of arXiv 2504.02034 (CHIMERA 2.0).

The functions named ``chimera_*`` mirror the C ABI of include/chimera.h one
to one and only marshal arguments (numpy / torch buffers -> pointers); every
stage of the likelihood runs in the CUDA kernels of libchimera.so.  There is
no CPU fallback: importing works without a GPU, but creating a context on a
machine without one raises, and a missing library raises at first use.

``Context`` is a small convenience layer over the same calls, and
``ChimeraLogLike`` is a ``torch.autograd.Function`` whose backward uses the
library's hand-written adjoint.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchimera.so")

CHIMERA_OK = 0
CHIMERA_ERR_INVALID_ARG = -1
CHIMERA_ERR_NOT_FOUND = -2
CHIMERA_ERR_ADMISSION = -3
CHIMERA_ERR_CUDA = -4
CHIMERA_ERR_TIMEOUT = -5
CHIMERA_ERR_CANCELLED = -6
CHIMERA_ERR_UNSUPPORTED = -7
PT_OK, PT_OUT_OF_SUPPORT, PT_NONMONOTONE, PT_NEFF_LOW = 0, 1, 2, 4
FP64, MIXED, MIXED_BINNED = 0, 1, 2
KERNEL_EPANECHNIKOV = 0x10  # OR'ed into the precision: Epanechnikov KDE kernel
JACOBIAN_PER_SAMPLE = 0x20  # OR'ed into the precision: the Jacobian of Eq. jacobian on each sample
PROFILE_CUDA_CORES, PROFILE_TENSOR_CORES = 0, 1  # catalog info "profile_path"
KDE_SINGLE_1D, KDE_MANY_1D, KDE_3D = 0, 1, 2
GAL_F32, GAL_F16, GAL_BF16 = 0, 1, 2
SERVE_GRAD, SERVE_MIXED = 1, 2
NPARAM = 12
PARAM_NAMES = ("H0", "Om", "Xi0", "n", "alpha", "mu_g", "sigma_g",
               "m_min", "m_max", "gamma", "kappa", "z_p")


class ChimeraError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        detail = ""
        if _lib is not None:
            detail = _lib.chimera_last_error().decode()
            name = _lib.chimera_strerror(code).decode()
        else:
            name = str(code)
        super().__init__("%s: %s (%d) %s" % (where, name, code, detail))


class CatalogDesc(C.Structure):
    _fields_ = [
        ("n_events", C.c_int32),
        ("sample_off", C.POINTER(C.c_int64)),
        ("dL_Mpc", C.POINTER(C.c_double)), ("m1_det", C.POINTER(C.c_double)),
        ("m2_det", C.POINTER(C.c_double)),
        ("pix_of_sample", C.POINTER(C.c_int32)),
        ("pix_off", C.POINTER(C.c_int64)),
        ("sky_S", C.POINTER(C.c_double)),
        ("gal_off", C.POINTER(C.c_int64)),
        ("gal_z", C.POINTER(C.c_double)), ("gal_sigma", C.POINTER(C.c_double)),
        ("n_gal_total", C.c_double),
        ("z_max", C.c_double),
        ("n_z", C.c_int32),
        ("n_inj_total", C.c_int64),
        ("n_det", C.c_int64),
        ("inj_dL", C.POINTER(C.c_double)), ("inj_m1d", C.POINTER(C.c_double)),
        ("inj_m2d", C.POINTER(C.c_double)), ("inj_log_pi", C.POINTER(C.c_double)),
        ("lambda_g", C.c_double), ("beta", C.c_double),
        ("kde_mode", C.c_int32),
        ("gal_storage", C.c_int32),
        ("f_R", C.c_double),
        ("pix_area", C.POINTER(C.c_double)),
        ("completeness", C.POINTER(C.c_double)),
        ("sky_xy", C.POINTER(C.c_double)),
        ("pix_xy", C.POINTER(C.c_double)),
    ]


class CatalogInfo(C.Structure):
    _fields_ = [("n_events", C.c_int32), ("n_z", C.c_int32), ("n_samples", C.c_int64),
                ("n_pixels", C.c_int64), ("n_galaxies", C.c_int64), ("n_det", C.c_int64),
                ("device_bytes", C.c_int64), ("max_samples_per_event", C.c_int32),
                ("max_pixels_per_event", C.c_int32), ("profile_path", C.c_int32),
                ("event_kernel_warps", C.c_int32)]


class ServeStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("batches", C.c_int64), ("points", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("admitted_bytes_peak", C.c_int64)]


_lib = None
_P = C.c_void_p
_pd = C.POINTER(C.c_double)
_pi32 = C.POINTER(C.c_int32)
_pi64 = C.POINTER(C.c_int64)

# name -> (restype, argtypes), the exported C ABI
ABI = {
    "chimera_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_size_t]),
    "chimera_destroy": (None, [_P]),
    "chimera_load_catalog": (C.c_int, [_P, C.POINTER(CatalogDesc), _pi32]),
    "chimera_unload_catalog": (C.c_int, [_P, C.c_int32]),
    "chimera_catalog_info": (C.c_int, [_P, C.c_int32, C.POINTER(CatalogInfo)]),
    "chimera_loglike": (C.c_int, [_P, C.c_int32, C.c_int32, _pd, C.c_int32, _pd, _pd, _pi32]),
    "chimera_loglike_device": (C.c_int, [_P, C.c_int32, C.c_int32, _P, C.c_int32, _P, _P, _P, _P]),
    "chimera_terms": (C.c_int, [_P, C.c_int32, C.c_int32, _pd, C.c_int32, _pd, _pd, _pd, _pd]),
    "chimera_grad": (C.c_int, [_P, C.c_int32, C.c_int32, _pd, C.c_int32, _pd, _pd, _pi32]),
    "chimera_serve_submit": (C.c_int, [_P, C.c_int32, C.c_int32, _pd, C.c_int32, C.POINTER(C.c_uint64)]),
    "chimera_serve_poll": (C.c_int, [_P, C.c_uint64, C.c_int64, _pd, _pd, _pi32]),
    "chimera_serve_cancel": (C.c_int, [_P, C.c_uint64]),
    "chimera_serve_stats": (C.c_int, [_P, C.POINTER(ServeStats)]),
    "chimera_serve_reset_stats": (C.c_int, [_P]),
    "chimera_strerror": (C.c_char_p, [C.c_int]),
    "chimera_last_error": (C.c_char_p, []),
    "chimera_set_trace": (C.c_int, [_P, C.c_int]),
    "chimera_stage_ms": (C.c_int, [_P, _pd]),
    "chimera_kde_pairs": (C.c_int, [_P, C.c_int32, C.c_int32, _pd, _pi64]),
    "chimera_peaks": (C.c_int, [_P, _pd]),
    "chimera_memory": (C.c_int, [_P, _pi64]),
    "chimera_selection_static": (C.c_int, [C.c_int32, _pd, C.c_int64, C.c_int64, _P, _P, _P, _P,
                                           C.c_double, C.c_double, C.c_double, _P, _P, _P]),
}


def lib():
    """The loaded libchimera.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libchimera.so is missing at %s; build it with "
                               "`python paper_2504_02034_b300/build.py` (no CPU fallback exists)"
                               % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in ABI.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ck(rc, where):
    if rc != CHIMERA_OK:
        raise ChimeraError(rc, where)


def _dp(a):
    return a.ctypes.data_as(_pd)


def _th(theta):
    t = np.ascontiguousarray(np.atleast_2d(np.asarray(theta, dtype=np.float64)))
    if t.shape[1] != NPARAM:
        raise ValueError("theta must have 12 columns")
    return t


# ---------------------------------------------------------------- thin ABI
def chimera_create(device=0, hbm_budget_bytes=0):
    h = _P()
    _ck(lib().chimera_create(C.byref(h), int(device), int(hbm_budget_bytes)), "chimera_create")
    return h


def chimera_destroy(h):
    lib().chimera_destroy(h)


def make_desc(cat):
    """Build a CatalogDesc from a catalog dict (see synth.catalog); returns
    (desc, keepalive) - keep the second item alive until the load returns."""
    keep = {}

    def arr(key, dt):
        a = np.ascontiguousarray(cat[key], dtype=dt)
        keep[key] = a
        return a.ctypes.data_as(C.POINTER(np.ctypeslib.as_ctypes_type(dt)))

    def opt(key):  # optional array: NULL when absent (the library reports what is missing)
        return arr(key, np.float64) if cat.get(key) is not None else None

    ndet = int(np.asarray(cat["inj_dL"]).size)
    d = CatalogDesc(
        int(cat["n_events"]), arr("sample_off", np.int64),
        arr("dL", np.float64), arr("m1_det", np.float64), arr("m2_det", np.float64),
        arr("pix_of_sample", np.int32), arr("pix_off", np.int64), arr("sky_S", np.float64),
        arr("gal_off", np.int64), arr("gal_z", np.float64), arr("gal_sigma", np.float64),
        float(cat["n_gal_total"]), float(cat["z_max"]), int(cat["n_z"]),
        int(cat["n_inj_total"]), ndet,
        arr("inj_dL", np.float64), arr("inj_m1d", np.float64), arr("inj_m2d", np.float64),
        arr("inj_log_pi", np.float64),
        float(cat["lambda_g"]), float(cat["beta"]),
        int(cat.get("kde_mode", KDE_MANY_1D)), int(cat.get("gal_storage", GAL_F32)),
        float(cat.get("f_R", 1.0)),
        opt("pix_area") if cat.get("completeness") is not None else None,
        opt("completeness"),
        opt("sky_xy") if int(cat.get("kde_mode", KDE_MANY_1D)) == KDE_3D else None,
        opt("pix_xy") if int(cat.get("kde_mode", KDE_MANY_1D)) == KDE_3D else None)
    return d, keep


def chimera_load_catalog(h, cat):
    d, keep = make_desc(cat)
    cid = C.c_int32()
    _ck(lib().chimera_load_catalog(h, C.byref(d), C.byref(cid)), "chimera_load_catalog")
    del keep
    return cid.value


def chimera_unload_catalog(h, cid):
    _ck(lib().chimera_unload_catalog(h, cid), "chimera_unload_catalog")


def chimera_catalog_info(h, cid):
    info = CatalogInfo()
    _ck(lib().chimera_catalog_info(h, cid, C.byref(info)), "chimera_catalog_info")
    return {k: getattr(info, k) for k, _ in CatalogInfo._fields_}


def chimera_loglike(h, cid, theta, precision=MIXED):
    t = _th(theta)
    n = t.shape[0]
    lnL, neff = np.zeros(n), np.zeros(n)
    st = np.zeros(n, dtype=np.int32)
    _ck(lib().chimera_loglike(h, cid, n, _dp(t), precision, _dp(lnL), _dp(neff),
                              st.ctypes.data_as(_pi32)), "chimera_loglike")
    return lnL, neff, st


def chimera_loglike_device(h, cid, theta_t, precision, lnL_t, neff_t=None, status_t=None, stream=None):
    """Device-pointer form: torch CUDA tensors (float64 [n,12], float64 [n],
    float64 [n], int32 [n]) on the context's device; stream is a
    torch.cuda.Stream or None for the current torch stream."""
    import torch
    n = theta_t.shape[0]
    dev = theta_t.device
    # the C side writes n elements of each output through raw pointers: check
    # types, lengths and placement here (a few microseconds of host time)
    if (theta_t.dtype != torch.float64 or theta_t.dim() != 2 or theta_t.shape[1] != NPARAM
            or not theta_t.is_contiguous() or dev.type != "cuda"):
        raise ValueError("theta_t must be a contiguous float64 CUDA tensor of shape [n, %d]" % NPARAM)
    for name, x, dt in (("lnL_t", lnL_t, torch.float64), ("neff_t", neff_t, torch.float64),
                        ("status_t", status_t, torch.int32)):
        if x is not None and (x.dtype != dt or x.device != dev or x.numel() < n or not x.is_contiguous()):
            raise ValueError("%s must be a contiguous %s tensor of >= %d elements on %s" % (name, dt, n, dev))
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    # torch's default stream has handle 0, which the C ABI would read as "the
    # context's own stream"; pass the legacy default stream handle instead
    sh = s.cuda_stream if s.cuda_stream != 0 else 0x1
    _ck(lib().chimera_loglike_device(
        h, cid, n, C.c_void_p(theta_t.data_ptr()), precision, C.c_void_p(lnL_t.data_ptr()),
        C.c_void_p(neff_t.data_ptr()) if neff_t is not None else None,
        C.c_void_p(status_t.data_ptr()) if status_t is not None else None,
        C.c_void_p(sh)), "chimera_loglike_device")


def chimera_terms(h, cid, theta, precision=MIXED, n_events=None):
    t = _th(theta)
    n = t.shape[0]
    if n_events is None:
        n_events = chimera_catalog_info(h, cid)["n_events"]
    lnI, bw = np.zeros((n, n_events)), np.zeros((n, n_events))
    xi, neff = np.zeros(n), np.zeros(n)
    _ck(lib().chimera_terms(h, cid, n, _dp(t), precision, _dp(lnI), _dp(bw), _dp(xi), _dp(neff)),
        "chimera_terms")
    return dict(lnI=lnI, bw=bw, xi=xi, neff=neff)


def chimera_grad(h, cid, theta, precision=MIXED):
    t = _th(theta)
    n = t.shape[0]
    lnL, g = np.zeros(n), np.zeros((n, NPARAM))
    st = np.zeros(n, dtype=np.int32)
    _ck(lib().chimera_grad(h, cid, n, _dp(t), precision, _dp(lnL), _dp(g), st.ctypes.data_as(_pi32)),
        "chimera_grad")
    return lnL, g, st


def chimera_serve_submit(h, cid, theta, flags=SERVE_MIXED):
    t = _th(theta)
    tk = C.c_uint64()
    _ck(lib().chimera_serve_submit(h, cid, t.shape[0], _dp(t), flags, C.byref(tk)),
        "chimera_serve_submit")
    return tk.value


def chimera_serve_poll(h, ticket, n, timeout_us=-1, grad=False):
    """Returns (lnL, dlnL or None, status), or None while pending (timeout)."""
    lnL = np.zeros(n)
    g = np.zeros((n, NPARAM)) if grad else None
    st = np.zeros(n, dtype=np.int32)
    rc = lib().chimera_serve_poll(h, ticket, int(timeout_us), _dp(lnL),
                                  _dp(g) if grad else None, st.ctypes.data_as(_pi32))
    if rc == CHIMERA_ERR_TIMEOUT:
        return None
    _ck(rc, "chimera_serve_poll")
    return lnL, g, st


def chimera_serve_cancel(h, ticket):
    _ck(lib().chimera_serve_cancel(h, ticket), "chimera_serve_cancel")


def chimera_serve_stats(h):
    s = ServeStats()
    _ck(lib().chimera_serve_stats(h, C.byref(s)), "chimera_serve_stats")
    return {k: getattr(s, k) for k, _ in ServeStats._fields_}


def chimera_serve_reset_stats(h):
    _ck(lib().chimera_serve_reset_stats(h), "chimera_serve_reset_stats")


def chimera_set_trace(h, enable=True):
    _ck(lib().chimera_set_trace(h, int(bool(enable))), "chimera_set_trace")


def chimera_stage_ms(h):
    ms = np.zeros(7)
    _ck(lib().chimera_stage_ms(h, _dp(ms)), "chimera_stage_ms")
    return dict(tables=ms[0], galaxy=ms[1], event=ms[2], selection=ms[3], combine=ms[4], adjoint=ms[5],
                reweight=ms[6])


def chimera_kde_pairs(h, cid, theta):
    t = _th(theta)
    out = np.zeros(t.shape[0], dtype=np.int64)
    _ck(lib().chimera_kde_pairs(h, cid, t.shape[0], _dp(t), out.ctypes.data_as(_pi64)),
        "chimera_kde_pairs")
    return out


def chimera_memory(h):
    """Device-memory accounting of a context: budget, held, catalogs, caches,
    workspaces (bytes)."""
    out = np.zeros(5, dtype=np.int64)
    _ck(lib().chimera_memory(h, out.ctypes.data_as(_pi64)), "chimera_memory")
    return dict(zip(("budget", "held", "catalogs", "caches", "workspaces"), (int(x) for x in out)))


def chimera_peaks(h):
    out = np.zeros(4)
    _ck(lib().chimera_peaks(h, _dp(out)), "chimera_peaks")
    return dict(pair_per_s=out[0], ex2_per_s=out[1], dfma_per_s=out[2], copy_bytes_per_s=out[3])


def chimera_selection_static(theta, inj, n_inj_total, lambda_g, beta, z_max, xi_t, neff_t, stream=None):
    """No-allocation selection term.  inj: dict of float64 CUDA tensors
    dL, m1d, m2d, log_pi (same length); xi_t, neff_t: float64 CUDA tensors
    [n_points] written on `stream` (torch stream or None = current)."""
    import torch
    t = _th(theta)
    dev = xi_t.device
    n = int(inj["dL"].numel())
    for name in ("dL", "m1d", "m2d", "log_pi"):
        x = inj[name]
        if x.dtype != torch.float64 or not x.is_contiguous() or x.device != dev or x.numel() != n:
            raise ValueError("inj[%r] must be a contiguous float64 tensor of %d elements on %s"
                             % (name, n, dev))
    for name, x in (("xi_t", xi_t), ("neff_t", neff_t)):
        if x.dtype != torch.float64 or not x.is_contiguous() or x.device != dev or x.numel() < t.shape[0]:
            raise ValueError("%s must be a contiguous float64 tensor of >= %d elements on %s"
                             % (name, t.shape[0], dev))
    if dev.type != "cuda":
        raise ValueError("xi_t, neff_t and the injection tensors must be CUDA tensors (got %s)" % dev)
    ptr = lambda x: C.c_void_p(x.data_ptr())
    # the C call runs on the calling thread's current device: make it the outputs' one
    with torch.cuda.device(dev):
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        sh = s.cuda_stream if s.cuda_stream != 0 else 0x1
        _ck(lib().chimera_selection_static(t.shape[0], _dp(t), n, int(n_inj_total),
                                           ptr(inj["dL"]), ptr(inj["m1d"]), ptr(inj["m2d"]), ptr(inj["log_pi"]),
                                           float(lambda_g), float(beta), float(z_max), ptr(xi_t), ptr(neff_t),
                                           C.c_void_p(sh)), "chimera_selection_static")


def chimera_strerror(code):
    return lib().chimera_strerror(code).decode()


# ---------------------------------------------------------------- classes
class Context:
    """One GPU, its resident catalogs and its serving loop."""

    def __init__(self, device=0, hbm_budget_bytes=0):
        self.h = chimera_create(device, hbm_budget_bytes)

    def close(self):
        if self.h:
            chimera_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, cat):
        return chimera_load_catalog(self.h, cat)

    def unload(self, cid):
        chimera_unload_catalog(self.h, cid)

    def info(self, cid):
        return chimera_catalog_info(self.h, cid)

    def loglike(self, cid, theta, precision=MIXED):
        return chimera_loglike(self.h, cid, theta, precision)

    def terms(self, cid, theta, precision=MIXED):
        return chimera_terms(self.h, cid, theta, precision)

    def grad(self, cid, theta, precision=MIXED):
        return chimera_grad(self.h, cid, theta, precision)


def _autograd():
    import torch

    class ChimeraLogLike(torch.autograd.Function):
        """ln L(theta) for theta [n, 12] (float64, any device); backward
        applies the library's adjoint gradient d ln L / d theta."""

        @staticmethod
        def forward(ctx, theta, context, catalog_id, precision=MIXED):
            t = theta.detach().to("cpu", torch.float64).numpy()
            if theta.requires_grad:
                lnL, g, st = chimera_grad(context.h, catalog_id, t, precision)
                ctx.save_for_backward(torch.from_numpy(g).to(theta.device))
            else:
                lnL, _, st = chimera_loglike(context.h, catalog_id, t, precision)
            return torch.from_numpy(lnL).to(theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out.unsqueeze(-1) * g, None, None, None

    return ChimeraLogLike


def __getattr__(name):
    if name == "ChimeraLogLike":
        return _autograd()
    raise AttributeError(name)
