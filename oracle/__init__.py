"""Python handle on the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by the cpu_baseline / reference legs of bench.py, never by the product
package.  The oracle shares no code with the CUDA path.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

OK, OUT_OF_SUPPORT, NONMONOTONE, NEFF_LOW = 0, 1, 2, 4
GAUSSIAN, EPANECHNIKOV = 0, 1  # KDE kernel shapes
JACOBIAN_GRID, JACOBIAN_PER_SAMPLE = 0, 1  # placement of the Jacobian of Eq. jacobian
KDE_SINGLE_1D, KDE_MANY_1D, KDE_3D = 0, 1, 2  # KDE variants (Sec. 2.3)


def build(force=False):
    """Compile oracle.c with gcc (plain IEEE double, no fast-math, no FMA
    contraction, OpenMP for the timed CPU baseline)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _SO
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-D_GNU_SOURCE",
           "-o", _SO, _SRC, "-lm"]
    subprocess.check_call(cmd)
    return _SO


class _Cat(C.Structure):
    _fields_ = [
        ("n_events", C.c_int64),
        ("sample_off", C.POINTER(C.c_int64)),
        ("dL", C.POINTER(C.c_double)), ("m1d", C.POINTER(C.c_double)), ("m2d", C.POINTER(C.c_double)),
        ("pix_of_sample", C.POINTER(C.c_int32)),
        ("pix_off", C.POINTER(C.c_int64)),
        ("sky_S", C.POINTER(C.c_double)),
        ("gal_off", C.POINTER(C.c_int64)),
        ("gal_z", C.POINTER(C.c_double)), ("gal_sigma", C.POINTER(C.c_double)),
        ("n_gal_total", C.c_double),
        ("z_max", C.c_double),
        ("n_z", C.c_int64),
        ("n_inj_total", C.c_int64),
        ("n_det", C.c_int64),
        ("inj_dL", C.POINTER(C.c_double)), ("inj_m1d", C.POINTER(C.c_double)),
        ("inj_m2d", C.POINTER(C.c_double)), ("inj_log_pi", C.POINTER(C.c_double)),
        ("lambda_g", C.c_double), ("beta", C.c_double),
        ("kde_mode", C.c_int32),
        ("kernel", C.c_int32),
        ("f_R", C.c_double),
        ("pix_area", C.POINTER(C.c_double)),
        ("completeness", C.POINTER(C.c_double)),
        ("jacobian", C.c_int32),
        ("sky_xy", C.POINTER(C.c_double)),
        ("pix_xy", C.POINTER(C.c_double)),
    ]


class _Hooks(C.Structure):
    _fields_ = [("psi_scale", C.c_double), ("mass_scale", C.c_double), ("flags", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        d, pd, pi32 = C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int32)
        for name, args in [("orc_E", [d, d]), ("orc_Dc", [d, d, d]), ("orc_Xi", [d, d, d]),
                           ("orc_dL_em", [d, d, d]), ("orc_dL_gw", [d, pd]), ("orc_J", [d, pd]),
                           ("orc_dVc_dz", [d, d, d]), ("orc_Vc", [d, d, d]),
                           ("orc_p_m1", [d, pd, d]), ("orc_p_m2", [d, d, pd, d]), ("orc_psi", [d, pd])]:
            f = getattr(L, name)
            f.argtypes = args
            f.restype = d
        L.orc_z_of_dL.argtypes = [d, pd, pd]
        L.orc_z_of_dL.restype = C.c_int
        L.orc_check_theta.argtypes = [pd]
        L.orc_monotone.argtypes = [pd]
        pc, ph = C.POINTER(_Cat), C.POINTER(_Hooks)
        L.orc_event_samples.argtypes = [pc, pd, C.c_int64, pd, pd, pi32]
        L.orc_event_bandwidth.argtypes = [pc, pd, C.c_int64, pd]
        L.orc_event_kde.argtypes = [pc, pd, C.c_int64, C.c_int32, pd]
        L.orc_galaxy_profile.argtypes = [pc, pd, C.c_int64, C.c_int32, ph, pd]
        L.orc_grid_factor.argtypes = [pc, pd, ph, pd]
        L.orc_event_lnI.argtypes = [pc, pd, C.c_int64, ph, pd]
        L.orc_selection.argtypes = [pc, pd, ph, C.c_int, pd, pd, pd]
        L.orc_loglike.argtypes = [pc, pd, ph, C.c_int, pd, pd, pd, pd, pi32]
        L.orc_loglike_binned.argtypes = [pc, pd, ph, C.c_int, pd, pd, pd, pd, pi32]
        L.orc_event_kde_binned.argtypes = [pc, pd, C.c_int64, C.c_int32, pd]
        L.orc_event_lnI_binned.argtypes = [pc, pd, C.c_int64, ph, pd]
        L.orc_linear_bins.argtypes = [C.c_int64, pd, pd, d, C.c_int64, C.c_int64, pd]
        L.orc_linear_bins.restype = C.c_int64
        L.orc_kde_arrays.argtypes = [C.c_int64, pd, pd, d, C.c_int64, d, C.c_int32, C.c_int32, pd]
        L.orc_event_kde3_bandwidth.argtypes = [pc, pd, C.c_int64, pd]
        L.orc_event_kde3.argtypes = [pc, pd, C.c_int64, C.c_int32, pd]
        L.orc_dDc_dOm.argtypes = [d, d, d]
        L.orc_dDc_dOm.restype = d
        L.orc_grad.argtypes = [pc, pd, C.c_int, pd, pd, pi32]
        _lib = L
    return _lib


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def _th(theta):
    t = np.ascontiguousarray(theta, dtype=np.float64)
    assert t.shape == (12,)
    return t


def hooks(psi_scale=1.0, mass_scale=1.0, flags=0):
    return _Hooks(psi_scale, mass_scale, flags)


class Catalog:
    """Oracle view of a catalog dict (see synth.catalog.make_catalog)."""

    def __init__(self, cat, kde_mode=None, kernel=0, jacobian=0):
        self.keep = {}

        def arr(key, dt):
            a = np.ascontiguousarray(cat[key], dtype=dt)
            self.keep[key] = a
            return a

        so = arr("sample_off", np.int64)
        self.n_events = int(cat["n_events"])
        self.n_z = int(cat["n_z"])
        self.z_max = float(cat["z_max"])
        inj = arr("inj_dL", np.float64)
        self.c = _Cat(
            self.n_events, _p(so, C.c_int64),
            _p(arr("dL", np.float64)), _p(arr("m1_det", np.float64)), _p(arr("m2_det", np.float64)),
            _p(arr("pix_of_sample", np.int32), C.c_int32),
            _p(arr("pix_off", np.int64), C.c_int64),
            _p(arr("sky_S", np.float64)),
            _p(arr("gal_off", np.int64), C.c_int64),
            _p(arr("gal_z", np.float64)), _p(arr("gal_sigma", np.float64)),
            float(cat["n_gal_total"]), float(cat["z_max"]), int(cat["n_z"]),
            int(cat["n_inj_total"]), int(inj.size),
            _p(inj), _p(arr("inj_m1d", np.float64)), _p(arr("inj_m2d", np.float64)),
            _p(arr("inj_log_pi", np.float64)),
            float(cat["lambda_g"]), float(cat["beta"]),
            int(cat["kde_mode"] if kde_mode is None else kde_mode),
            int(kernel),
            float(cat.get("f_R", 1.0)),
            _p(arr("pix_area", np.float64)) if cat.get("completeness") is not None else None,
            _p(arr("completeness", np.float64)) if cat.get("completeness") is not None else None,
            int(jacobian),
            _p(arr("sky_xy", np.float64)) if cat.get("sky_xy") is not None else None,
            _p(arr("pix_xy", np.float64)) if cat.get("pix_xy") is not None else None,
        )

    @property
    def ref(self):
        return C.byref(self.c)

    def n_samples(self, ev):
        so = self.keep["sample_off"]
        return int(so[ev + 1] - so[ev])

    # ---- stages
    def samples(self, theta, ev):
        n = self.n_samples(ev)
        z, w = np.zeros(n), np.zeros(n)
        v = np.zeros(n, dtype=np.int32)
        lib().orc_event_samples(self.ref, _p(_th(theta)), ev, _p(z), _p(w), _p(v, C.c_int32))
        return z, w, v.astype(bool)

    def bandwidth(self, theta, ev):
        b = C.c_double()
        lib().orc_event_bandwidth(self.ref, _p(_th(theta)), ev, C.byref(b))
        return b.value

    def kde(self, theta, ev, pixel=-1, binned=False):
        K = np.zeros(self.n_z)
        f = lib().orc_event_kde_binned if binned else lib().orc_event_kde
        f(self.ref, _p(_th(theta)), ev, pixel, _p(K))
        return K

    def kde3_bandwidth(self, theta, ev):
        """Bandwidth matrix of the "3D" kernel over (z, x, y) (None if degenerate)."""
        H = np.zeros(9)
        rc = lib().orc_event_kde3_bandwidth(self.ref, _p(_th(theta)), ev, _p(H))
        return None if rc else H.reshape(3, 3)

    def kde3(self, theta, ev, pixel):
        """The "3D" KDE at the grid points of one pixel's centre."""
        K = np.zeros(self.n_z)
        lib().orc_event_kde3(self.ref, _p(_th(theta)), ev, pixel, _p(K))
        return K

    def galaxy_profile(self, theta, ev, pixel, hk=None):
        G = np.zeros(self.n_z)
        lib().orc_galaxy_profile(self.ref, _p(_th(theta)), ev, pixel, C.byref(hk or hooks()), _p(G))
        return G

    def grid_factor(self, theta, hk=None):
        F = np.zeros(self.n_z)
        lib().orc_grid_factor(self.ref, _p(_th(theta)), C.byref(hk or hooks()), _p(F))
        return F

    def event_lnI(self, theta, ev, hk=None, binned=False):
        v = C.c_double()
        f = lib().orc_event_lnI_binned if binned else lib().orc_event_lnI
        f(self.ref, _p(_th(theta)), ev, C.byref(hk or hooks()), C.byref(v))
        return v.value

    def selection(self, theta, hk=None, nthreads=0, want_s=False):
        xi, ne = C.c_double(), C.c_double()
        n = int(self.c.n_det)
        s = np.zeros(max(n, 1)) if want_s else None
        lib().orc_selection(self.ref, _p(_th(theta)), C.byref(hk or hooks()), nthreads,
                            C.byref(xi), C.byref(ne), _p(s) if want_s else None)
        return (xi.value, ne.value, s[:n]) if want_s else (xi.value, ne.value)

    def loglike(self, theta, hk=None, nthreads=0, binned=False):
        """Returns dict(lnL, lnI[n_events], xi, neff, status)."""
        lnL, xi, ne = C.c_double(), C.c_double(), C.c_double()
        st = C.c_int32()
        lnI = np.zeros(max(self.n_events, 1))
        f = lib().orc_loglike_binned if binned else lib().orc_loglike
        f(self.ref, _p(_th(theta)), C.byref(hk or hooks()), nthreads,
                          C.byref(lnL), _p(lnI), C.byref(xi), C.byref(ne), C.byref(st))
        return dict(lnL=lnL.value, lnI=lnI[: self.n_events], xi=xi.value, neff=ne.value,
                    status=st.value)

    def grad(self, theta, nthreads=0):
        """ln L and its analytic gradient (12), the hand-derived FP64 chain
        (Gaussian kernel, Jacobian on the grid): returns (lnL, grad, status)."""
        lnL = C.c_double()
        st = C.c_int32()
        g = np.zeros(12)
        lib().orc_grad(self.ref, _p(_th(theta)), nthreads, C.byref(lnL), _p(g), C.byref(st))
        return lnL.value, g, st.value

    def grad_fd(self, theta, rel_step=1e-4, nthreads=0, hk=None):
        """Central finite differences of the oracle ln L, step rel_step*|theta_k|
        (the definition of the derivative; the oracle's gradient)."""
        th = _th(theta).copy()
        g = np.zeros(12)
        for k in range(12):
            h = rel_step * max(abs(th[k]), 1e-3)
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            g[k] = (self.loglike(tp, hk, nthreads)["lnL"] - self.loglike(tm, hk, nthreads)["lnL"]) / (2 * h)
        return g


# scalar helpers (theta-vector functions)
def E(z, Om):
    return lib().orc_E(z, Om)


def Dc(z, H0, Om):
    return lib().orc_Dc(z, H0, Om)


def Xi(z, Xi0, n):
    return lib().orc_Xi(z, Xi0, n)


def dL_em(z, H0, Om):
    return lib().orc_dL_em(z, H0, Om)


def dL_gw(z, theta):
    return lib().orc_dL_gw(z, _p(_th(theta)))


def J(z, theta):
    return lib().orc_J(z, _p(_th(theta)))


def dVc_dz(z, H0, Om):
    return lib().orc_dVc_dz(z, H0, Om)


def Vc(z, H0, Om):
    return lib().orc_Vc(z, H0, Om)


def dDc_dOm(z, H0, Om):
    return lib().orc_dDc_dOm(z, H0, Om)


def z_of_dL(d, theta):
    z = C.c_double()
    rc = lib().orc_z_of_dL(d, _p(_th(theta)), C.byref(z))
    return z.value if rc == 0 else None


def p_m1(m1, theta, lambda_g):
    return lib().orc_p_m1(m1, _p(_th(theta)), lambda_g)


def p_m2(m2, m1, theta, beta):
    return lib().orc_p_m2(m2, m1, _p(_th(theta)), beta)


def psi(z, theta):
    return lib().orc_psi(z, _p(_th(theta)))


def check_theta(theta):
    return lib().orc_check_theta(_p(_th(theta)))


def monotone(theta):
    return lib().orc_monotone(_p(_th(theta)))


def linear_bins(z, w, dz, b0, nb):
    """Linear binning of weighted samples onto nodes b0 .. b0+nb-1 of the
    lattice b dz; returns (node weights, parts that fell outside)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    cb = np.zeros(int(nb))
    lost = lib().orc_linear_bins(z.size, _p(z), _p(w), float(dz), int(b0), int(nb), _p(cb))
    return cb, int(lost)


def kde_arrays(z, w, b, n_z, z_max, binned=False, kernel=GAUSSIAN):
    """Weighted KDE (Gaussian of width b or Epanechnikov of width sqrt(5) b;
    1/N normalisation, support: sample range +- 6 b) of the samples (z, w) on
    the grid of n_z points on [0, z_max]."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    K = np.zeros(int(n_z))
    lib().orc_kde_arrays(z.size, _p(z), _p(w), float(b), int(n_z), float(z_max), int(binned), int(kernel), _p(K))
    return K
