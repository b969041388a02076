"""Benchmark: ln L evaluations per second (hyperpoints x events) of the
hierarchical standard-siren likelihood on the 300-event O5-like catalog
(300 events x 5000 PE samples, 1-64 pixels, lognormal galaxy counts,
1000-point redshift grid, 2e6 injections), 16 walker hyperpoints per launch,
mixed precision, beside the plain FP64 one-point-per-call path.

One step = one chimera_loglike call over the batch (cosmology tables,
reweighting + KDE x galaxy integrals, selection term, combine).  The catalog
is resident in HBM; `value` times the device-pointer entry point with CUDA
events, `e2e` times the host-pointer entry point (hyperpoints copied in,
ln L copied out) end to end.  L2 is flushed (a 256 MiB write) between timed
steps because the catalog (~100 MB) would otherwise stay L2-resident.

Beside the headline: the plain FP64 one-point-per-call path, ln L with its
gradient (chimera_grad, mixed and FP64), serving streams (Poisson arrivals
over four resident catalogs of 100 to 5000 events, 1-512 points per request,
a quarter with gradients: one at the configuration's 2 ms mean interarrival,
beyond one GPU's capacity, and one offered at 0.7 x the capacity that run
measures) with their p50/p99 latency, the batched photometric workload (512
points per launch, BF16 galaxies; Om fixed and Om varying) and the
differentiation workload (5000 events, 64 points, ln L + gradient).

Run: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun): every rank evaluates its own walkers on its own GPU
(independent replicas, weak scaling); only a barrier and a max of the times
cross ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ln L evals/s (hyperpoints x events) at 300 events, mixed vs FP64; p50/p99 ms"
UNIT = "evals/s"
WORKLOAD = "O5-like catalog: 300 events x 5000 PE, 1-64 pixels, lognormal galaxies (median 2e3), n_z=1000, 2e6 injections, many-1D KDE, 16 hyperpoints per launch"
SM_COUNT = 148
FP32_LANES = 128
OPS_PER_PAIR = 1  # one FFMA per (sample, grid point): Horner step in exp(2 u ds)


def algorithmic_bytes(cat, H):
    """Algorithmic DRAM bytes of one event-kernel launch over H points (the
    scope table's count, amortised over the points of the launch): the PE
    samples (16 B each: distance coordinate and the two log masses), the
    galaxy profile rows (4 B per pixel and grid point, shared by the points
    of one Om) and the grid factor F (4 B per grid point and point)."""
    ns = int(cat["sample_off"][-1])
    npix = int(cat["pix_off"][-1])
    return 16 * ns + 4 * npix * int(cat["n_z"]) + 4 * int(cat["n_z"]) * H


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class _Nvml:
    """Read-only NVML queries through the driver's libnvidia-ml (ctypes)."""
    SW_POWER_CAP, HW_SLOWDOWN, SW_THERMAL, HW_THERMAL = 0x4, 0x8, 0x20, 0x40
    CLOCK_SM = 1

    def __init__(self, gpu):
        import ctypes as C
        self.C = C
        self.lib = C.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = C.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(gpu), C.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn if fn is not None else self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def clock(self, maximum=False):
        v = self.C.c_uint()
        f = self.lib.nvmlDeviceGetMaxClockInfo if maximum else self.lib.nvmlDeviceGetClockInfo
        if f(self.h, self.C.c_int(self.CLOCK_SM), self.C.byref(v)) != 0:
            raise OSError("clock query failed")
        return float(v.value)

    def reasons(self):
        v = self.C.c_ulonglong()
        if self.reasons_fn(self.h, self.C.byref(v)) != 0:
            raise OSError("reason query failed")
        return v.value


class Clocks:
    """SM clock and throttle-reason samples taken while the timed region runs:
    NVML (read-only) polled from a background thread every ~1 ms, with the
    nvidia-smi sampler as the fallback when NVML is unavailable."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.samples = []
        self.stop_flag = False
        self.th = None
        self.smi = None
        try:
            self.nv = _Nvml(gpu)
            self.max_mhz = self.nv.clock(maximum=True)
        except Exception:
            self.nv = None

    def _poll(self):
        nv = self.nv
        names = [("hw_slowdown", nv.HW_SLOWDOWN), ("hw_thermal_slowdown", nv.HW_THERMAL),
                 ("sw_thermal_slowdown", nv.SW_THERMAL), ("sw_power_cap", nv.SW_POWER_CAP)]
        while not self.stop_flag:
            try:
                mhz = nv.clock()
                bits = nv.reasons()
                self.samples.append((mhz, [n for n, b in names if bits & b]))
            except Exception:
                pass
            time.sleep(0.001)

    def start(self):
        if self.nv is not None:
            import threading
            self.th = threading.Thread(target=self._poll, daemon=True)
            self.th.start()
            return
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        fields = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                  "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.smi = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + fields,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.smi = None

    def stop(self):
        if self.th is not None:
            self.stop_flag = True
            self.th.join()
            if not self.samples:
                return None
            sm = [m for m, _ in self.samples]
            reasons = sorted({r for _, rs in self.samples for r in rs})
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": self.max_mhz, "reasons": reasons,
                    "samples": len(sm), "source": "nvml"}
        if self.smi is None:
            return None
        self.smi.terminate()
        try:
            self.smi.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.smi.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f.read().splitlines() if l.strip()]
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except (OSError, ValueError):
        return {}


def traffic_from_profiles():
    """DRAM bytes per event-kernel launch from the committed ncu summary, if
    it was taken on the current kernel source (event.cu with the headers it
    includes, whose constants set the kernel's windows and layout)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("event.cu", "internal.cuh", "mass.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2504_02034_b300", "csrc", name), "rb").read())
    sha = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", "event_mixed_o5_c2.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != sha:
        return None
    try:
        return float(vals["traffic_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def cpu_baseline(cat, thetas, budget_s=20.0):
    """The FP64 oracle, as it stands, on the host cores: hyperpoints of the
    benchmark batch over the first E events (with the matching share of
    injections), E and then the number of hyperpoints grown until the sample
    takes about budget_s / 2 of wall time."""
    import oracle
    cores = os.cpu_count() or 1
    ne = cat["n_events"]
    E, P = 8, 1
    while True:
        sub = _sub_catalog(cat, E)
        oc = oracle.Catalog(sub)
        t0 = time.perf_counter()
        for k in range(P):
            oc.loglike(thetas[k % len(thetas)], nthreads=cores)
        dt = time.perf_counter() - t0
        if dt * 2 > budget_s or (E >= ne and P >= len(thetas)):
            break
        grow = max(2.0, min(8.0, budget_s / max(dt, 1e-3) / 2))
        if E < ne:
            E = min(ne, int(E * grow))
        else:
            P = min(len(thetas), int(P * grow))
    # the same oracle on one thread, over a smaller slice of the same sample
    # (the first point, a quarter of the events, at least 4)
    E1 = max(4, min(E, E // 4))
    oc1 = oracle.Catalog(_sub_catalog(cat, E1))
    t1 = time.perf_counter()
    oc1.loglike(thetas[0], nthreads=1)
    dt1 = time.perf_counter() - t1
    return {"value": P * E / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d hyperpoint(s) x first %d of %d events with %d of %d detected injections, FP64, %d threads, %.1f s"
                      % (P, E, ne, sub["inj_dL"].size, cat["inj_dL"].size, cores, dt),
            "single_thread": {"value": E1 / dt1, "unit": UNIT,
                              "sample": "1 hyperpoint x first %d events (matching injections), FP64, 1 thread, %.1f s"
                                        % (E1, dt1)}}


def _sub_catalog(cat, E):
    ne = cat["n_events"]
    so, po, go = cat["sample_off"], cat["pix_off"], cat["gal_off"]
    ns, npx = so[E], po[E]
    nd = int(round(cat["inj_dL"].size * E / ne))
    sub = dict(cat)
    sub.update(n_events=E, sample_off=so[:E + 1], dL=cat["dL"][:ns], m1_det=cat["m1_det"][:ns],
               m2_det=cat["m2_det"][:ns], pix_of_sample=cat["pix_of_sample"][:ns], pix_off=po[:E + 1],
               sky_S=cat["sky_S"][:npx], gal_off=go[:npx + 1], gal_z=cat["gal_z"][:go[npx]],
               gal_sigma=cat["gal_sigma"][:go[npx]],
               n_inj_total=int(round(cat["n_inj_total"] * nd / max(cat["inj_dL"].size, 1))),
               inj_dL=cat["inj_dL"][:nd], inj_m1d=cat["inj_m1d"][:nd], inj_m2d=cat["inj_m2d"][:nd],
               inj_log_pi=cat["inj_log_pi"][:nd])
    return sub


def grad_stats(pkg, ctx, cid, theta, NE, reps=3):
    """ln L and its 12-component gradient through chimera_grad (host buffers),
    mixed and FP64, on the benchmark batch; adjoint stage time from the trace."""
    out = {}
    for name, prec, pts in (("mixed", pkg.MIXED, theta), ("fp64_single_point", pkg.FP64, theta[:1])):
        pkg.chimera_grad(ctx.h, cid, pts, prec)
        t, adj = [], []
        for _ in range(reps if prec == pkg.MIXED else 1):
            t0 = time.perf_counter()
            pkg.chimera_grad(ctx.h, cid, pts, prec)
            t.append(time.perf_counter() - t0)
            adj.append(pkg.chimera_stage_ms(ctx.h)["adjoint"])
        out[name] = {"value": pts.shape[0] * NE * len(t) / sum(t), "unit": "evals/s (ln L + 12 derivatives)",
                     "ms_per_call": 1e3 * sum(t) / len(t), "adjoint_ms": sum(adj) / len(adj),
                     "hyperpoints": int(pts.shape[0])}
    return out


def binned_stats(pkg, ctx, torch, dev, theta, steps):
    """The binned-KDE option (CHIMERA_MIXED_BINNED) against the unbinned mixed
    path on the benchmark catalog in its single-1D form (300 events x 5000
    PE, one KDE per event), 16 hyperpoints per launch, device-timed as the
    main step (CUDA events, L2 flushed between steps)."""
    from synth import catalog as sc
    cat = sc.config_catalog(2, kde_mode=sc.KDE_SINGLE_1D)
    cid = ctx.load(cat)
    H, NE = theta.shape[0], cat["n_events"]
    th_dev = torch.tensor(theta, device=dev, dtype=torch.float64)
    out = torch.empty(H, device=dev, dtype=torch.float64)
    neff = torch.empty_like(out)
    st = torch.empty(H, device=dev, dtype=torch.int32)
    flush = torch.empty(256 << 20, device=dev, dtype=torch.uint8)
    stream = torch.cuda.current_stream(dev)
    res = {"catalog": "300 events x 5000 PE, single-1D KDE, 16 hyperpoints per launch"}
    for name, prec in (("mixed", pkg.MIXED), ("binned", pkg.MIXED_BINNED)):
        for _ in range(3):
            pkg.chimera_loglike_device(ctx.h, cid, th_dev, prec, out, neff, st, stream)
        torch.cuda.synchronize()
        ms, ev_ms = [], []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pkg.chimera_loglike_device(ctx.h, cid, th_dev, prec, out, neff, st, stream)
            e1.record(stream)
            ev_ms.append(pkg.chimera_stage_ms(ctx.h)["event"])
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = sum(ms) / len(ms)
        res[name] = {"value": H * NE / (t * 1e-3), "unit": UNIT, "ms_per_step": t,
                     "event_kernel_ms": sum(ev_ms) / len(ev_ms)}
    lnL_b, _, _ = pkg.chimera_loglike(ctx.h, cid, theta, pkg.MIXED_BINNED)
    lnL_m, _, _ = pkg.chimera_loglike(ctx.h, cid, theta, pkg.MIXED)
    res["binned_over_mixed"] = res["binned"]["value"] / res["mixed"]["value"]
    res["max_abs_delta_lnL"] = float(np.max(np.abs(lnL_b - lnL_m)))
    ctx.unload(cid)
    return res


def kernel_option_stats(pkg, ctx, torch, dev, cid, theta, NE, steps):
    """The kernel options on the benchmark catalog and batch, device-timed as
    the main step: the Epanechnikov kernel (CHIMERA_KERNEL_EPANECHNIKOV) and
    the per-sample Jacobian (CHIMERA_JACOBIAN_PER_SAMPLE), mixed precision."""
    H = theta.shape[0]
    th_dev = torch.tensor(theta, device=dev, dtype=torch.float64)
    out = torch.empty(H, device=dev, dtype=torch.float64)
    neff = torch.empty_like(out)
    st = torch.empty(H, device=dev, dtype=torch.int32)
    flush = torch.empty(256 << 20, device=dev, dtype=torch.uint8)
    stream = torch.cuda.current_stream(dev)

    def timed(prec):
        for _ in range(3):
            pkg.chimera_loglike_device(ctx.h, cid, th_dev, prec, out, neff, st, stream)
        torch.cuda.synchronize()
        ms, ev_ms, rw_ms = [], [], []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pkg.chimera_loglike_device(ctx.h, cid, th_dev, prec, out, neff, st, stream)
            e1.record(stream)
            sm = pkg.chimera_stage_ms(ctx.h)
            ev_ms.append(sm["event"])
            rw_ms.append(sm["reweight"])
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = sum(ms) / len(ms)
        return {"value": H * NE / (t * 1e-3), "unit": UNIT, "ms_per_step": t,
                "event_kernel_ms": sum(ev_ms) / len(ev_ms), "reweight_ms": sum(rw_ms) / len(rw_ms)}

    epan = timed(pkg.MIXED | pkg.KERNEL_EPANECHNIKOV)
    epan["window"] = "|z - z_j| <= sqrt(5) b, one evaluation per pair"
    jac = timed(pkg.MIXED | pkg.JACOBIAN_PER_SAMPLE)
    jac["note"] = "the Jacobian evaluated per sample in the reweighting kernel, psi alone on the grid"
    return {"epanechnikov_mixed": epan, "jacobian_per_sample_mixed": jac}


def kde3_stats(pkg, ctx, cat, theta, calls=2):
    """The "3D" kernel (CHIMERA_KDE_3D, FP64, the cross-check variant) on the
    benchmark catalog loaded as a 3D-kernel catalog: one point per call
    through chimera_loglike, wall time per call (the FP64 many-1D path is
    fp64_single_point)."""
    c3 = dict(cat)
    c3["kde_mode"] = pkg.KDE_3D
    cid = ctx.load(c3)
    try:
        ts = []
        for k in range(calls + 1):
            t0 = time.perf_counter()
            pkg.chimera_loglike(ctx.h, cid, theta[k % theta.shape[0]:k % theta.shape[0] + 1], pkg.FP64)
            if k > 0:
                ts.append(time.perf_counter() - t0)
    finally:
        ctx.unload(cid)
    ms = 1e3 * sum(ts) / len(ts)
    return {"value": cat["n_events"] / (ms * 1e-3), "unit": UNIT, "ms_per_call": ms, "hyperpoints": 1,
            "precision": "FP64"}


def om_varying_stats(pkg, ctx, cid, theta, NE, calls=3):
    """Walkers whose Om is new at every point (the differentiation workload's
    pattern): every call brings 16 Om values never seen before, so each pays
    its distance tables and galaxy profiles (and, with the gradient, their Om
    derivatives).  ln L and ln L + gradient through the host entry points,
    mixed precision, on the benchmark catalog; wall time per call."""
    out = {}
    for name, fn in (("loglike", lambda t: pkg.chimera_loglike(ctx.h, cid, t, pkg.MIXED)),
                     ("gradient", lambda t: pkg.chimera_grad(ctx.h, cid, t, pkg.MIXED))):
        ts = []
        for k in range(calls + 1):
            t = theta.copy()
            t[:, 1] = 0.28 + 0.04 * np.random.default_rng(1000 * k + len(name)).random(theta.shape[0])
            t0 = time.perf_counter()
            fn(t)
            if k > 0:  # the first call warms the code paths
                ts.append(time.perf_counter() - t0)
        ms = 1e3 * sum(ts) / len(ts)
        out[name] = {"ms_per_call": ms, "value": theta.shape[0] * NE / (ms * 1e-3), "unit": UNIT,
                     "new_om_per_call": int(theta.shape[0])}
    return out


def serving_stream(pkg, ctx, bench_cid, bench_cat, n_req, n_paced, fp64_evals_per_s, seed=2504020345):
    """Request streams over four resident catalogs (spectroscopic 100 / 300 /
    1000 events at Xi0 = 0.6 / 1 / 1.8, photometric 5000 events x 4000 PE with
    x3 galaxies in BF16), 1-512 hyperpoints per request (log-uniform),
    gradient flag with probability 0.25, mixed precision:
    * "overloaded": n_req requests with Poisson arrivals of mean 2 ms (the
      configuration's rate, more than one GPU carries), whose achieved request
      rate measures the capacity and whose latencies are queue backlog;
    * "paced": n_paced requests offered at 0.7 x that capacity, where the
      latencies show the batching loop rather than a queue.
    Beside them, the plain FP64 one-point-per-call path in the same unit."""
    from synth import catalog as sc
    t_gen = time.perf_counter()
    cats = [(sc.config_catalog(2, variant=0, n_events=100), 0.6),
            (bench_cat, 1.0),
            (sc.config_catalog(2, variant=2, n_events=1000), 1.8),
            (sc.config_catalog(3, n_events=5000, n_pe=4000), 1.0)]
    cids = [ctx.load(c) if c is not bench_cat else bench_cid for c, _ in cats]
    nev = [c["n_events"] for c, _ in cats]
    t_gen = time.perf_counter() - t_gen
    # warm the per-catalog caches (galaxy profiles and their Om derivatives)
    for cid, (c, xi0) in zip(cids, cats):
        for flags in (pkg.SERVE_MIXED, pkg.SERVE_MIXED | pkg.SERVE_GRAD):
            tk = pkg.chimera_serve_submit(ctx.h, cid, sc.make_hyperpoints(1, seed=seed, Xi0=xi0), flags)
            pkg.chimera_serve_poll(ctx.h, tk, 1, grad=bool(flags & pkg.SERVE_GRAD))

    def run(n, mean_s, sd):
        rng = np.random.default_rng(sd)
        arrive = np.cumsum(rng.exponential(mean_s, n))
        which = rng.integers(0, len(cats), n)
        npts = np.clip(np.floor(np.exp(rng.uniform(0.0, np.log(513.0), n))), 1, 512).astype(int)
        want_grad = rng.random(n) < 0.25
        thetas = [sc.make_hyperpoints(int(k), seed=sd + 7 * i, Xi0=cats[w][1]) for i, (k, w) in enumerate(zip(npts, which))]
        pkg.chimera_serve_reset_stats(ctx.h)
        t0 = time.perf_counter()
        tickets = []
        for i in range(n):
            dt = t0 + arrive[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            flags = pkg.SERVE_MIXED | (pkg.SERVE_GRAD if want_grad[i] else 0)
            tickets.append(pkg.chimera_serve_submit(ctx.h, cids[which[i]], thetas[i], flags))
        for i, tk in enumerate(tickets):
            pkg.chimera_serve_poll(ctx.h, tk, int(npts[i]), grad=bool(want_grad[i]))
        wall = time.perf_counter() - t0
        st = pkg.chimera_serve_stats(ctx.h)
        evals = int(sum(int(k) * nev[w] for k, w in zip(npts, which)))
        return {"requests": n, "gradient_requests": int(want_grad.sum()), "hyperpoints": int(npts.sum()),
                "mean_interarrival_ms": 1e3 * mean_s, "offered_req_per_s": n / float(arrive[-1]),
                "achieved_req_per_s": n / wall, "evals_per_s": evals / wall, "unit": "evals/s",
                "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                "batches": st["batches"], "wall_s": wall}

    over = run(n_req, 2e-3, seed)
    out = {"catalog_events": nev, "precision": "mixed", "catalog_setup_s": t_gen, "overloaded": over,
           "fp64_single_point_evals_per_s": fp64_evals_per_s}
    if n_paced > 0:
        cap = over["achieved_req_per_s"]
        out["paced"] = run(n_paced, 1.0 / (0.7 * cap), seed + 1)
        out["paced"]["offered_fraction_of_capacity"] = 0.7
    for cid, (c, _) in zip(cids, cats):
        if c is not bench_cat:
            ctx.unload(cid)
    return out


def launch_stats(times_ms):
    t = np.sort(np.asarray(times_ms))
    return {"p50_ms": float(np.percentile(t, 50)), "p99_ms": float(np.percentile(t, 99)),
            "mean_ms": float(t.mean()), "launches": int(t.size)}


def config3_stats(pkg, ctx, torch, dev, flush, launches):
    """The batched photometric workload: 512 walker points per launch over
    the 300-event catalog with sigma_z = 0.05(1+z), x3 galaxies in BF16,
    mixed: per-launch time (device entry, CUDA events, L2 flushed) with Om
    fixed, and with a new Om at every point (the Om-varying run: 512
    profiles built per call, host entry, wall time)."""
    from synth import catalog as sc
    cat = sc.config_catalog(3)
    th = sc.config_hyperpoints(3)
    H, NE = th.shape[0], cat["n_events"]
    cid = ctx.load(cat)
    stream = torch.cuda.current_stream(dev)
    tt = torch.tensor(th, device=dev, dtype=torch.float64)
    out_t = torch.empty(H, device=dev, dtype=torch.float64)
    for _ in range(2):
        pkg.chimera_loglike_device(ctx.h, cid, tt, pkg.MIXED, out_t, None, None, stream)
    times = []
    for _ in range(launches):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pkg.chimera_loglike_device(ctx.h, cid, tt, pkg.MIXED, out_t, None, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    pkg.chimera_set_trace(ctx.h, True)
    pkg.chimera_loglike_device(ctx.h, cid, tt, pkg.MIXED, out_t, None, None, stream)
    torch.cuda.synchronize()
    stage = pkg.chimera_stage_ms(ctx.h)
    fixed = launch_stats(times)
    fixed.update(evals_per_s=H * NE / (1e-3 * fixed["mean_ms"]), stage_ms=stage,
                 tile_buffer_bytes_per_launch=int(2 * 8 * int(cat["sample_off"][-1]) * H))
    # Om varying: every point brings a new Om; the first such call (the
    # profile cache growing to its Om-varying size) is not timed
    rng = np.random.default_rng(91)
    wall = []
    for k in range(4):
        t2 = th.copy()
        t2[:, 1] = 0.25 + 0.1 * rng.random(H)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pkg.chimera_loglike(ctx.h, cid, t2, pkg.MIXED)
        if k:
            wall.append(time.perf_counter() - t0)
    stage_om = pkg.chimera_stage_ms(ctx.h)
    pkg.chimera_set_trace(ctx.h, False)
    ctx.unload(cid)
    return {"workload": "300 events x 5000 PE, photometric sigma_z = 0.05(1+z), x3 galaxies (BF16), "
                        "512 walker points per launch, mixed",
            "om_fixed": fixed,
            "om_varying": {"ms_per_call": 1e3 * float(np.mean(wall)), "calls": len(wall),
                           "evals_per_s": H * NE / float(np.mean(wall)), "stage_ms": stage_om}}


def config4_stats(pkg, ctx, calls):
    """The differentiation workload: ln L and the 12-component gradient at 64
    points (Om varying) over the 5000-event catalog (4000 PE, 5e6
    injections), mixed; and ln L alone at the same points."""
    from synth import catalog as sc
    cat = sc.config_catalog(4)
    th = sc.config_hyperpoints(4)
    H, NE = th.shape[0], cat["n_events"]
    cid = ctx.load(cat)
    pkg.chimera_grad(ctx.h, cid, th, pkg.MIXED)
    pkg.chimera_loglike(ctx.h, cid, th, pkg.MIXED)
    g, l = [], []
    for _ in range(calls):
        t0 = time.perf_counter()
        pkg.chimera_grad(ctx.h, cid, th, pkg.MIXED)
        g.append(1e3 * (time.perf_counter() - t0))
    for _ in range(calls):
        t0 = time.perf_counter()
        pkg.chimera_loglike(ctx.h, cid, th, pkg.MIXED)
        l.append(1e3 * (time.perf_counter() - t0))
    ctx.unload(cid)
    gs, ls = launch_stats(g), launch_stats(l)
    gs["evals_per_s"] = H * NE / (1e-3 * gs["mean_ms"])
    ls["evals_per_s"] = H * NE / (1e-3 * ls["mean_ms"])
    return {"workload": "5000 events x 4000 PE, 5e6 injections, 64 points with Om varying, mixed, host entry",
            "gradient": gs, "loglike": ls}


def run_reference(args, ws, rank):
    """Reference arm: the FP64 CPU oracle on the host cores."""
    if rank != 0:
        return
    from synth import catalog as sc
    cat = sc.config_catalog(2)
    th = sc.config_hyperpoints(2)
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    E = 16
    sub = _sub_catalog(cat, E)
    oc = oracle.Catalog(sub)
    for _ in range(args.warmup):
        oc.loglike(th[0], nthreads=cores)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oc.loglike(th[k % th.shape[0]], nthreads=cores)
        times.append(time.perf_counter() - t0)
    T = sum(times)
    val = E * args.steps / T
    sample = ("each step: 1 hyperpoint x first %d of 300 events with %d of %d detected injections, FP64, %d threads"
              % (E, sub["inj_dL"].size, cat["inj_dL"].size, cores))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--serve-requests", type=int, default=120,
                    help="length of the overloaded serving stream (0 skips serving)")
    ap.add_argument("--serve-paced", type=int, default=2000,
                    help="length of the serving stream offered at 0.7 x capacity (0 skips it)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the photometric 512-point and 5000-event gradient workloads")
    ap.add_argument("--profile", action="store_true",
                    help="run W warm-up launches and one more launch of the timed step, then exit (for ncu)")
    ap.add_argument("--profile-grad", action="store_true",
                    help="run W warm-up gradient calls (mixed, the benchmark batch) and one more, then exit (for ncu)")
    ap.add_argument("--profile-om", action="store_true",
                    help="run W warm-up ln L calls and one more, each bringing 16 new Om values "
                         "(mixed, the benchmark batch; one batched profile pass per call), then exit (for ncu)")
    ap.add_argument("--profile-photo-om", action="store_true",
                    help="load the photometric catalog (configuration 3) and run W warm-up ln L calls and one "
                         "more, each bringing 128 new Om values (tensor-core galaxy profiles), then exit (for ncu)")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        barrier(ws)
        return

    import torch
    import paper_2504_02034_b300 as pkg
    from paper_2504_02034_b300 import build as pkg_build
    from synth import catalog as sc

    pkg_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.profile_photo_om:
        pcat = sc.config_catalog(3)
        with pkg.Context(local) as pctx:
            pcid = pctx.load(pcat)
            for k in range(args.warmup + 1):
                t = sc.config_hyperpoints(3, n=128)
                t[:, 1] = np.linspace(0.2 + 0.06 * k, 0.25 + 0.06 * k, 128)
                pkg.chimera_loglike(pctx.h, pcid, t, pkg.MIXED)
        return
    cat = sc.config_catalog(2)
    theta = sc.make_hyperpoints(16, seed=sc.SEED_BASE + 25 + 1000 * rank, Xi0=1.0)
    H, NE = theta.shape[0], cat["n_events"]
    ctx = pkg.Context(local)
    cid = ctx.load(cat)
    peaks = None if (args.profile or args.profile_grad or args.profile_om) else pkg.chimera_peaks(ctx.h)

    th_dev = torch.tensor(theta, device=dev, dtype=torch.float64)
    out = torch.empty(H, device=dev, dtype=torch.float64)
    neff = torch.empty_like(out)
    st = torch.empty(H, device=dev, dtype=torch.int32)
    flush = torch.empty(256 << 20, device=dev, dtype=torch.uint8)
    stream = torch.cuda.current_stream(dev)

    def step():
        pkg.chimera_loglike_device(ctx.h, cid, th_dev, pkg.MIXED, out, neff, st, stream)

    if args.profile:
        for _ in range(args.warmup + 1):
            step()
        torch.cuda.synchronize()
        ctx.close()
        return
    if args.profile_grad:
        for _ in range(args.warmup + 1):
            pkg.chimera_grad(ctx.h, cid, theta, pkg.MIXED)
        ctx.close()
        return
    if args.profile_om:
        for k in range(args.warmup + 1):
            t = theta.copy()
            t[:, 1] = 0.28 + 0.04 * np.random.default_rng(500 + k).random(H)
            pkg.chimera_loglike(ctx.h, cid, t, pkg.MIXED)
        ctx.close()
        return
    pkg.chimera_set_trace(ctx.h, True)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    pairs = int(pkg.chimera_kde_pairs(ctx.h, cid, theta).sum())

    clocks = Clocks(local)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kern_ms, stage = [], []
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record(stream)
        step()
        ev1[k].record(stream)
        s = pkg.chimera_stage_ms(ctx.h)  # events on the library stream, around each kernel
        kern_ms.append(s["event"])
        stage.append(s)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(ws)
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    T = allmax(ws, sum(step_ms) / 1e3)
    value = ws * H * NE * args.steps / T
    step_sorted = sorted(step_ms)

    # e2e: host theta in, host ln L out, through chimera_loglike
    e2e_t = []
    for k in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lnL, _, _ = pkg.chimera_loglike(ctx.h, cid, theta, pkg.MIXED)
        e2e_t.append(time.perf_counter() - t0)
    e2e_T = allmax(ws, sum(e2e_t))
    e2e_val = ws * H * NE * len(e2e_t) / e2e_T

    # plain FP64 one point per call
    fp = []
    for k in range(args.fp64_steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pkg.chimera_loglike(ctx.h, cid, theta[k % H:k % H + 1], pkg.FP64)
        if k > 0:
            fp.append(time.perf_counter() - t0)
    fp64_val = NE * len(fp) / sum(fp)

    grads = grad_stats(pkg, ctx, cid, theta, NE)
    binned = binned_stats(pkg, ctx, torch, dev, theta, max(3, args.steps // 2)) if rank == 0 else None
    om_var = om_varying_stats(pkg, ctx, cid, theta, NE) if rank == 0 else None
    kern_opt = kernel_option_stats(pkg, ctx, torch, dev, cid, theta, NE, max(3, args.steps // 2)) if rank == 0 else None
    kde3 = kde3_stats(pkg, ctx, cat, theta) if rank == 0 else None
    serving = (serving_stream(pkg, ctx, cid, cat, args.serve_requests, args.serve_paced, fp64_val)
               if args.serve_requests > 0 and rank == 0 else None)
    c3 = config3_stats(pkg, ctx, torch, dev, flush, 10) if rank == 0 and not args.no_configs else None
    c4 = config4_stats(pkg, ctx, 3) if rank == 0 and not args.no_configs else None

    kern = sum(kern_ms) / len(kern_ms)
    clock_mhz = (clk or {}).get("sm_max_mhz") or 2032.0
    # The roofline of the scope table: the event kernel's windowed Gaussian
    # evaluations E per launch (pairs), each one SFU exponential and three
    # FP32 operations in the direct method, against the slowest of
    # E / (ex2 rate), 3 E / (FFMA rate) and the algorithmic bytes at the copy
    # bandwidth, with the rates K8 measured on this GPU.  The exponential
    # term binds, so achieved = E / t and peak = the measured ex2 rate.
    # (The kernel evaluates the Gaussians by Horner's rule, one FFMA per
    # pair, and could in principle run faster than this bound; its own
    # one-FFMA bound is reported beside it as "ffma_bound".)
    bw = (measured_peaks().get("hbm_gbs") or peaks["copy_bytes_per_s"] / 1e9) * 1e9
    alg_bytes = algorithmic_bytes(cat, H)
    t_bound = max(pairs / peaks["ex2_per_s"], 3 * pairs / peaks["pair_per_s"], alg_bytes / bw)
    achieved = pairs / (kern * 1e-3)
    roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peaks["ex2_per_s"] / 1e9, "unit": "Geval/s",
            "frac": t_bound / (kern * 1e-3),
            "traffic": traffic_from_profiles(),
            "kernel": "k_event_mixed", "pairs_per_launch": pairs, "kernel_ms": kern,
            "t_bound_ms": 1e3 * t_bound, "algorithmic_bytes_per_launch": alg_bytes,
            "peak_basis": "K8-measured MUFU ex2 rate (max of E/ex2 rate, 3E/FFMA rate, bytes/copy bandwidth binds on ex2)"}
    peak_pairs = SM_COUNT * FP32_LANES * clock_mhz * 1e6 / OPS_PER_PAIR
    roof["ffma_bound"] = {"achieved_gpair_s": achieved / 1e9, "peak_gpair_s": peak_pairs / 1e9,
                          "frac": achieved / peak_pairs,
                          "measured_pair_peak": peaks["pair_per_s"] / 1e9,
                          "frac_of_measured": achieved / peaks["pair_per_s"],
                          "basis": "148 SMs x 128 FP32 lanes x %.0f MHz x 1 FFMA per pair (derived)" % clock_mhz}
    mean_stage = {k: sum(s[k] for s in stage) / len(stage) for k in stage[0]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": T * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "hyperpoints_per_launch": H, "events": NE,
                   "pe_samples": int(cat["sample_off"][-1]), "n_z": int(cat["n_z"]),
                   "detected_injections": int(cat["inj_dL"].size), "l2": "flushed (256 MiB write) between steps",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "p50_ms": statistics.median(step_ms), "p99_ms": step_sorted[min(len(step_sorted) - 1, int(0.99 * len(step_sorted)))],
        "fp64_single_point": {"value": fp64_val, "unit": UNIT, "ms_per_call": 1e3 * sum(fp) / len(fp)},
        "mixed_over_fp64": value / ws / fp64_val,
        "stage_ms": mean_stage,
        "gradient": grads,
        "binned_kde": binned,
        "om_varying": om_var,
        "kernel_options": kern_opt,
        "kde_3d_fp64": kde3,
        "serving": serving,
        "photometric_512": c3,
        "differentiation_5000": c4,
        "device_memory_end": pkg.chimera_memory(ctx.h),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(theta.nbytes),
                "d2h_bytes_per_step": int(H * (8 + 8 + 4))},
        # per step: k_nodes_grid, k_inv_nodes, k_hyper_final, k_reweight,
        # k_event_mixed, k_select_mixed, k_combine (the forward table and galaxy
        # profile are cached)
        "gpu_launches": 7 * args.steps,
        "roofline": roof,
        "peaks_measured": {k: v for k, v in peaks.items()},
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cat, theta)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    barrier(ws)


if __name__ == "__main__":
    main()
