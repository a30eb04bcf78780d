#!/usr/bin/env python
"""Throughput benchmark: position-updates/s of the abc iteration at 256^2 patterns.

Workload ("large"): one blind scan of 1024 positions (32 x 32 raster, step 32 px,
jitter +-4), 256 x 256 patterns, 1300 x 1300 object, disk probe of radius 64 with
defocus, Poisson noise at 1e6 photons per pattern; RAAR(beta = 0.9), i.e.
(a, b, c) = (0.5, 1.8, 2.0), FP32.  Synthetic, seeded inputs.

A step is one iteration of x <- a P^b_C P^c_D x + (1 - a) x over all 1024 exit
waves (divide, object and probe concur, re-split); value = positions x steps /
device time, timed with CUDA events on the stream the library runs on.  The
working set (x, y, sqrt I: 1.3 GB) is ten times the L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the 4 x 4 block of positions at the top-left of the raster).
Multi-GPU: every rank runs an independent replica (the path has no exchange
that needs a collective here); value is the sum over ranks / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "position-updates/s at 256² patterns (FP32 vs BF16-split); p50/p99 recon latency"
UNIT = "position-updates/s"
RAAR = (0.5, 1.8, 2.0)
FALLBACK_HBM_GBS = 6800.0
KERNELS_PER_ITER = 6   # divide + object gather + object normalise + probe partial/reduce/normalise
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device) -> float:
    """Largest value over all ranks of the default process group (or value)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job rate of independent replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / seconds_max


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if re.match(r"^[\d.]+$", r[1])]
        mx = [float(r[2]) for r in rows if re.match(r"^[\d.]+$", r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


class NvmlClockSampler:
    """SM clock and clock-event reasons read through NVML (libnvidia-ml, read
    only) every millisecond on a background thread, so a timed region of tens
    of milliseconds still gets samples; `ok` is False when NVML cannot be
    loaded (the nvidia-smi sampler then stands alone)."""
    # public NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index: int):
        import ctypes
        import threading
        self.samples = []
        self.ok = False
        self._stop = threading.Event()
        self._thread = None
        try:
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                return
            self.dev = ctypes.c_void_p()
            if self.lib.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.dev)) != 0:
                return
            self.mx = ctypes.c_uint(0)
            self.lib.nvmlDeviceGetMaxClockInfo(self.dev, 1, ctypes.byref(self.mx))  # 1: SM clock
            self.ok = True
        except OSError:
            return

    def _run(self):
        import ctypes
        clk, rsn = ctypes.c_uint(0), ctypes.c_ulonglong(0)
        get_r = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self._stop.is_set():
            if self.lib.nvmlDeviceGetClockInfo(self.dev, 1, ctypes.byref(clk)) == 0 and \
                    get_r(self.dev, ctypes.byref(rsn)) == 0:
                self.samples.append((clk.value, rsn.value))
            time.sleep(0.001)

    def start(self):
        import threading
        if self.ok:
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()

    def stop(self) -> dict | None:
        if not self.ok or self._thread is None:
            return None
        self._stop.set()
        self._thread.join(timeout=2)
        if not self.samples:
            return None
        sm = [c for c, _ in self.samples]
        reasons = sorted({name for _, r in self.samples for bit, name in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(sm), "sm_min_mhz": min(sm), "sm_max_mhz": float(self.mx.value),
                "reasons": reasons, "samples": len(self.samples), "source": "nvml, 1 ms"}


def _bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        # a kernel timed inside a long step: the sustained figure
        return float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured (sustained)"
    return 1700.0, "fallback (sustained)"


def _kernel_hash(design: str = "cluster") -> str:
    h = hashlib.sha256()
    for f in ("divide2p.cu" if design == "twopass" else "divide.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2311_11466_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(N: int, J: int, design: str = "cluster"):
    """DRAM bytes per divide launch of the 1024 x 256^2 workload from the
    committed ncu summary of that divide design, if it was taken on the
    current kernel source (else None; None for any other workload)."""
    if (N, J) != (256, 1024):
        return None
    name = "divide2p_large_traffic.md" if design == "twopass" else "divide_large_traffic.md"
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != _kernel_hash(design):
        return None
    return float(t.group(1))


def _sub_scan(scan, side: int):
    import numpy as np
    nx = scan.spec.nx
    idx = np.array([iy * nx + ix for iy in range(side) for ix in range(side)])
    return idx


def oracle_rate(scan, side: int, min_seconds: float, max_iters: int):
    """Oracle position-updates/s on the side x side block of the raster."""
    import numpy as np
    from oracle import ptycho as optycho
    idx = _sub_scan(scan, side)
    prob = optycho.Problem(scan.intensity[idx].astype(np.float64), scan.pos[idx],
                           scan.obj0.astype(np.complex128), scan.probe0.astype(np.complex128))
    x = optycho.exit_waves(prob.P, prob.O, scan.pos[idx])
    times = []
    t_all = time.perf_counter()
    while len(times) < max_iters:
        t0 = time.perf_counter()
        x = prob.iterate(x, *RAAR)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all >= min_seconds:
            break
    return len(idx) * len(times) / sum(times), len(times), len(idx)


def tiny_both(local: int, iters: int = 100):
    """The 64-position 64 x 64 scan timed in full on both sides: 100 DC
    iterations of the FP64 oracle on the host cores and of the library on the
    GPU (CUDA events, after 5 warm-up iterations).  At this size the GPU is
    bound by kernel launches, not by the kernels."""
    import numpy as np
    import torch
    from oracle import ptycho as optycho
    from paper_2311_11466_gb300 import native, synth
    scan = synth.make_scan(synth.named_spec("tiny"))
    prob = optycho.Problem(scan.intensity.astype(np.float64), scan.pos,
                           scan.obj0.astype(np.complex128), scan.probe0.astype(np.complex128))
    x = optycho.exit_waves(prob.P, prob.O, scan.pos)
    t0 = time.perf_counter()
    for _ in range(iters):
        x = prob.iterate(x, 1.0, 1.0, 1.0)
    t_cpu = time.perf_counter() - t0
    stream = torch.cuda.Stream(device=local)
    with native.Reconstruction(device=local, stream=stream.cuda_stream) as r:
        r.load_scan(scan.pos, scan.intensity, scan.obj0, scan.probe0)
        r.iterate(1.0, 1.0, 1.0, 5)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.iterate(1.0, 1.0, 1.0, iters)
        e1.record(stream)
        e1.synchronize()
        t_gpu = e0.elapsed_time(e1) / 1e3
    return {"workload": f"tiny: J={scan.J}, N={scan.N}, DC, {iters} iterations",
            "oracle": {"value": scan.J * iters / t_cpu, "unit": UNIT, "cores": _cores()},
            "gpu": {"value": scan.J * iters / t_gpu, "unit": UNIT, "ms_per_iteration": t_gpu * 1e3 / iters}}


def _oracle_one_thread(scan, side: int, seconds: float):
    """The same oracle timing with one BLAS/OpenMP thread, in a child process
    (the thread count of numpy's BLAS is fixed when numpy loads)."""
    import numpy as np
    idx = _sub_scan(scan, side)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "sample.npz")
        np.savez(path, intensity=scan.intensity[idx], pos=scan.pos[idx], obj0=scan.obj0,
                 probe0=scan.probe0)
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = "1"
        code = ("import sys, json; sys.path.insert(0, %r); import bench; "
                "print(json.dumps(bench._oracle_sample_rate(%r, %r)))" % (ROOT, path, seconds))
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=600)
    if out.returncode != 0:
        return None
    return json.loads(out.stdout.strip().splitlines()[-1])


def _oracle_sample_rate(path: str, seconds: float):
    import numpy as np
    from oracle import ptycho as optycho
    d = np.load(path)
    prob = optycho.Problem(d["intensity"].astype(np.float64), d["pos"],
                           d["obj0"].astype(np.complex128), d["probe0"].astype(np.complex128))
    x = optycho.exit_waves(prob.P, prob.O, d["pos"])
    times = []
    t_all = time.perf_counter()
    while time.perf_counter() - t_all < seconds or not times:
        t0 = time.perf_counter()
        x = prob.iterate(x, *RAAR)
        times.append(time.perf_counter() - t0)
    return {"value": len(d["pos"]) * len(times) / sum(times), "iterations": len(times)}


def cufft_divide_ms(scan, c: float, device, reps: int = 10):
    """For comparison only (not the library's path): the same divide step as
    separate library calls (torch.fft, i.e. cuFFT, plus elementwise kernels)
    on the same workload -- forward 2-D FFT, modulus projection with the c
    relaxation, inverse 2-D FFT, and the Fourier-error sum -- and the two
    FFTs alone.  The fused kernel also forms x_k (the re-split), which these
    sequences leave out.  Returns (whole sequence ms, FFTs only ms)."""
    import torch
    J, N = scan.J, scan.N
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.complex(torch.randn(J, N, N, generator=g), torch.randn(J, N, N, generator=g)).to(device)
    sq = torch.from_numpy(scan.intensity).to(device).sqrt_()
    st = torch.cuda.Stream(device=device)

    def step():
        Psi = torch.fft.fft2(x)
        a = Psi.abs()
        err = ((a - sq) ** 2).sum(dtype=torch.float64)
        Psi2 = torch.where(a > 0, (c * sq / a + (1.0 - c)) * Psi, (c * sq).to(Psi.dtype))
        return torch.fft.ifft2(Psi2), err

    def ffts_only():
        return torch.fft.ifft2(torch.fft.fft2(x))

    out = []
    with torch.cuda.stream(st):
        for fn in (step, ffts_only):
            for _ in range(3):
                fn()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                fn()
            e1.record(st)
            e1.synchronize()
            out.append(e0.elapsed_time(e1) / reps)
    del x, sq
    torch.cuda.empty_cache()
    return out[0], out[1]


def _cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, spec):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2311_11466_gb300 import synth
    scan = synth.make_scan(spec)
    side = 4
    # warm-up steps, then K timed steps, each one oracle iteration of the sample
    # exactly W untimed and K timed iterations (no time bound)
    oracle_rate(scan, side, float("inf"), max(args.warmup, 0)) if args.warmup > 0 else None
    rate, n, npos = oracle_rate(scan, side, float("inf"), max(args.steps, 1))
    sample = (f"{npos} positions ({side}x{side} block of the 32x32 raster, 256^2 patterns, "
              f"full 1300^2 object), {n} RAAR iterations of the FP64 oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": npos / rate * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "large: J=1024, N=256, M=1300, RAAR(0.9), Poisson 1e6",
                   "sample": sample},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batch_mode(args):
    """16 uneven scans (N in {128, 256}, J log-uniform in [100, 2000], raster or
    Fermat, presets cycled DC, AR, DR, SF, RAAR, RRR) advanced together through
    one captured graph per round, against the same scans run one after another."""
    import torch
    from paper_2311_11466_gb300 import build as _build, native, serve, synth
    _build.build()
    specs = synth.batch_specs(16)
    scans = [synth.make_scan(sp) for sp in specs]
    names = ["DC", "AR", "DR", "SF", "RAAR", "RRR"]
    settings = [native.PRESETS[names[i % 6]] for i in range(len(scans))]
    n = args.steps
    units = sum(sc.J for sc in scans) * n

    def load():
        rs = []
        for sc in scans:
            r = native.Reconstruction()
            r.load_scan(sc.pos, sc.intensity, sc.obj0, sc.probe0)
            rs.append(r)
        return rs

    modes = {}
    tuning = None
    for name, mode in (("auto", serve.PTYCHO_BATCH_AUTO), ("groups", serve.PTYCHO_BATCH_GROUPS),
                       ("branches", serve.PTYCHO_BATCH_BRANCHES)):
        rs = load()
        serve.run_batch(rs, settings, args.warmup, mode=mode)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = serve.run_batch(rs, settings, n, mode=mode)
        modes[name] = dict(info, value=units / (time.perf_counter() - t0))
        if tuning is None:
            tuning = [r.tuning() for r in rs]
        for r in rs:
            r.close()
    t_batch = units / modes["auto"]["value"]
    rs = load()
    for r, abc in zip(rs, settings):
        r.iterate(*abc, args.warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r, abc in zip(rs, settings):
        r.iterate(*abc, n)
        r.object_probe()       # synchronises this scan before the next starts
    t_seq = time.perf_counter() - t0
    for r in rs:
        r.close()
    line = {"metric": "position-updates/s, 16 uneven scans", "mode": "batch", "value": units / t_batch,
            "unit": UNIT, "sequential": units / t_seq, "speedup": t_seq / t_batch, "steps": n,
            "warmup": args.warmup, "dtype": "f32", "data": "synthetic",
            "modes": modes,
            "config": {"scans": [{"J": sc.J, "N": sc.N, "M": list(sc.M_shape),
                                  "geometry": sc.spec.geometry,
                                  "gather_tile": list(t["gather_tile"]),
                                  "probe_pixels_per_thread": t["probe_pixels_per_thread"],
                                  "cluster_size": t["cluster_size"]}
                                 for sc, t in zip(scans, tuning)],
                       "settings": [names[i % 6] for i in range(len(scans))],
                       "tuner_measurements": {f"N={sc.N},J={sc.J}": {"gather_ms": t["gather_ms"],
                                                                    "probe_ms": t["probe_ms"],
                                                                    "divide128_ms": t["divide128_ms"]}
                                              for sc, t in zip(scans, tuning)}}}
    print(json.dumps(line), flush=True)
    return 0


def run_serve_mode(args):
    """Poisson arrivals of blind RAAR(0.9) reconstructions (N in {128, 256}, J
    log-uniform in [100, 4096] drawn from a pool of distinct synthetic scans),
    served with admission by HBM budget and interleaved rounds; p50/p99
    latency and aggregate throughput, against serving the same requests one
    after another."""
    import numpy as np
    from paper_2311_11466_gb300 import build as _build, native, serve, synth
    _build.build()
    pool_specs = synth.serving_specs(8)
    pool = [synth.make_scan(sp) for sp in pool_specs]
    rng = np.random.default_rng(4)
    pick = rng.integers(0, len(pool), size=args.requests)
    scans = [pool[i] for i in pick]
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=args.requests))
    arrivals -= arrivals[0]
    iters = args.e2e_iters
    settings = [native.PRESETS["RAAR"]] * len(scans)
    budget = 180 << 30
    # warm the kernels once
    serve.run_stream(scans[:1], settings[:1], 2, [0.0], budget, 1)
    recs, wall = serve.run_stream(scans, settings, iters, arrivals, budget, max_active=16,
                                  iters_per_round=10)
    lat = np.array([r["latency_s"] for r in recs])
    per100 = np.array([r["per100_s"] for r in recs])
    units = sum(sc.J for sc in scans) * iters
    # the same requests one at a time, back to back (no queueing model)
    t0 = time.perf_counter()
    for sc in scans:
        with native.Reconstruction() as r:
            r.load_scan(sc.pos, sc.intensity, sc.obj0, sc.probe0)
            r.iterate(*settings[0], iters)
            r.object_probe()
    t_seq = time.perf_counter() - t0
    line = {"metric": "serving: aggregate position-updates/s; p50/p99 latency", "mode": "serve",
            "value": units / wall, "unit": UNIT, "sequential": units / t_seq,
            "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
            "per100_p50_s": float(np.percentile(per100, 50)), "per100_p99_s": float(np.percentile(per100, 99)),
            "requests": len(scans), "rate_per_s": args.rate, "iterations": iters,
            "wall_s": wall, "dtype": "f32", "data": "synthetic",
            "config": {"pool": [{"J": sc.J, "N": sc.N} for sc in pool], "max_active": 16,
                       "iters_per_round": 10, "budget_gb": 180}}
    print(json.dumps(line), flush=True)
    return 0


def run_compare_mode(args):
    """The shape of the paper's comparison (Figs. 6-8): every (a, b, c) setting,
    a big and a small probe on the same synthetic object and scan, under two
    readings of when the probe update starts (from the first iteration; after
    `--probe-start` iterations with the probe held), with the Fourier error
    curve every 10 iterations and the final ambiguity-corrected object error."""
    from paper_2311_11466_gb300 import build as _build, metrics, native, synth
    _build.build()
    iters = args.e2e_iters
    out = {}
    for start in (0, args.probe_start):
        for label, radius in (("big", 32.0), ("small", 16.0)):
            spec = synth.ScanSpec(N=128, ny=12, nx=12, step=16, jitter=2, radius=radius,
                                  defocus=0.02 * (16.0 / radius) ** 2, photons=1e6, seed=6)
            scan = synth.make_scan(spec)
            rows = {}
            for name in ["DC", "AR", "DR", "SF", "RAAR", "RRR"]:
                with native.Reconstruction() as r:
                    r.set_probe_start(start)
                    r.load_scan(scan.pos, scan.intensity, scan.obj0, scan.probe0)
                    r.iterate(*native.PRESETS[name], iters)
                    e = r.errors()
                    O, _ = r.object_probe()
                    rows[name] = {"E_F_curve_every_10": [float(e[k]) for k in range(0, iters, 10)] +
                                                        [float(e[-1])],
                                  "model_E_F": r.model_error(),
                                  "object_error": metrics.object_error(O, scan.obj_true, scan.N)}
            out[f"probe_start_{start}/{label}"] = {"probe_start": start, "probe_radius": radius,
                                                   "J": scan.J, "N": scan.N,
                                                   "M": list(scan.M_shape), "results": rows}
    line = {"metric": "error after iterations, every preset, big vs small probe, two probe-start readings",
            "mode": "compare", "iterations": iters, "data": "synthetic", "dtype": "f32",
            "results": out}
    print(json.dumps(line), flush=True)
    return 0


def measure_iterate(spec, precision: str, preset: str, steps: int, warmup: int, e2e_iters: int,
                    local: int, ws: int, rank: int, concur: str = "deterministic",
                    fp32_compare: bool = False, divide: str = "auto", scan=None,
                    with_e2e: bool = True, shapes=None):
    """Time `steps` abc iterations of one scan on this rank's GPU (CUDA events on
    the library's stream, after `warmup` iterations), the dominant kernel's
    roofline, the clocks during the timed region, and one end-to-end
    reconstruction through the C ABI from pinned host buffers.  `shapes`
    (gather rows, gather columns, probe pixels per thread[, cluster size])
    pins the launch shapes instead of tuning them.  Returns a dict (the `scan`
    entry is the synthetic scan itself)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2311_11466_gb300 import native, synth

    if scan is None:
        scan = synth.make_scan(spec)
    J, N = scan.J, scan.N
    # one dedicated stream for the library and for the timing events
    stream = torch.cuda.Stream(device=local)
    r = native.Reconstruction(device=local, stream=stream.cuda_stream, precision=precision,
                              concur=concur, divide=divide)
    if shapes:
        r.set_tuning(False)
    r.load_scan(scan.pos, scan.intensity, scan.obj0, scan.probe0)
    if shapes:
        r.set_launch_shapes(*shapes)
    design = r.divide_design()
    tuning = None
    abc = native.PRESETS[preset]
    r.iterate(*abc, warmup)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    fine = NvmlClockSampler(local)
    if rank == 0:
        sampler.start()
        fine.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    native.ptycho_profile_enable(r.h, True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    r.iterate(*abc, steps)
    t1.record(stream)
    t1.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    clocks = None
    if rank == 0:
        coarse = sampler.stop()
        fine_rec = fine.stop()
        # the 1 ms NVML record when there is one; the nvidia-smi record beside it
        clocks = dict(fine_rec, nvidia_smi=coarse) if fine_rec else coarse
    native.ptycho_profile_enable(r.h, False)
    div_ms, con_ms, nrec = native.ptycho_profile_read(r.h)
    tuning = r.tuning()
    ms = max_over_ranks(ms, torch.device("cuda", local))
    value = replica_throughput(J * steps, ws, ms / 1e3)

    # roofline of the dominant kernel (the divide step)
    NN = N * N
    # algorithmic bytes per pixel of the divide kernel: sqrt I (4) and y_k (8)
    # always; y_{k-1} (8) when b != 1; x_{k-1} read and x_k written (8 + 8) when a != 1
    a_, b_, _ = abc
    div_px = 12.0 + (8.0 if b_ != 1.0 else 0.0) + (16.0 if a_ != 1.0 else 0.0)
    div_bytes = div_px * J * NN
    div_avg = div_ms / max(nrec, 1) / 1e3
    if precision == "bf16x3":
        flops = 96.0 * N ** 3 * J   # four GEMMs of 2 x N x 2N x 6N per exit wave
        tflops, tkind = _bf16_peak()
        roof = {"bound": "tensor", "achieved": flops / div_avg / 1e12, "peak": tflops,
                "unit": "TFLOP/s", "frac": flops / div_avg / 1e12 / tflops, "traffic": None,
                "kernel": "divide on tensor cores (prologue + 4 BF16x3 DFT GEMMs, tcgen05)",
                "algorithmic_flops_per_launch": flops, "avg_launch_ms": div_avg * 1e3,
                "peak_source": tkind}
    else:
        hbm, peak_kind = _peaks()
        achieved = div_bytes / div_avg / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": _profiled_traffic(N, J, design),
                "kernel": f"divide, {design} design (fused re-split + FFT + modulus + IFFT)",
                "algorithmic_bytes_per_launch": div_bytes,
                "avg_launch_ms": div_avg * 1e3, "peak_source": peak_kind}

    if not with_e2e:
        r.close()
        del stream
        return {"scan": scan, "value": value, "ms": ms, "abc": abc, "div_px": div_px,
                "roofline": roof, "design": design, "clocks": clocks,
                "kernel_ms_per_step": {"divide": div_ms / max(nrec, 1),
                                       "concur": con_ms / max(nrec, 1)}}

    # end to end through the public API with host buffers (pinned)
    def pin(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    I_h, pos_h = pin(scan.intensity), pin(scan.pos)
    O_h, P_h = pin(scan.obj0), pin(scan.probe0)
    O_out = pin(np.empty(scan.M_shape, dtype=np.complex64))
    P_out = pin(np.empty((N, N), dtype=np.complex64))
    e2e_iters = max(e2e_iters, 1)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    w0 = time.perf_counter()
    re2e = native.Reconstruction(device=local, stream=stream.cuda_stream, precision=precision,
                                 concur=concur, divide=divide)
    re2e.load_scan(pos_h, I_h, O_h, P_h)
    re2e.iterate(*abc, e2e_iters)
    native.ptycho_get_object_probe(re2e.h, O_out, P_out)
    errs = re2e.errors()
    w1 = time.perf_counter()
    e2e_s = max_over_ranks(w1 - w0, torch.device("cuda", local))
    final_model_err = re2e.model_error()
    re2e.close()
    h2d = I_h.nbytes + pos_h.nbytes + O_h.nbytes + P_h.nbytes
    d2h = O_out.nbytes + P_out.nbytes + errs.nbytes
    e2e = {"value": replica_throughput(J * e2e_iters, ws, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": h2d / e2e_iters, "d2h_bytes_per_step": d2h / e2e_iters,
           "step": f"one reconstruction = load_scan (host, pinned) + {e2e_iters} {preset} iterations "
                   f"+ object/probe/error read-back; bytes per iteration",
           "final_fourier_error": final_model_err,
           "fourier_error_iter1": float(errs[0]), f"fourier_error_iter{len(errs)}": float(errs[-1])}
    if fp32_compare and rank == 0:
        # the FP32 path on the same scan and iteration count, for the error comparison
        with native.Reconstruction(device=local, stream=stream.cuda_stream) as r32:
            r32.load_scan(scan.pos, scan.intensity, scan.obj0, scan.probe0)
            r32.iterate(*abc, e2e_iters)
            e32 = r32.errors()
            m32 = r32.model_error()
        e2e["fp32_same_scan"] = {"fourier_error_iter1": float(e32[0]),
                                 f"fourier_error_iter{len(e32)}": float(e32[-1]),
                                 "final_fourier_error": m32}
        e2e["rel_diff_vs_fp32"] = {
            "iter1": abs(float(errs[0]) - float(e32[0])) / float(e32[0]),
            f"iter{len(e32)}": abs(float(errs[-1]) - float(e32[-1])) / float(e32[-1]),
            "final_model": abs(final_model_err - m32) / m32}
    r.close()
    del stream
    return {"scan": scan, "value": value, "ms": ms, "abc": abc, "div_px": div_px, "roofline": roof,
            "kernel_ms_per_step": {"divide": div_ms / max(nrec, 1), "concur": con_ms / max(nrec, 1)},
            "clocks": clocks, "e2e": e2e, "design": design, "tuning": tuning}


def measure_sp(passes: int = 3):
    """Sequential projections (Fig. 2): passes over the 256 positions of the
    medium workload (256^2 patterns), one divide-kernel launch (one cluster) per
    position in scan order, timed with CUDA events on the library's stream
    after one untimed pass.  The steps depend on each other (each updates the
    object and the probe the next one reads), so only one cluster works at a
    time: this is the sequential algorithm the product-space update is
    contrasted with, not a tuned path."""
    import torch
    from paper_2311_11466_gb300 import native, synth
    scan = synth.make_scan(synth.named_spec("medium"))
    stream = torch.cuda.Stream()
    with native.Reconstruction(stream=stream.cuda_stream) as r:
        r.load_scan(scan.pos, scan.intensity, scan.obj0, scan.probe0)
        r.sp_iterate(1.0, 1)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        r.sp_iterate(1.0, passes)
        t1.record(stream)
        t1.synchronize()
        ms = t0.elapsed_time(t1)
    return {"value": scan.J * passes / (ms / 1e3), "unit": UNIT, "passes": passes,
            "ms_per_pass": ms / passes, "us_per_step": ms * 1e3 / (scan.J * passes),
            "workload": f"medium: J={scan.J}, N={scan.N}, lambda=1, scan order",
            "timed_launches": scan.J * passes}


def measure_serving(requests: int, rate: float, iters: int, max_active: int = 16,
                    iters_per_round: int = 10, budget_gb: int = 180):
    """The serving workload: `requests` blind RAAR(0.9) reconstructions drawn
    from a pool of 8 synthetic scans (N in {128, 256}, J log-uniform in
    [100, 4096]), each `iters` iterations.  Four runs of the same requests:
      saturation: every request submitted at t = 0; continuous batching
        (max_active in flight) against the same requests back to back, one
        reconstruction at a time through the context API;
      at `rate` req/s (Poisson arrivals): continuous batching against the same
        server admitting one request at a time (sequential FIFO service).
    Latency is submission to completion (host wall time, queueing included);
    per-100 is the service time per 100 iterations.  Each request's final model
    Fourier error is kept, so equal final error can be checked."""
    import numpy as np
    from paper_2311_11466_gb300 import native, serve, synth
    pool = [synth.make_scan(sp) for sp in synth.serving_specs(8)]
    rng = np.random.default_rng(4)
    pick = rng.integers(0, len(pool), size=requests)
    scans = [pool[i] for i in pick]
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=requests))
    arrivals -= arrivals[0]
    settings = [native.PRESETS["RAAR"]] * len(scans)
    budget = budget_gb << 30
    units = sum(sc.J for sc in scans) * iters
    serve.run_stream(scans[:2], settings[:2], 2, [0.0, 0.0], budget, 2)  # warm the kernels

    def summarise(recs, wall):
        lat = np.array([r_["latency_s"] for r_ in recs])
        per100 = np.array([r_["per100_s"] for r_ in recs])
        return {"value": units / wall, "wall_s": wall,
                "latency_p50_s": float(np.percentile(lat, 50)),
                "latency_p99_s": float(np.percentile(lat, 99)),
                "per100_p50_s": float(np.percentile(per100, 50)),
                "per100_p99_s": float(np.percentile(per100, 99))}, \
            np.array([r_["final_error"] for r_ in recs])

    zero = np.zeros(len(scans))
    sat, fe_sat = summarise(*serve.run_stream(scans, settings, iters, zero, budget, max_active,
                                              iters_per_round))
    # the same requests back to back, one reconstruction at a time
    fe_seq = np.empty(len(scans))
    t0 = time.perf_counter()
    for i, sc in enumerate(scans):
        with native.Reconstruction() as r:
            r.load_scan(sc.pos, sc.intensity, sc.obj0, sc.probe0)
            r.iterate(*settings[i], iters)
            r.object_probe()
            fe_seq[i] = r.model_error()
    t_seq = time.perf_counter() - t0
    at_rate, fe_rate = summarise(*serve.run_stream(scans, settings, iters, arrivals, budget,
                                                   max_active, iters_per_round))
    fifo, fe_fifo = summarise(*serve.run_stream(scans, settings, iters, arrivals, budget, 1,
                                                iters_per_round))

    def rel(a, b):
        return float(np.max(np.abs(a - b) / np.abs(b)))

    return {
        "metric": "aggregate position-updates/s; p50/p99 latency (s), queueing included",
        "unit": UNIT, "requests": len(scans), "iterations": iters, "preset": "RAAR(0.9)",
        "pool": [{"J": sc.J, "N": sc.N, "geometry": sc.spec.geometry} for sc in pool],
        "max_active": max_active, "iters_per_round": iters_per_round, "budget_gb": budget_gb,
        "saturation": {"continuous_batching": sat,
                       "back_to_back": {"value": units / t_seq, "wall_s": t_seq},
                       "speedup": sat["value"] / (units / t_seq)},
        f"at_{rate:g}_req_per_s": {"continuous_batching": at_rate, "sequential_fifo": fifo,
                                   "speedup": at_rate["value"] / fifo["value"]},
        "final_model_error": {"mean": float(fe_seq.mean()), "max": float(fe_seq.max()),
                              "max_rel_diff_vs_back_to_back": {
                                  "saturation": rel(fe_sat, fe_seq), "at_rate": rel(fe_rate, fe_seq),
                                  "sequential_fifo": rel(fe_fifo, fe_seq)}},
        "data": "synthetic", "dtype": "f32",
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "precision", "medium", "tiny", "large128"])
    ap.add_argument("--e2e-iters", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the cuFFT comparison timing")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the tensor-core (bf16x3) and serving sub-results of the default line")
    ap.add_argument("--mode", default="iterate", choices=["iterate", "batch", "serve", "compare"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16x3"])
    ap.add_argument("--preset", default="RAAR", choices=["DC", "AR", "DR", "SF", "RAAR", "RRR"])
    ap.add_argument("--concur", default="deterministic", choices=["deterministic", "atomic"])
    ap.add_argument("--divide", default="auto", choices=["auto", "cluster", "twopass"])
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--probe-start", type=int, default=10,
                    help="compare mode: the second reading holds the probe for this many iterations")
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--launch-shapes", default=None,
                    type=lambda v: tuple(int(t) for t in v.split(",")),
                    help="pin the launch shapes (gather rows,cols,probe pixels per thread[,cluster size]) "
                         "instead of tuning them, e.g. for a profile of one kernel instance")
    args = ap.parse_args()
    if args.mode == "batch":
        return run_batch_mode(args)
    if args.mode == "serve":
        return run_serve_mode(args)
    if args.mode == "compare":
        return run_compare_mode(args)

    from paper_2311_11466_gb300 import synth
    if args.precision == "bf16x3" and args.workload == "large":
        args.workload = "precision"
    spec = synth.named_spec(args.workload)
    if args.impl == "reference":
        return run_reference(args, spec)

    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2311_11466_gb300 import build as _build, native
    if rank == 0:
        _build.build()
    if ws > 1:
        dist.barrier()
    native.lib()

    m = measure_iterate(spec, args.precision, args.preset, args.steps, args.warmup, args.e2e_iters,
                        local, ws, rank, concur=args.concur,
                        fp32_compare=args.precision == "bf16x3", divide=args.divide,
                        shapes=args.launch_shapes)
    scan, value, ms, abc = m["scan"], m["value"], m["ms"], m["abc"]
    J, N = scan.J, scan.N
    NN = N * N

    unfused = None
    if rank == 0 and args.precision == "fp32" and not args.no_compare:
        cm, fft_ms = cufft_divide_ms(scan, abc[2], torch.device("cuda", local))
        div_ms = m["roofline"]["avg_launch_ms"]
        unfused = {"divide_ms": cm, "fft2_ifft2_only_ms": fft_ms, "fused_divide_ms": div_ms,
                   "speedup": cm / div_ms,
                   "kind": "comparison only: torch.fft (cuFFT) fft2 + modulus + ifft2 + error sum "
                           "on the same workload; the fused kernel also forms x_k"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, n, npos = oracle_rate(scan, 4, args.cpu_seconds, 1000)
        cpu = {"value": rate, "unit": UNIT, "cores": _cores(), "kind": "oracle",
               "sample": f"{npos} positions (4x4 block of the raster, 256^2 patterns, full object), "
                         f"{n} RAAR iterations of the FP64 oracle"}
        one = _oracle_one_thread(scan, 4, min(args.cpu_seconds, 6.0))
        if one is not None:
            cpu["one_thread"] = {"value": one["value"], "unit": UNIT, "cores": 1,
                                 "sample": f"same sample, {one['iterations']} iterations, "
                                           f"one BLAS thread"}
        cpu["tiny_in_full"] = tiny_both(local)
    # both divide designs at 256^2 on the same scan (the default line uses the
    # one AUTO picks; this races the two)
    variants = None
    if ws == 1 and not args.no_extras and args.precision == "fp32" and N == 256:
        variants = {"default": m["design"]}
        for design in ("cluster", "twopass"):
            v = measure_iterate(spec, "fp32", args.preset, 20, 3, 0, local, ws, rank,
                                divide=design, scan=scan, with_e2e=False)
            variants[design] = {"value": v["value"], "ms_per_step": v["ms"] / 20,
                                "divide_ms": v["roofline"]["avg_launch_ms"],
                                "divide_hbm_frac": v["roofline"]["frac"],
                                "divide_gbs": v["roofline"]["achieved"],
                                "traffic": v["roofline"]["traffic"], "steps": 20, "warmup": 3,
                                "clocks": v["clocks"]}
    # the atomic concur mode (shared-memory-staged object atomics, register-
    # staged probe atomics) against the deterministic gather, same scan
    concur_modes = None
    if (ws == 1 and not args.no_extras and args.precision == "fp32" and N == 256
            and args.concur == "deterministic"):
        a = measure_iterate(spec, "fp32", args.preset, 20, 3, 0, local, ws, rank,
                            concur="atomic", scan=scan, with_e2e=False)
        concur_modes = {
            "deterministic": {"concur_ms": m["kernel_ms_per_step"]["concur"], "value": value},
            "atomic": {"concur_ms": a["kernel_ms_per_step"]["concur"], "value": a["value"],
                       "ms_per_step": a["ms"] / 20, "steps": 20, "warmup": 3,
                       "clocks": a["clocks"]},
            "note": "concur_ms: object + probe halves of the concur step per iteration (CUDA "
                    "events); the atomic mode is not bitwise reproducible"}
    del scan, m["scan"]
    extra_launches = 2 * KERNELS_PER_ITER * 20 if variants is not None else 0
    if concur_modes is not None:
        extra_launches += (KERNELS_PER_ITER + 2) * 20
    if cpu and cpu.get("tiny_in_full"):
        extra_launches += KERNELS_PER_ITER * 100

    # the rest of the metric (tensor-core path; serving) on a single GPU only
    extras = {}
    if ws == 1 and not args.no_extras and args.precision == "fp32" and args.workload == "large":
        steps_tc = 20
        t = measure_iterate(synth.named_spec("precision"), "bf16x3", "RAAR", steps_tc, 3, 200,
                            local, ws, rank, fp32_compare=True)
        extras["bf16x3"] = {
            "value": t["value"], "unit": UNIT, "steps": steps_tc, "warmup": 3,
            "ms_per_step": t["ms"] / steps_tc,
            "config": {"workload": f"precision: J={t['scan'].J}, N={t['scan'].N}, "
                                   f"M={t['scan'].M_shape[0]}x{t['scan'].M_shape[1]}, RAAR(0.9), "
                                   "BF16x3 tensor-core DFT, FP32 accumulation"},
            "roofline": t["roofline"], "kernel_ms_per_step": t["kernel_ms_per_step"],
            "clocks": t["clocks"], "e2e": t["e2e"],
            "errors": {"note": "E_F of the tensor-core path and of the FP32 path on the same scan "
                               "from the same start, at iterations 1 and 200, and the final model "
                               "error; rel_diff_vs_fp32 gives their relative differences",
                       **{k: v for k, v in t["e2e"].items() if k.startswith(("fourier", "final", "fp32", "rel"))}},
        }
        extra_launches += (KERNELS_PER_ITER + 4) * steps_tc
        del t
        torch.cuda.empty_cache()
        extras["serving"] = measure_serving(args.requests, args.rate, args.e2e_iters)
        extras["sequential_projections"] = measure_sp()
        extra_launches += extras["sequential_projections"]["timed_launches"]

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "bf16x3 (f32 accumulate)", "data": "synthetic",
            "config": {"workload": f"{args.workload}: J={J}, N={N}, "
                                   f"{args.preset} (a,b,c)={tuple(abc)}, {args.precision}, Poisson {spec.photons}",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": "working set > L2 (no flush needed)"},
            "roofline": m["roofline"],
            "kernel_ms_per_step": m["kernel_ms_per_step"],
            "launch_shapes": m["tuning"],
            # the survey's FFT rate: 10 N^2 log2(N^2) flops per position-update (a
            # forward and an inverse 2-D FFT at 5 N^2 log2(N^2) each), against the
            # nominal FP32 CUDA-core peak (152 SMs x 128 lanes x 2 flops x 2.07 GHz)
            "fft_rate": {"tflops": value * 10.0 * NN * math.log2(NN) / 1e12,
                         "flops_per_update": 10.0 * NN * math.log2(NN),
                         "of_fp32_nominal_peak": value * 10.0 * NN * math.log2(NN) / 1e12 / FP32_NOMINAL_TFLOPS,
                         "peak_source": "nominal (not measured)"},
            "per_step_bytes": (m["div_px"] + 16.0) * J * NN,
            "step_hbm_gbs": (m["div_px"] + 16.0) * J * NN / (ms / args.steps / 1e3) / 1e9,
            # the atomic concur mode adds two launches (the maxima of the
            # atomically built denominators) and the tensor-core path four
            "gpu_launches": (KERNELS_PER_ITER + (4 if args.precision == "bf16x3" else 0)
                             + (2 if args.concur == "atomic" else 0)) * args.steps,
            "clocks": m["clocks"],
            "e2e": m["e2e"],
            "cpu_baseline": cpu,
        }
        if unfused is not None:
            line["unfused_cufft"] = unfused
        if variants is not None:
            line["divide_variants"] = variants
        if concur_modes is not None:
            line["concur_modes"] = concur_modes
        if extra_launches:
            line["extra_timed_launches"] = extra_launches
        line.update(extras)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
