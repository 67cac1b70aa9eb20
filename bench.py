#!/usr/bin/env python3
"""Benchmark of the Gauss-Legendre SHT round trip on GB300.

One step = one scalar round trip (synthesis then analysis, each with its
Legendre stage and longitude FFT) over a batch of seeded synthetic fields at
N = 1023 (nlat = 1024, nphi = 2048), batch 16, inputs resident in HBM.  The
metric is round trips per second (fields x steps / time), with nominal
GFLOP/s; the plain FP64 path is timed on the same workload for the ratio.

The headline path (default --mode tc_f64) is the batched tensor-core form at
the paper's FP64 accuracy (digit-sliced contraction, double-float FFTs).  The
same line carries, as first-class secondary results, the split-bf16
tensor-core path (key "bf16x3"), the plain FP64 and FP32 paths, the other
workloads of the study (N = 511, the vector transform, the uneven batch, the
differentiable form, high N, the polar threshold sweep, accuracy versus N), and
the FP64 CPU oracle on the host cores (cpu_baseline), which after its timing
also measures the errors of sampled GPU outputs of each workload against the
oracle ("eps_vs_oracle" of each entry).

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas
(each rank transforms its own batch, no collective): weak scaling.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode tc_f64|tc|otf|f32|f64|auto]
                  [--impl ours|reference] [--no-extras] [--no-cpu-baseline]
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LMAX, NLAT, NPHI, BATCH = 1023, 1024, 2048, 16
WORKLOAD = f"scalar SHT round trip N={LMAX} nlat={NLAT} nphi={NPHI} batch={BATCH}"
METRIC = "SHT round-trips/s (N=1023, batch 16)"
UNIT = "round-trips/s"
E2E_MIN_SECONDS = 1.0


def bench_config(world):
    """The workload, identical for this implementation's arm and the reference arm."""
    return {"workload": WORKLOAD, "lmax": LMAX, "nlat": NLAT, "nphi": NPHI, "batch": BATCH,
            "l2": "inputs larger than L2 (spectra + grids > 129 MB), no flush needed",
            "parallelism": f"replicas x{world}"}


def nlm_of(lmax, mmax=None):
    mmax = lmax if mmax is None else mmax
    return (mmax + 1) * (lmax + 1) - mmax * (mmax + 1) // 2


def nominal_flops_per_rt(lmax=LMAX, nlat=NLAT, nphi=NPHI):
    """Nominal flop count of one round trip of one field: per direction
    4 flops per (mode, latitude) plus 2.5 nphi log2(nphi) per FFT row."""
    per_dir = 4.0 * nlm_of(lmax) * nlat + 2.5 * nphi * math.log2(nphi) * nlat
    return 2.0 * per_dir


def legendre_flops_per_launch(batch, lmax=LMAX, nlat=NLAT):
    """Algorithmic flops of one Legendre launch on `batch` fields: per
    (mode, latitude pair) the recurrence (2 mul + 1 fma = 4 flops, shared by
    the batch) plus one complex x real accumulate per field (4 flops), before
    the polar optimisation's skip."""
    npairs = (nlat + 1) // 2
    return nlm_of(lmax) * npairs * (4.0 + 4.0 * batch)


def tc64_algorithmic_bytes(batch, lmax=LMAX, nlat=NLAT, zero_skip=0.0):
    """Bytes one FP64-accurate tensor-core Legendre stage must move: 7 bf16
    digit slices (14 B) of every P_n^m(x_j) of one hemisphere, less the
    all-zero 8-row groups it skips, plus the FP64 spectra and the FP64 E/O (or s/d)
    intermediate of the batch (the digit data the stage writes and reads
    back, and the tile padding, are not counted)."""
    npairs = (nlat + 1) // 2
    panel = nlm_of(lmax) * npairs * 14 * (1.0 - zero_skip)
    spec = batch * nlm_of(lmax) * 16
    inter = batch * (lmax + 1) * npairs * 32
    return panel + spec + inter


def tc_algorithmic_bytes(batch, lmax=LMAX, nlat=NLAT, polar_skip=0.0):
    """Bytes one tensor-core Legendre launch must move: every P_n^m(x_j) of one
    hemisphere as a bf16 hi+lo pair (4 B; the library's tile padding is not
    counted) less the share the polar optimisation of Sec. 3.1 leaves out,
    the FP32 spectra of the batch and the FP32 E/O (or s/d) intermediate of
    the batch."""
    npairs = (nlat + 1) // 2
    panel = nlm_of(lmax) * npairs * 4 * (1.0 - polar_skip)
    spec = batch * nlm_of(lmax) * 8
    inter = batch * (lmax + 1) * npairs * 16
    return panel + spec + inter


def fft_algorithmic_bytes(batch, lmax=LMAX, nlat=NLAT, nphi=NPHI, elem=4):
    """Bytes one longitude-FFT launch must move: the grid and the E/O (or s/d)
    intermediate of the batch, each read or written once."""
    npairs = (nlat + 1) // 2
    return batch * (nlat * nphi * elem + (lmax + 1) * npairs * 4 * elem)


def fp32_alu_peak(sm_mhz):
    """FP32 FMA peak: 152 SMs x 128 FP32 lanes x 2 flops x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6


FP64_PEAK_NOMINAL = 1.25e12  # GB300 FP64 rate (nominal table of the pool)


# ---------------------------------------------------------------------------
# DRAM traffic of a kernel, from a committed ncu summary under profiles/: the
# summary names the kernel's source file and its SHA-256 at capture time; the
# figure is reported only while the source file is unchanged, else null.
def profiled_traffic(kernel):
    prof = os.path.join(ROOT, "profiles")
    try:
        names = sorted(os.listdir(prof))
    except OSError:
        return None
    for name in names:
        if not name.endswith(".md"):
            continue
        with open(os.path.join(prof, name)) as fh:
            text = fh.read()
        for m in re.finditer(r"^traffic: kernel=(\S+) source=(\S+) sha256=([0-9a-f]{64}) bytes_per_launch=([0-9.e+]+)",
                             text, re.M):
            if m.group(1) != kernel:
                continue
            try:
                with open(os.path.join(ROOT, m.group(2)), "rb") as sf:
                    if hashlib.sha256(sf.read()).hexdigest() != m.group(3):
                        return None
            except OSError:
                return None
            return float(m.group(4))
    return None


# ---------------------------------------------------------------------------
def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return json.load(fh)
    except Exception:
        return {}


class ClockSampler:
    """SM clock and clock-event reasons during a timed region.  A background
    thread reads them through NVML (libnvidia-ml, part of the driver) every
    2 ms; where NVML cannot be loaded, nvidia-smi samples every 100 ms."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    SMI_FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                  "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None, period=0.002):
        self.uuid = uuid
        self.period = period
        self.samples = []
        self.smax = None
        self._stop = threading.Event()
        self._thread = None
        self._proc = None
        self._path = None
        self._nvml = None
        self._dev = None

    def _nvml_open(self):
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        dev = ctypes.c_void_p()
        if not self.uuid or lib.nvmlDeviceGetHandleByUUID(self.uuid.encode(), ctypes.byref(dev)) != 0:
            raise RuntimeError("no NVML handle for the device")
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(dev, 1, ctypes.byref(mx)) == 0:
            self.smax = float(mx.value)
        self._nvml, self._dev = lib, dev

    def _loop(self):
        lib, dev = self._nvml, self._dev
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(dev, 1, ctypes.byref(clk)) == 0 and reasons_fn(dev, ctypes.byref(rs)) == 0:
                self.samples.append((float(clk.value), int(rs.value)))
            time.sleep(self.period)

    def start(self):
        try:
            self._nvml_open()
            self._thread = threading.Thread(target=self._loop, daemon=True)
            self._thread.start()
            return
        except Exception:
            self._nvml = None
        try:
            fd, self._path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.SMI_FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self._proc = subprocess.Popen(cmd, stdout=open(self._path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self._proc = None

    def stop(self):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(timeout=5)
            sm = [c for c, _ in self.samples]
            reasons = sorted({name for _, r in self.samples for bit, name in self.REASONS.items() if r & bit})
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.smax,
                    "samples": len(sm), "source": "NVML every 2 ms", "reasons": reasons}
        if self._proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "samples": 0, "reasons": ["no clock source"]}
        self._proc.terminate()
        try:
            self._proc.wait(timeout=5)
        except Exception:
            self._proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self._path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[4:8]):
                    if v.lower() == "active":
                        reasons.add(name)
        os.unlink(self._path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "source": "nvidia-smi every 100 ms", "reasons": sorted(reasons)}


def job_throughput(ms_local, world, units_per_rank, device=None):
    """Whole-job throughput of `world` replicas: the slowest rank's time (max
    over ranks of the local ms) for all ranks' units.  Returns (ms, units/s)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * units_per_rank / (ms / 1e3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def eps_measures(got, ref):
    """max |got - ref|, rms |got - ref| (Sec. 3.5 measures over the given
    entries) and max |got - ref| / max |ref| (normwise)."""
    import numpy as np
    d = np.abs(np.asarray(got, dtype=np.complex128) - np.asarray(ref, dtype=np.complex128))
    scale = float(np.abs(ref).max()) or 1.0
    return {"eps_max": float(d.max()), "eps_rms": float(np.sqrt(np.mean(d * d))), "normwise": float(d.max()) / scale}


# ---------------------------------------------------------------------------
# CPU baseline and the oracle checks of sampled GPU outputs
# ---------------------------------------------------------------------------
def cpu_baseline():
    """The oracle as it stands, one field round trip at the bench size, on all host cores."""
    import numpy as np

    import oracle
    from paper_1202_6522_gb300 import synthetic
    oracle.build()
    a = synthetic.spectrum(LMAX, seed=0)
    t0 = time.perf_counter()
    g = oracle.synth(LMAX, LMAX, NLAT, NPHI, a)
    r = oracle.analys(LMAX, LMAX, NLAT, NPHI, g)
    dt = time.perf_counter() - t0
    assert np.isfinite(r).all()
    return {"value": 1.0 / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"1 field round trip at N={LMAX} ({dt:.1f} s, direct Fourier sums)"}


def oracle_checks(samples):
    """Errors of sampled GPU outputs against the oracle (run in the CPU
    baseline leg, after every GPU timing).  Each sample names the transform,
    its sizes, the input and the GPU output on a subset of rows or orders."""
    import numpy as np

    import oracle
    out = {}
    for key, s in samples.items():
        kind = s["kind"]
        L, M, nl, nph = s["lmax"], s.get("mmax", s["lmax"]), s["nlat"], s["nphi"]
        if kind == "synth":
            ref = oracle.synth(L, M, nl, nph, s["input"], rows=s["rows"])[s["rows"]]
        elif kind == "analys":
            ref = oracle.analys(L, M, nl, nph, s["input"], ms=s["ms"])[s["idx"]]
        elif kind == "synth_vec":
            rt, rp = oracle.synth_vec(L, M, nl, nph, s["input"][0], s["input"][1], rows=s["rows"])
            ref = np.concatenate([rt[s["rows"]].ravel(), rp[s["rows"]].ravel()])
        elif kind == "analys_vec":
            rS, rT = oracle.analys_vec(L, M, nl, nph, s["input"][0], s["input"][1], ms=s["ms"])
            ref = np.concatenate([rS[s["idx"]], rT[s["idx"]]])
        elif kind == "loss_grad":
            resid = oracle.synth(L, M, nl, nph, s["input"][0]) - s["input"][1]
            ref = 2.0 * oracle.synth_adj(L, M, nl, nph, resid, ms=s["ms"])[s["idx"]]
        else:
            continue
        e = eps_measures(np.asarray(s["got"]).ravel(), np.asarray(ref).ravel())
        e["sample"] = s["what"]
        out[key] = e
    return out


def oracle_sample_step(oracle, a, stride):
    """One bounded sample of a field round trip: synthesis of every stride-th
    latitude row and analysis of every stride-th order m.  Each synthesis row
    costs the same; the orders 0, stride, 2 stride, .. carry about 1/stride of
    the analysis work, so stride x the sample's time estimates one round trip."""
    rows = list(range(0, NLAT, stride)) if stride > 1 else None
    ms = list(range(0, LMAX + 1, stride)) if stride > 1 else None
    g = oracle.synth(LMAX, LMAX, NLAT, NPHI, a, rows=rows)   # rows outside the sample are 0
    r = oracle.analys(LMAX, LMAX, NLAT, NPHI, g, ms=ms)
    return r


def run_reference(args):
    """The oracle, as it stands, on the host cores: each step is a bounded sample
    of one field's round trip at the bench size, scaled to round trips."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    import numpy as np
    from paper_1202_6522_gb300 import synthetic
    a = synthetic.spectrum(LMAX, seed=0)
    # size the sample so that warm-up + timed steps take about two minutes
    # (stride <= 8: coarser samples overstate the time through per-call overheads)
    t0 = time.perf_counter()
    oracle_sample_step(oracle, a, 8)
    t_full = 8 * (time.perf_counter() - t0)
    budget = 120.0
    stride = 1
    while stride < 8 and (args.steps + args.warmup) * t_full / stride > budget:
        stride *= 2
    for _ in range(args.warmup):
        oracle_sample_step(oracle, a, stride)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = oracle_sample_step(oracle, a, stride)
    dt = time.perf_counter() - t0
    assert np.isfinite(r).all()
    # each oracle call first computes the Gauss nodes and weights, a fixed cost
    # that a full round trip pays once per call, not stride times
    t_fixed = []
    for _ in range(3):
        t1 = time.perf_counter()
        oracle.gauss(NLAT)
        t_fixed.append(time.perf_counter() - t1)
    t_fixed = 2 * statistics.median(t_fixed)
    t_rt = stride * max(dt / args.steps - t_fixed, 0.0) + t_fixed
    value = 1.0 / t_rt
    sample = (f"per step: synthesis of every {stride}-th of {NLAT} rows and analysis of every "
              f"{stride}-th order of 1 field at N={LMAX}; round trip = {stride} x (step - quadrature "
              f"setup {1e3 * t_fixed:.0f} ms) + setup")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded N(0,1)/(n+1) spectra)",
        "config": bench_config(world),
        "path": "FP64 CPU oracle (direct Legendre and Fourier sums, OpenMP over orders)",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# timed paths
# ---------------------------------------------------------------------------
PATHS = {
    # mode: (dtype label, SHT kwargs, description)
    "tc_f64": ("f64", {"fp64_path": "tc"},
               "tcgen05 contraction on 7-bit digit slices (FP64 accuracy), double-float FFTs"),
    "tc": ("bf16x3 (f32 data, f32 accumulate)", {"fp32_path": "tc"},
           "tcgen05 split-bf16 contraction vs FP64-built P panels"),
    "otf": ("bf16x3 (f32 data, f32 accumulate)", {"fp32_path": "otf"},
            "tcgen05 split-bf16 contraction, P generated on the fly (FP32, restarted every 32 degrees)"),
    "f32": ("f32", {}, "FP32 on-the-fly recurrence (exponent scale, restarted every 32 degrees)"),
    "f64": ("f64", {}, "plain FP64 on-the-fly recurrence"),
    "auto": ("f32 / bf16x3 (tuned)", {}, "runtime-tuned: FP32 on-the-fly, tcgen05 panels or tcgen05 on-the-fly P"),
}


def is_fp64(mode):
    return mode in ("f64", "tc_f64")


def make_plan(mode, dev, lmax=LMAX, nlat=NLAT, nphi=NPHI):
    from paper_1202_6522_gb300 import SHT
    return SHT(lmax, lmax, nlat, nphi, device=dev, **PATHS[mode][1])


def device_timed(sht, torch, a, steps, warmup, stream, barrier, clocks=False, uuid=None):
    """W warm-up round trips, then exactly `steps` round trips between CUDA
    events on the launching stream, bracketed by barrier + synchronize; the
    per-kernel table from the library's own events; clocks sampled during the
    timed region.  Returns (ms total, kernel table, clocks)."""
    from paper_1202_6522_gb300 import _capi as C
    for _ in range(warmup):
        sht.analys_(sht.synth_(a))
    barrier()
    C.sht_profile(sht._h, True)
    C.sht_profile_read(sht._h)
    sampler = ClockSampler(uuid) if clocks else None
    if sampler:
        sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(steps):
        sht.analys_(sht.synth_(a))
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = sampler.stop() if sampler else None
    table = C.sht_profile_read(sht._h)
    C.sht_profile(sht._h, False)
    return ms, table, clk


def e2e_timed(sht, torch, dev, a_np, cdt, stream, min_steps, barrier, nbuf=2):
    """The same round trips end to end through the public API from pinned host
    memory: every step uploads its own input and downloads its result.
    Uploads, transforms and downloads run on three streams with nbuf device
    buffers, so step k+1's upload and step k-1's download overlap step k's
    transforms.  The pipeline is first filled (nbuf + 2 steps); the timed
    region then runs at least `min_steps` steps and at least E2E_MIN_SECONDS.
    Returns (seconds, steps, bytes in, bytes out per step)."""
    host_in = [torch.from_numpy(a_np).to(cdt).pin_memory() for _ in range(nbuf)]
    host_out = [torch.empty_like(host_in[0]).pin_memory() for _ in range(nbuf)]
    d_in = [torch.empty_like(host_in[0], device=dev) for _ in range(nbuf)]
    s_up, s_down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    up_done = [torch.cuda.Event() for _ in range(nbuf)]
    comp_done = [torch.cuda.Event() for _ in range(nbuf)]
    down_done = [torch.cuda.Event() for _ in range(nbuf)]

    def run(n):
        for k in range(n):
            i = k % nbuf
            with torch.cuda.stream(s_up):
                s_up.wait_event(comp_done[i])          # buffer i no longer read by step k - nbuf
                d_in[i].copy_(host_in[i], non_blocking=True)
                up_done[i].record(s_up)
            d_in[i].record_stream(stream)
            stream.wait_event(up_done[i])
            stream.wait_event(down_done[i])            # host_out[i] of step k - nbuf downloaded
            r = sht.analys_(sht.synth_(d_in[i]))
            comp_done[i].record(stream)
            with torch.cuda.stream(s_down):
                s_down.wait_event(comp_done[i])
                host_out[i].copy_(r, non_blocking=True)
                r.record_stream(s_down)                # keep r's memory until the download ran
                down_done[i].record(s_down)

    run(nbuf + 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run(nbuf + 2)
    torch.cuda.synchronize()
    per = (time.perf_counter() - t0) / (nbuf + 2)
    n = max(min_steps, int(math.ceil(E2E_MIN_SECONDS / max(per, 1e-6))))
    barrier()
    t0 = time.perf_counter()
    run(n)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    b = host_in[0].numel() * host_in[0].element_size()
    return dt, n, b, b


def roofline(mode, sht, table, peaks, alu_peaks, sm_max, batch=BATCH, lmax=LMAX, nlat=NLAT, nphi=NPHI):
    """Roofline of the dominant kernel kind of a timed region."""
    from paper_1202_6522_gb300 import _capi as C
    dom_name, (dom_ms, dom_n) = max(table.items(), key=lambda kv: kv[1][0])
    dom_avg = dom_ms / dom_n
    hbm = peaks.get("hbm_gbs", 6800.0) * 1e9
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s"
    if dom_name.startswith("tc_") and mode == "otf":
        skip_s, skip_a = C.sht_tc_polar_skip(sht._h)
        skip = max(0.0, skip_a if dom_name == "tc_analys" else skip_s)
        flops = nlm_of(lmax) * ((nlat + 1) // 2) * 5.0 * (1.0 - skip)
        peak = (alu_peaks[0] * 1e12) if alu_peaks else fp32_alu_peak(sm_max)
        ach = flops / (dom_avg / 1e3)
        return {"bound": "alu", "kernel": dom_name, "achieved": ach / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "peak_source": "measured FP32 FMA throughput (sht_alu_peaks)" if alu_peaks else "FP32 nominal",
                "algorithmic_flops": flops, "kernel_avg_ms": dom_avg, "launches": dom_n}
    if dom_name.startswith("tc_"):
        skip_s, skip_a = C.sht_tc_polar_skip(sht._h)
        skip = max(0.0, skip_a if dom_name == "tc_analys" else skip_s)
        if mode == "tc_f64":
            algo = tc64_algorithmic_bytes(batch, lmax, nlat, zero_skip=skip)
            kern = dom_name      # the stage's kernels, timed together
            note = ("digit-data pass + contraction, timed together; bytes: digit panels less the all-zero "
                    "8-row groups + FP64 data in and out")
        else:
            algo = tc_algorithmic_bytes(batch, lmax, nlat, polar_skip=skip)
            kern = "k_tc_ws<0>" if dom_name == "tc_analys" else "k_tc_ws<1>"
            note = "bytes: bf16 hi+lo panels less the polar skip + FP32 data in and out"
        ach = algo / (dom_avg / 1e3)
        return {"bound": "hbm", "kernel": dom_name, "achieved": ach / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
                "frac": ach / hbm, "traffic": profiled_traffic(kern) if (lmax, batch) == (LMAX, BATCH) else None,
                "peak_source": hbm_src, "algorithmic_bytes": algo, "kernel_avg_ms": dom_avg, "launches": dom_n,
                "skip": {"synth": skip_s, "analys": skip_a}, "note": note}
    if dom_name.startswith("fft") and not is_fp64(mode):
        algo = fft_algorithmic_bytes(batch, lmax, nlat, nphi, 4)
        ach = algo / (dom_avg / 1e3)
        return {"bound": "hbm", "kernel": dom_name, "achieved": ach / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
                "frac": ach / hbm, "traffic": None, "peak_source": hbm_src, "algorithmic_bytes": algo,
                "kernel_avg_ms": dom_avg, "launches": dom_n}
    skip = None
    if dom_name.startswith("legendre"):
        # terms before their pair's first live segment (static polar
        # optimisation) are not algorithmic work; warps skip only whole
        # groups of 32 pairs, so this count is at most the work done
        skip = C.sht_cc_polar_skip(sht._h, C.SHT_F64 if is_fp64(mode) else C.SHT_F32)
        flops = legendre_flops_per_launch(batch, lmax, nlat) * (1.0 - max(0.0, skip))
    else:
        flops = batch * nlat * 2.5 * nphi * math.log2(nphi)
    if is_fp64(mode) and mode != "tc_f64":
        peak, src = ((alu_peaks[1] * 1e12, "measured FP64 FMA throughput (sht_alu_peaks)") if alu_peaks
                     else (FP64_PEAK_NOMINAL, "FP64 nominal 1.25 TFLOP/s"))
    else:
        peak, src = ((alu_peaks[0] * 1e12, "measured FP32 FMA throughput (sht_alu_peaks)") if alu_peaks
                     else (fp32_alu_peak(sm_max), "FP32 nominal"))
    ach = flops / (dom_avg / 1e3)
    res = {"bound": "alu", "kernel": dom_name, "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
           "frac": ach / peak, "traffic": None, "peak_source": src, "algorithmic_flops": flops,
           "kernel_avg_ms": dom_avg, "launches": dom_n}
    if skip is not None:
        res["polar_terms_skipped"] = skip
    return res


def kernels_per_launch(mode, kind):
    """Kernels the library launches per profiled call of a kind (the timer
    brackets each call): the panel contraction converts its operands in-kernel
    (a separate operand-prep kernel runs first only for a synthesis with an odd
    coefficient count); the on-the-fly contraction always has a prep kernel;
    the FP64-accurate synthesis finds the field exponents (fill + reduction)
    and writes the data digits before its contraction, its analysis FFT fills
    the exponent words first and its contraction has a digit pass."""
    if mode == "tc_f64":
        return {"tc_synth": 4, "tc_analys": 2, "fft_analys": 2}.get(kind, 1)
    if not kind.startswith("tc_"):
        return 1
    if mode == "otf":
        return 2
    return 2 if (kind == "tc_synth" and nlm_of(LMAX) % 2) else 1


def round_trip_errors(sht, torch, dev, cdt, lmax=LMAX):
    """Sec. 3.5 error measures of one round trip of uniform [-1, 1] spectra."""
    import numpy as np
    from paper_1202_6522_gb300 import synthetic
    Q = synthetic.spectrum(lmax, seed=0, uniform=True)
    Qd = torch.from_numpy(Q).to(dev, cdt)
    R = sht.analys_(sht.synth_(Qd)).cpu().numpy().astype(np.complex128)
    Qr = Qd.cpu().numpy().astype(np.complex128)
    d = np.abs(R - Qr)
    return {"eps_max": float(d.max()), "eps_rms": float(np.sqrt(2.0 / ((lmax + 1) * (lmax + 2)) * np.sum(d * d)))}


def collect_samples(key, sht, torch, dev, cdt, samples, lmax=LMAX, nlat=NLAT, nphi=NPHI, seed=0):
    """GPU outputs on sampled rows (synthesis) and orders (analysis) of one
    field, stored for the oracle check of the CPU baseline leg."""
    import numpy as np
    from paper_1202_6522_gb300 import synthetic
    a = synthetic.spectrum(lmax, seed=seed)
    if cdt == torch.complex64:
        a = a.astype(np.complex64).astype(np.complex128)
    rows = [0, 1, nlat // 4, nlat // 2 - 1, nlat - 1]
    g = sht.synth_(torch.from_numpy(a).to(dev, cdt)).cpu().numpy().astype(np.float64)
    samples[key + "_synth"] = {"kind": "synth", "lmax": lmax, "nlat": nlat, "nphi": nphi, "input": a, "rows": rows,
                               "got": g[rows], "what": f"synthesis, 1 field, rows {rows}"}
    grid = synthetic.grid(nlat, nphi, seed=seed + 1)
    if cdt == torch.complex64:
        grid = grid.astype(np.float32).astype(np.float64)
    rdt = torch.float64 if cdt == torch.complex128 else torch.float32
    s = sht.analys_(torch.from_numpy(grid).to(dev, rdt)).cpu().numpy().astype(np.complex128)
    ms = [0, 1, lmax // 3, lmax]
    idx = packed_index(lmax, ms)
    samples[key + "_analys"] = {"kind": "analys", "lmax": lmax, "nlat": nlat, "nphi": nphi, "input": grid, "ms": ms,
                                "idx": idx, "got": s[idx], "what": f"analysis, 1 field, orders {ms}"}


def packed_index(lmax, ms):
    import numpy as np
    return np.concatenate([[m * (2 * lmax + 3 - m) // 2 + (n - m) for n in range(m, lmax + 1)] for m in ms])


# ---------------------------------------------------------------------------
# the other workloads of the study
# ---------------------------------------------------------------------------
def uneven_batch(torch, dev, samples, replays=200):
    """96 FP32 fields with N drawn from {63, 127, 255, 511} (nlat = N+1, nphi =
    2(N+1)): round-trip latency of one graph launch per direction (persistent
    CUDA-core kernels, and the tensor-core mode with one contraction per shape
    group) vs the persistent kernels launched directly vs one launch pair per
    field, and the path the automatic mode picks."""
    import numpy as np
    from paper_1202_6522_gb300 import SHT, UnevenBatch, synthetic
    lmaxs = synthetic.uneven_truncations(96)
    hist = {str(n): lmaxs.count(n) for n in sorted(set(lmaxs))}
    specs_np = [synthetic.spectrum(l, seed=i).astype(np.complex64) for i, l in enumerate(lmaxs)]
    specs = [torch.from_numpy(s).to(dev) for s in specs_np]
    plans = {l: SHT(l, l, l + 1, 2 * (l + 1), device=dev) for l in set(lmaxs)}
    stream = torch.cuda.current_stream(dev)

    def per_field():
        for l, sp in zip(lmaxs, specs):
            plans[l].analys_(plans[l].synth_(sp))

    def measure(fn):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        lat = []
        t0 = time.perf_counter()
        for _ in range(replays):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            lat.append(e0.elapsed_time(e1))
        wall = time.perf_counter() - t0
        lat.sort()
        return {"p50_ms": lat[len(lat) // 2], "p99_ms": lat[int(0.99 * (len(lat) - 1))],
                "round_trips_per_s": len(lmaxs) * replays / wall}

    out = {"fields": len(lmaxs), "truncations": hist, "replays": replays}
    for name, graph, path in (("graph", True, "f32"), ("persistent_no_graph", False, "f32"),
                              ("tc_graph", True, "tc")):
        ub = UnevenBatch(lmaxs, device=dev, use_graph=graph, path=path)
        grids = ub.synth_(specs)
        back = ub.analys_(grids)
        out[name] = measure(lambda: ub.analys_(ub.synth_(specs, out=grids), out=back))
        if graph:
            # Sec. 3.5 round trip over all fields, and two fields per path for the oracle check
            torch.cuda.synchronize()
            d = np.concatenate([np.abs(b.cpu().numpy().astype(np.complex128) - s.astype(np.complex128))
                                for b, s in zip(back, specs_np)])
            out[name]["round_trip_error_sec35"] = {"eps_max": float(d.max()), "eps_rms": float(np.sqrt(np.mean(d * d)))}
            for i in (0, 95):
                l = lmaxs[i]
                rows = [0, l // 2, l]
                samples[f"uneven_{name}_field{i}"] = {
                    "kind": "synth", "lmax": l, "nlat": l + 1, "nphi": 2 * (l + 1),
                    "input": specs_np[i].astype(np.complex128), "rows": rows,
                    "got": grids[i].cpu().numpy().astype(np.float64)[rows],
                    "what": f"uneven batch ({name}) synthesis, field {i} (N={l}), rows {rows}"}
        del ub
    auto = UnevenBatch(lmaxs, device=dev, path="auto")
    out["auto"] = {"chosen": auto.path, "tuned_round_trip_ms": auto.tuned_ms}
    del auto
    out["per_field_launches"] = measure(per_field)
    return out


def vector_config(torch, dev, samples, steps=5):
    """Spheroidal/toroidal round trip, N = 511 (nlat 512, nphi 1024), 64 shells,
    FP32 data: round trips (shells) per second on the CUDA-core path ("f32")
    and on the tensor-core path ("tc"), with the Sec. 3.5 round-trip error and
    sampled outputs for the oracle check."""
    import numpy as np
    from paper_1202_6522_gb300 import SHT, synthetic
    n, shells, nlat, nphi = 511, 64, 512, 1024
    S_np = synthetic.spectrum(n, batch=shells, seed=4, power=1.5).astype(np.complex64)
    T_np = synthetic.spectrum(n, batch=shells, seed=5, power=1.5).astype(np.complex64)
    S = torch.from_numpy(S_np).to(dev)
    T = torch.from_numpy(T_np).to(dev)
    out = {"workload": "vector round trip N=511 nlat=512 nphi=1024, 64 shells, FP32 data"}
    for path in ("f32", "tc"):
        sht = SHT(n, n, nlat, nphi, device=dev, fp32_path=path)
        for _ in range(2):
            sht.analys_vec_(*sht.synth_vec_(S, T))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            sht.analys_vec_(*sht.synth_vec_(S, T))
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        # Sec. 3.5 measures of the round trip (n = 0 carries no vector information)
        vt, vp = sht.synth_vec_(S, T)
        S2, T2 = sht.analys_vec_(vt, vp)
        ns, _ = synthetic.packed_degrees_orders(n)
        keep = ns > 0
        d = np.concatenate([np.abs(S2.cpu().numpy() - S_np)[:, keep].ravel(),
                            np.abs(T2.cpu().numpy() - T_np)[:, keep].ravel()]).astype(np.float64)
        out[path] = {"ms_per_step": ms, "round_trips_per_s": shells / (ms / 1e3),
                     "round_trip_error_sec35": {"eps_max": float(d.max()), "eps_rms": float(np.sqrt(np.mean(d * d)))}}
        rows = [0, 127, 255, 511]
        b = 33
        samples[f"vector_{path}_synth"] = {
            "kind": "synth_vec", "lmax": n, "nlat": nlat, "nphi": nphi,
            "input": (S_np[b].astype(np.complex128), T_np[b].astype(np.complex128)), "rows": rows,
            "got": np.concatenate([vt[b].cpu().numpy()[rows].ravel(), vp[b].cpu().numpy()[rows].ravel()]),
            "what": f"vector synthesis ({path}), shell {b}, rows {rows}, v_theta and v_phi"}
        gt = synthetic.grid(nlat, nphi, seed=6).astype(np.float32)
        gp = synthetic.grid(nlat, nphi, seed=7).astype(np.float32)
        S3, T3 = sht.analys_vec_(torch.from_numpy(gt).to(dev)[None], torch.from_numpy(gp).to(dev)[None])
        ms_ = [0, 1, 200, 511]
        idx = packed_index(n, ms_)
        samples[f"vector_{path}_analys"] = {
            "kind": "analys_vec", "lmax": n, "nlat": nlat, "nphi": nphi,
            "input": (gt.astype(np.float64), gp.astype(np.float64)), "ms": ms_, "idx": idx,
            "got": np.concatenate([S3[0].cpu().numpy()[idx], T3[0].cpu().numpy()[idx]]),
            "what": f"vector analysis ({path}), 1 field, orders {ms_}, S and T"}
        del sht
    return out


def differentiable_config(torch, dev, samples, steps=10):
    """loss = ||synth(a) - target||^2 and its gradient (through the adjoint
    kernels) at the bench size on the split-bf16 tensor-core path: forward +
    backward steps per second x batch; the gradient's directional central
    difference (exact for a quadratic loss at any step) and sampled orders for
    the oracle check."""
    import numpy as np
    from paper_1202_6522_gb300 import synthetic
    sht = make_plan("tc", dev)
    a_np = synthetic.spectrum(LMAX, batch=BATCH, seed=2).astype(np.complex64)
    t_np = synthetic.grid(NLAT, NPHI, batch=BATCH, seed=2).astype(np.float32)
    a = torch.from_numpy(a_np).to(dev).requires_grad_(True)
    tgt = torch.from_numpy(t_np).to(dev)

    def step():
        a.grad = None
        loss = ((sht.synth(a) - tgt) ** 2).sum()
        loss.backward()
        return loss

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    g = a.grad.detach().cpu().numpy().astype(np.complex128)
    d = synthetic.spectrum(LMAX, batch=BATCH, seed=9).astype(np.complex64)

    def L(x):
        with torch.no_grad():
            r = sht.synth(torch.from_numpy(x).to(dev)).double() - tgt.double()
            return float((r * r).sum())
    fd = (L(a_np + d) - L(a_np - d)) / 2.0
    an = float(np.sum(g.real * d.real + g.imag * d.imag))
    ms_ = [0, 1, 64, 500, 1023]
    idx = packed_index(LMAX, ms_)
    samples["differentiable_gradient"] = {
        "kind": "loss_grad", "lmax": LMAX, "nlat": NLAT, "nphi": NPHI,
        "input": (a_np[0].astype(np.complex128), t_np[0].astype(np.float64)), "ms": ms_, "idx": idx,
        "got": g[0][idx], "what": f"loss gradient, field 0, orders {ms_}"}
    del sht
    return {"workload": f"loss=||synth(a)-target||^2 + gradient, N={LMAX}, batch {BATCH}, split-bf16 tensor cores",
            "ms_per_step": ms, "fields_per_s": BATCH / (ms / 1e3),
            "directional_fd": {"fd": fd, "analytic": an, "rel_diff": abs(fd - an) / abs(an)}}


def accuracy_vs_n(torch, dev, sizes=(255, 511, 1023, 2047, 4095)):
    """The Sec. 3.5 error measures of one round trip of uniform [-1, 1] spectra
    against N (nlat = N + 1, nphi = 2 (N + 1)), for the FP64 path, the FP32
    recurrence, (N <= 2047) the tensor-core path and (N <= 1023) the
    FP64-accurate tensor-core path: the analogue of the paper's
    error-versus-N study (its 1e-11 target is for N < 2048)."""
    from paper_1202_6522_gb300 import SHT
    out = {}
    for n in sizes:
        row = {}
        for path in ("f64", "f32", "tc", "tc_f64"):
            if path == "tc" and n > 2047:
                continue
            if path == "tc_f64" and n > 1023:
                continue
            sht = make_plan(path, dev, n, n + 1, 2 * (n + 1))
            row[path] = round_trip_errors(sht, torch, dev, torch.complex128 if is_fp64(path) else torch.complex64, n)
            del sht
            torch.cuda.empty_cache()
        out[str(n)] = row
    return out


def n511_config(torch, dev, steps=20):
    """Scalar round trips per second at N = 511 (nlat 512, nphi 1024), batch
    16, on every path (the metric's second size)."""
    import numpy as np
    from paper_1202_6522_gb300 import synthetic
    out = {"workload": "scalar SHT round trip N=511 nlat=512 nphi=1024 batch=16"}
    a_np = synthetic.spectrum(511, batch=16, seed=0)
    for path in ("f64", "f32", "tc", "tc_f64"):
        sht = make_plan(path, dev, 511, 512, 1024)
        a = torch.from_numpy(a_np).to(dev, torch.complex128 if is_fp64(path) else torch.complex64)
        n = max(3, steps // 5) if path == "f64" else steps
        for _ in range(3):
            sht.analys_(sht.synth_(a))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            sht.analys_(sht.synth_(a))
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / n
        out[path] = {"ms_per_step": ms, "round_trips_per_s": 16 / (ms / 1e3),
                     "gflops_nominal": 16 / (ms / 1e3) * nominal_flops_per_rt(511, 512, 1024) / 1e9}
        del sht, a
    return out


def high_n_config(torch, dev, peaks, alu_peaks, sm_max):
    """Round trips per second, nominal GFLOP/s and the dominant kernel's roofline
    at N = 2047 (4096 longitudes) and N = 4095 (8192), batch 4, on the FP64,
    FP32 and tensor-core (panel) paths: the high-degree regime of the paper's
    Table 1, where the rescaling of Sec. 3.5 is needed."""
    import numpy as np
    from paper_1202_6522_gb300 import _capi as C
    from paper_1202_6522_gb300 import synthetic
    out = {}
    batch = 4
    for n in (2047, 4095):
        nlat, nphi = n + 1, 2 * (n + 1)
        a_np = synthetic.spectrum(n, batch=batch, seed=0)
        row = {"workload": f"scalar SHT round trip N={n} nlat={nlat} nphi={nphi} batch={batch}"}
        for path in ("f64", "f32", "tc"):
            sht = make_plan(path, dev, n, nlat, nphi)
            a = torch.from_numpy(a_np).to(dev, torch.complex128 if is_fp64(path) else torch.complex64)
            steps = 2 if path == "f64" else 5
            sht.analys_(sht.synth_(a))
            torch.cuda.synchronize()
            C.sht_profile(sht._h, True)
            C.sht_profile_read(sht._h)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                sht.analys_(sht.synth_(a))
            e1.record()
            e1.synchronize()
            table = C.sht_profile_read(sht._h)
            C.sht_profile(sht._h, False)
            ms = e0.elapsed_time(e1) / steps
            rt = batch / (ms / 1e3)
            row[path] = {"ms_per_step": ms, "round_trips_per_s": rt,
                         "gflops_nominal": rt * nominal_flops_per_rt(n, nlat, nphi) / 1e9,
                         "elements_per_s": rt * (n + 1) ** 3,
                         "roofline": roofline(path, sht, table, peaks, alu_peaks, sm_max, batch, n, nlat, nphi)}
            del sht, a
            torch.cuda.empty_cache()
        out[str(n)] = row
    return out


def polar_sweep(torch, dev, thresholds=(0.0, 2.0 ** -40, 2.0 ** -32, 2.0 ** -26, 2.0 ** -20), steps=20):
    """The static polar optimisation of Sec. 3.1 (threshold left open by the
    paper): tensor-core round-trip time, fraction of panel chunks skipped and
    round-trip error (Sec. 3.5 measures, uniform spectra) per threshold, at
    the bench size."""
    import numpy as np
    from paper_1202_6522_gb300 import _capi as C
    from paper_1202_6522_gb300 import synthetic
    sht = make_plan("tc", dev)
    a = torch.from_numpy(synthetic.spectrum(LMAX, batch=BATCH, seed=0).astype(np.complex64)).to(dev)
    out = []
    for thr in thresholds:
        C.sht_set_polar_threshold(sht._h, thr)
        for _ in range(3):
            sht.analys_(sht.synth_(a))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            sht.analys_(sht.synth_(a))
        e1.record()
        e1.synchronize()
        fs, fa = C.sht_tc_polar_skip(sht._h)
        out.append({"threshold": thr, "ms_per_step": e0.elapsed_time(e1) / steps, "skip_synth": fs,
                    "skip_analys": fa, **round_trip_errors(sht, torch, dev, torch.complex64)})
    del sht
    return out


def polar_sweep_cc(torch, dev, thresholds=(0.0, 2.0 ** -64, 2.0 ** -40, 2.0 ** -26, 2.0 ** -20), steps=3):
    """The same sweep on the paper's own on-the-fly design: the plain FP64
    CUDA-core path, whose kernels skip the 32-degree segments before each
    pair's first live one (the FP64 default threshold is 2^-64)."""
    import numpy as np
    from paper_1202_6522_gb300 import _capi as C
    from paper_1202_6522_gb300 import synthetic
    sht = make_plan("f64", dev)
    a = torch.from_numpy(synthetic.spectrum(LMAX, batch=BATCH, seed=0)).to(dev)
    out = []
    for thr in thresholds:
        C.sht_set_polar_threshold(sht._h, thr)
        sht.analys_(sht.synth_(a))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            sht.analys_(sht.synth_(a))
        e1.record()
        e1.synchronize()
        out.append({"threshold": thr, "ms_per_step": e0.elapsed_time(e1) / steps,
                    "terms_below_first_live": C.sht_cc_polar_skip(sht._h, C.SHT_F64),
                    **round_trip_errors(sht, torch, dev, torch.complex128)})
    del sht
    return out


# ---------------------------------------------------------------------------
def timed_leg(mode, torch, dev, stream, a_np, steps, warmup, world, barrier, peaks, alu_peaks, uuid, samples,
              clocks=True, e2e=True):
    """One path on the bench workload: the device-timed region, its kernel
    table and roofline, the end-to-end measurement, the Sec. 3.5 round-trip
    error and sampled outputs for the oracle check."""
    sht = make_plan(mode, dev)
    cdt = torch.complex128 if is_fp64(mode) else torch.complex64
    tune = None
    if mode == "auto":
        from paper_1202_6522_gb300 import _capi as C
        f32_ms, tc_ms, otf_ms = C.sht_tune(sht._h, BATCH, C.SHT_F32_AUTO, stream.cuda_stream)
        sht.fp32_mode = C.SHT_F32_AUTO
        cands = {"f32": f32_ms, "tc": tc_ms, "otf": otf_ms}
        tune = {"f32_round_trip_ms": f32_ms, "tc_round_trip_ms": tc_ms, "tc_otf_round_trip_ms": otf_ms,
                "chosen": min((v, k) for k, v in cands.items() if v > 0)[1]}
    a = torch.from_numpy(a_np).to(dev, cdt)
    ms_total, table, clk = device_timed(sht, torch, a, steps, warmup, stream, barrier, clocks, uuid)
    ms_total, value = job_throughput(ms_total, world, BATCH * steps, dev)
    path_used = (tune or {}).get("chosen", mode)
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    res = {"value": value, "unit": UNIT, "ms_per_step": ms_total / steps, "steps": steps, "warmup": warmup,
           "dtype": PATHS[mode][0], "path": PATHS[mode][2], "path_used": path_used,
           "gflops_nominal": value * nominal_flops_per_rt() / 1e9, "elements_per_s": value * (LMAX + 1) ** 3,
           "roofline": roofline(path_used, sht, table, peaks, alu_peaks, sm_max),
           "kernels": {k: {"avg_ms": v[0] / v[1], "launches": v[1],
                           "share": v[0] / sum(x[0] for x in table.values())} for k, v in table.items()},
           "gpu_launches": sum(v[1] * kernels_per_launch(path_used, k) for k, v in table.items())}
    if clk is not None:
        res["clocks"] = clk
    if tune:
        res["tuning"] = tune
    if e2e:
        dt, n, bi, bo = e2e_timed(sht, torch, dev, a_np, cdt, stream, steps, barrier)
        _, ev = job_throughput(1e3 * dt, world, BATCH * n, dev)
        res["e2e"] = {"value": ev, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "steps": n,
                      "seconds": dt, "note": "pinned host buffers, upload/transform/download overlapped across "
                                             "steps on 3 streams; pipeline filled first, >= 1 s timed"}
    res["round_trip_error_sec35"] = round_trip_errors(sht, torch, dev, cdt)
    if samples is not None:
        collect_samples(mode, sht, torch, dev, cdt, samples)
    del sht, a
    torch.cuda.empty_cache()
    return res


def run_ours(args):
    import torch

    from paper_1202_6522_gb300 import _capi as C
    from paper_1202_6522_gb300 import build as B
    from paper_1202_6522_gb300 import synthetic
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    B.build()
    stream = torch.cuda.current_stream(dev)
    peaks = read_peaks()
    try:
        alu_peaks = C.sht_alu_peaks(stream.cuda_stream)   # ALU roofline denominators (FP32, FP64)
    except Exception:
        alu_peaks = None
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    extras = rank == 0 and not args.no_extras
    samples = {} if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    a_np = synthetic.spectrum(LMAX, batch=BATCH, seed=rank)
    head = timed_leg(args.mode, torch, dev, stream, a_np, args.steps, args.warmup, world, barrier, peaks,
                     alu_peaks, uuid, samples)

    # --- the other paths on the same workload ---
    others = {}
    legs = [m for m in ("tc", "f32", "f64", "tc_f64") if m != args.mode] if extras else \
        ([] if args.mode == "f64" else ["f64"])
    for m in legs:
        k_steps = max(2, args.steps // 4) if m == "f64" else args.steps
        k_warm = 1 if m == "f64" else args.warmup
        others[m] = timed_leg(m, torch, dev, stream, a_np, k_steps, k_warm, world, barrier, peaks, alu_peaks, uuid,
                              samples if m in ("tc",) else None, clocks=m == "tc", e2e=m == "tc")

    extra = {}
    if extras:
        extra["vector"] = vector_config(torch, dev, samples if samples is not None else {})
        extra["uneven_batch"] = uneven_batch(torch, dev, samples if samples is not None else {})
        extra["differentiable"] = differentiable_config(torch, dev, samples if samples is not None else {})
        extra["n511"] = n511_config(torch, dev)
        extra["high_n"] = high_n_config(torch, dev, peaks, alu_peaks, (head.get("clocks") or {}).get("sm_max_mhz") or 2070.0)
        extra["polar_threshold_sweep"] = polar_sweep(torch, dev)
        extra["polar_threshold_sweep_fp64_cuda_cores"] = polar_sweep_cc(torch, dev)
        extra["accuracy_vs_n"] = accuracy_vs_n(torch, dev)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    plain = others.get("f64") if args.mode != "f64" else head
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": head["dtype"], "data": "synthetic (seeded N(0,1)/(n+1) spectra)",
        "config": bench_config(world), "path": head["path"], "path_used": head["path_used"],
        "gflops_nominal": head["gflops_nominal"], "elements_per_s": head["elements_per_s"],
        "roofline": head["roofline"], "kernels": head["kernels"], "gpu_launches": head["gpu_launches"],
        "clocks": head.get("clocks"), "e2e": head["e2e"], "round_trip_error_sec35": head["round_trip_error_sec35"],
    }
    if "tuning" in head:
        line["tuning"] = head["tuning"]
    if plain is not None:
        line["speedup_vs_fp64_plain"] = head["value"] / plain["value"]
    if "tc" in others:
        line["bf16x3"] = others["tc"]
    for m, key in (("f64", "fp64_plain"), ("f32", "fp32"), ("tc_f64", "fp64_tensor_core")):
        if m in others:
            line[key] = others[m]
    if plain is not None:
        for key in ("bf16x3", "fp32", "fp64_tensor_core"):
            if key in line:
                line[key]["speedup_vs_fp64_plain"] = line[key]["value"] / plain["value"]
    if alu_peaks:
        line["alu_peaks_measured"] = {"fp32_tflops": alu_peaks[0], "fp64_tflops": alu_peaks[1]}
    line.update(extra)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        eps = oracle_checks(samples or {})
        line["eps_vs_oracle"] = eps
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=list(PATHS), default="tc_f64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", "--no-uneven", dest="no_extras", action="store_true",
                    help="time the headline path and the plain FP64 path only")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
