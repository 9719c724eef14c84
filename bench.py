#!/usr/bin/env python
"""Throughput of the GB300 FX correlator on the 10-station space-VLBI scan.

Workload: 10 stations (1 spacecraft + 9 ground), 8 subbands x 16 MHz x 2 pols
(32 Msample/s real, 2-bit), a 10 s scan, 1024 channels (2048-point FFTs),
1 s integrations, quintic delay segments (spacecraft delay ~0.3-1.2 s, rate up
to 3e-5 s/s; ground delays up to 20 ms), a segment boundary inside the scan.
One step correlates the whole scan (all 10 integrations) through the C ABI.

  value  station-samples/s with the packed samples already in device memory
         (corr_attach_samples_device + corr_correlate_device), timed with CUDA
         events on the library's stream over K steps;
  e2e    the same metric through the host API: every step pushes all stations'
         packed bytes from pinned host memory (corr_push_samples) and reads
         every integration back to host memory (corr_correlate).

A station-sample is one real 2-bit sample of one stream (station x subband x
pol).  Inputs (14 GB) exceed the 129 MB L2, so no flush is needed between
steps.  Synthetic data: independent 2-bit quantised Gaussian noise (codes
drawn with the probabilities of +-0.98 sigma quantisation) made on the device
from a seeded generator; the correlator's cost does not depend on the values.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample (the first 0.1 s of the same scan, one 0.1 s integration).
Multi-GPU (torchrun): independent replicas, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "cfg2: 10 stations (1 space + 9 ground), 8 subbands x 16 MHz, 2 pols, 2-bit, 10 s, 1024 channels, 1 s integrations"
METRIC = "station-samples/s"
CPU_SAMPLE_S = 0.1
DENSE_SAMPLE_S = 0.004   # 64-station sample for the measured error (16 of its 32 streams)
DENSE_SAMPLE_STREAMS = 16
# 2-bit code probabilities of +-0.98 sigma quantisation of a unit Gaussian
P_OUTER = 0.5 * (1.0 - 0.6729121)
FALLBACK_HBM_GBS = 6800.0
SM_COUNT, FP32_LANES, MAX_SM_MHZ = 152, 128, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tc", action="store_true", help="skip the FP16 tensor-core leg")
    ap.add_argument("--no-fp8", action="store_true", help="skip the FP8 tensor-core leg")
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--chunk-blocks", type=int, default=0, help="FFT blocks per F/X chunk (0: library default)")
    ap.add_argument("--duration", type=float, default=10.0,
                    help="scan length in seconds (10 s is the benchmark; shorter only for profiling)")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense 64-station X-step leg")
    ap.add_argument("--dense-duration", type=float, default=0.5,
                    help="seconds of the 64-station scan in the dense leg (the named scan is 4 s)")
    ap.add_argument("--dense-tint", type=float, default=0.25,
                    help="integration time of the dense leg (0.25 s is the workload; shorter only for profiling)")
    ap.add_argument("--dense-chunk-blocks", type=int, default=0,
                    help="FFT blocks per chunk in the dense leg (0: library default; smaller only for profiling)")
    ap.add_argument("--dense-stations", type=int, default=64,
                    help="stations of the dense leg (64 is the workload; fewer only for profiling its F kernel)")
    ap.add_argument("--dense-only", action="store_true",
                    help="run only the dense 64-station leg and print its result (for profiling)")
    ap.add_argument("--no-fringe", action="store_true", help="skip the delay-rate fringe-search leg")
    ap.add_argument("--no-peaks", action="store_true", help="skip the library-GEMM peak measurements")
    ap.add_argument("--no-batch", action="store_true", help="skip the 96-scan batched leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the served leg")
    ap.add_argument("--batch-scans", type=int, default=96)
    ap.add_argument("--serve-rates", default="2,5,10,20,40", help="Poisson arrival rates of the sweep, jobs/s")
    ap.add_argument("--serve-window", type=float, default=3.0,
                    help="seconds of arrivals per rate (the served workload names 120 s at 40 jobs/s)")
    ap.add_argument("--hbm-cap", type=float, default=180e9)
    ap.add_argument("--hbm-reserve", type=float, default=30e9)
    return ap.parse_args()


def max_over_ranks(x: float, device) -> float:
    """The largest x over all ranks of the process group (the slowest
    replica sets the step time); x itself with no group or one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_step: float, world_size: int, ms_per_step: float) -> float:
    """Whole-job throughput of independent replicas (weak scaling): every rank
    processes units_per_step in each step, and the step takes the slowest
    rank's time."""
    return units_per_step * world_size / (ms_per_step / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def profile_value(table, kernel):
    """Per-launch figure of `kernel` from a committed ncu summary table under
    profiles/ (captured at the benchmark's launch shape), else None."""
    p = os.path.join(ROOT, "profiles", table)
    if not os.path.exists(p):
        return None
    for line in open(p):
        parts = line.split()
        if len(parts) >= 2 and not line.startswith("#") and parts[0] == kernel:
            return float(parts[1])
    return None


def traffic_per_launch(kernel):
    """DRAM bytes (read + write) per launch of `kernel`."""
    return profile_value("traffic.txt", kernel)


def issue_frac(warp_instructions, launch_s, sm_mhz):
    """Fraction of the instruction-issue ceiling a launch reaches: its warp
    instructions over launch time x 4 issue slots per SM per clock x the SM
    count x the SM clock; None when an input is missing."""
    if not warp_instructions or not launch_s or not sm_mhz:
        return None
    return float(warp_instructions) / (float(launch_s) * 4.0 * SM_COUNT * float(sm_mhz) * 1e6)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "copy_gbs"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def device_codes(nbytes: int, gen, device):
    """Packed bytes of independent 2-bit codes with the quantised-Gaussian
    code probabilities, made on the device in chunks."""
    import torch
    out = torch.empty(nbytes, dtype=torch.uint8, device=device)
    t1 = int(round(P_OUTER * 65536))
    t2 = 32768
    t3 = 65536 - t1
    chunk = 1 << 26
    for o in range(0, nbytes, chunk):
        n = min(chunk, nbytes - o)
        u = torch.randint(0, 65536, (n, 4), generator=gen, device=device, dtype=torch.int32)
        c = (u >= t1).to(torch.uint8) + (u >= t2).to(torch.uint8) + (u >= t3).to(torch.uint8)
        out[o:o + n] = c[:, 0] | (c[:, 1] << 2) | (c[:, 2] << 4) | (c[:, 3] << 6)
    return out


def make_scan(seed, duration=10.0):
    import synth
    return synth.config2(seed=seed, duration=duration, tint=1.0, boundary=min(5.0, duration / 2))


def samples_per_step(scan):
    return scan.stations * scan.G * int(round(scan.duration / scan.tint)) * int(round(scan.fs * scan.tint))


def cpu_oracle_sample(scan, host_streams, seconds=CPU_SAMPLE_S, nj=None):
    """Time the FP64 oracle on the first `seconds` of the scan as one
    integration (all stations; the first nj streams, default all).
    Returns (samples/s, cores, secs, min weight, visibilities [nbl, nj, nchan])."""
    import oracle
    spi = int(round(scan.fs * seconds))
    nj = scan.G if nj is None else nj
    ns = []
    streams = []
    for s in range(scan.stations):
        n = min(scan.nsamp[s], (spi + 4 * scan.N + 70000) // 16 * 16)
        ns.append(n)
        streams.append(np.ascontiguousarray(host_streams[s][: n * scan.G // 4]))
    o = oracle.Oracle(scan.stations, scan.nsub, scan.npol, scan.nchan, scan.fs, seconds, scan.nu0,
                      scan.polys, streams, scan.sample0, ns)
    t0 = time.perf_counter()
    vis, w = o.correlate(0, 1, 0, nj)
    dt = time.perf_counter() - t0
    nblk = -(-spi // scan.N)
    samples = scan.stations * nj * nblk * scan.N
    cores = min(oracle.threads(), nj)
    return samples / dt, cores, dt, float(w.min()), vis[0]


def sample_errors(corr, scan, host_streams, ref, seconds=CPU_SAMPLE_S, precisions=(0, 1, 2), units=(0, 2)):
    """Largest relative RMS per baseline of the GPU path (through the C ABI,
    host-pushed samples) against the oracle's visibilities `ref` of the same
    sample, per precision (FP16 / FP8 for each X unit: CORR_X_AUTO, and
    CORR_X_TENSOR_CORES as "..._tensor_cores"): the measured error of the
    benchmarked workload."""
    spi = int(round(scan.fs * seconds))
    nj = ref.shape[1]
    out = {}
    for prec, unit in [(p, u) for p in precisions for u in (units if p else (0,))]:
        c = corr.Correlator(scan.stations, scan.nsub, scan.npol, scan.nchan, seconds, fs=scan.fs)
        for sb, nu in enumerate(scan.nu0):
            if nu:
                c.set_sky_freq(sb, nu)
        c.set_precision(prec)
        c.set_x_unit(unit)
        for s, segs in enumerate(scan.polys):
            for g in segs:
                c.set_delay_poly(s, g.t0, g.coeffs)
            c.set_stream_start(s, scan.sample0[s])
            n = min(scan.nsamp[s], (spi + 4 * scan.N + 70000) // 16 * 16)
            c.push(s, np.ascontiguousarray(host_streams[s][: n * scan.G // 4]))
        c.flush()
        v, _ = c.correlate()
        c.close()
        v = v.reshape(scan.nbl, scan.G, scan.nchan)[:, :nj]
        err = np.sqrt(np.sum(np.abs(v - ref) ** 2, axis=(1, 2)) / np.sum(np.abs(ref) ** 2, axis=(1, 2)))
        out[("fp32", "fp16", "fp8")[prec] + ("_tensor_cores" if unit == 2 else "")] = float(err.max())
    return out


def host_stream_prefix(dev_streams, scan, seconds=CPU_SAMPLE_S):
    spi = int(round(scan.fs * seconds))
    out = []
    for s, t in enumerate(dev_streams):
        n = min(scan.nsamp[s], (spi + 4 * scan.N + 70000) // 16 * 16)
        out.append(t[: n * scan.G // 4].cpu().numpy())
    return out


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import torch
    scan = make_scan(args.seed)
    gen = torch.Generator(device="cpu")
    gen.manual_seed(args.seed)
    spi = int(round(scan.fs * CPU_SAMPLE_S))
    streams = []
    for s in range(scan.stations):
        n = min(scan.nsamp[s], (spi + 4 * scan.N + 70000) // 16 * 16)
        streams.append(device_codes(n * scan.G // 4, gen, "cpu").numpy())
    for _ in range(args.warmup):
        cpu_oracle_sample(scan, streams)
    rates, secs = [], []
    cores = 1
    for _ in range(args.steps):
        r, cores, dt, _, _ = cpu_oracle_sample(scan, streams)
        rates.append(r)
        secs.append(dt)
    value = float(np.mean(rates))
    sample = "first %.1f s of the %s scan as one integration (all 10 stations, 16 streams)" % (CPU_SAMPLE_S, "cfg2")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def dense_leg(args, torch, corr, dev):
    """The X step where the station count makes it dense: 64 stations,
    16 subbands x 2 pols at 64 Msample/s, 4096 channels (8192-point FFTs),
    0.25 s integrations, on a --dense-duration slice of the 4 s scan.  Each
    precision correlates the same device-resident samples; reported per
    precision: station-samples/s, the X step's algorithmic TFLOP/s
    (8 flop per baseline, channel and block) and, on the tensor cores, the
    issued MMA rate (the real [Re; Im] product does about twice the
    algorithmic work) against the measured dense BF16 peak (x2 for FP8)."""
    import synth
    D = args.dense_duration
    sc = synth.config2(seed=3, duration=D, tint=args.dense_tint, boundary=D / 2, nchan=4096,
                       stations=args.dense_stations, nsub=16, npol=2, fs=64e6, nu0_base=1.6e9)
    gen = torch.Generator(device=dev)
    gen.manual_seed(3003)
    streams = [device_codes(sc.nsamp[s] * sc.G // 4, gen, dev) for s in range(sc.stations)]
    torch.cuda.synchronize()
    nint = int(round(D / sc.tint))
    spi = int(round(sc.fs * sc.tint))
    N = 2 * sc.nchan
    blocks = sum(-(-(i + 1) * spi // N) - (-(-i * spi // N)) for i in range(nint))
    x_flops = 8.0 * blocks * sc.G * sc.nchan * sc.nbl
    mma_flops = 2.0 * blocks * sc.G * (sc.nchan // 2) * 2 * 128 * 128  # 2 tiles of 128 rows per 2 channels
    sps = sc.stations * sc.G * nint * spi
    out = torch.empty((sc.nbl, sc.G, sc.nchan), dtype=torch.complex64, device=dev)
    w = torch.empty(sc.nbl, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    bf16 = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
    except Exception:
        bf16 = 1900.0
    res = {"workload": "cfg3 slice: %d stations, 16 subbands x 32 MHz, 2 pols, 2-bit, %.2f s of the 4 s scan, "
                       "4096 channels, %.2f s integrations" % (args.dense_stations, D, args.dense_tint),
           "schedule": "F and X in turn on one stream (stage times are each kernel's own)",
           "station_samples_per_step": sps, "input_bytes": int(sum(int(t.numel()) for t in streams))}
    for name, prec, bound in (("fp32", corr.CORR_PREC_FP32, 1e-5), ("fp16", corr.CORR_PREC_FP16_TC, 1e-3),
                              ("fp8", corr.CORR_PREC_FP8_TC, 8e-2)):
        c = corr.from_scan(sc, device_streams=streams)
        c.set_precision(prec)
        # F and X in turn: the stage times are each kernel's own
        c.set_pipeline(0)
        if args.dense_chunk_blocks:
            c.set_chunk_blocks(args.dense_chunk_blocks)
        c.set_stream(stream.cuda_stream)
        c.flush()

        def step():
            c.rewind()
            for _ in range(nint):
                rc = c.correlate_device(out, w)
                if rc != corr.CORR_OK:
                    raise RuntimeError("correlate_device returned %d" % rc)

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        c.read_profile()
        c.set_profiling(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        k = max(1, min(args.steps, 3))
        e0.record(stream)
        for _ in range(k):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        prof = c.read_profile()
        cb, _ = c.launch_shape()
        c.close()
        x_ms = prof["xstage"][0] / k
        r = {"value": sps / (ms / 1e3), "unit": METRIC, "ms_per_step": ms, "steps": k, "chunk_blocks": cb,
             "fstage_ms_per_step": prof["fstage"][0] / k, "xstep_ms_per_step": x_ms,
             "xstep_tflops": x_flops / (x_ms / 1e3) / 1e12 if x_ms > 0 else None,
             "error_bound_rel_rms": bound, "measured_rel_rms": None}
        if prec != corr.CORR_PREC_FP32 and x_ms > 0:
            peak = bf16 * (2.0 if prec == corr.CORR_PREC_FP8_TC else 1.0)
            r["xstep_mma_tflops_issued"] = mma_flops / (x_ms / 1e3) / 1e12
            r["tensor_peak_tflops"] = peak
            r["tensor_frac"] = r["xstep_mma_tflops_issued"] / peak
        res[name] = r
    for name in ("fp16", "fp8"):
        if res["fp32"]["xstep_ms_per_step"] > 0:
            res[name]["xstep_vs_fp32_xstep"] = res["fp32"]["xstep_ms_per_step"] / res[name]["xstep_ms_per_step"]
    # host copy of the scan's first samples, for the measured error of each
    # precision against the oracle (computed in the CPU-baseline leg)
    prefix = host_stream_prefix(streams, sc, DENSE_SAMPLE_S)
    del streams
    torch.cuda.empty_cache()
    return res, (sc, prefix)


def peaks_leg(args, torch, dev):
    """Throughput of library GEMMs on this GPU, as measured denominators for
    the per-stage rooflines: FP32 on CUDA cores (cuBLAS SGEMM with TF32 off),
    FP64, BF16 and, where this torch has it, scaled E4M3 (torch._scaled_mm).
    Square GEMMs, 2 n^3 flops, best of several timed with CUDA events."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False

    def best(fn, flops, reps=5):
        fn()
        torch.cuda.synchronize()
        t = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1) / 1e3)
        return flops / min(t) / 1e12

    try:
        for name, dt, n in (("fp32_tflops", torch.float32, 8192), ("fp64_tflops", torch.float64, 4096),
                            ("bf16_tflops", torch.bfloat16, 8192)):
            a = torch.randn((n, n), device=dev, dtype=torch.float32).to(dt)
            b = torch.randn((n, n), device=dev, dtype=torch.float32).to(dt)
            out[name] = best(lambda: torch.matmul(a, b), 2.0 * n ** 3)
            del a, b
        if hasattr(torch, "_scaled_mm") and hasattr(torch, "float8_e4m3fn"):
            n = 8192
            a = torch.randn((n, n), device=dev).to(torch.float8_e4m3fn)
            b = torch.randn((n, n), device=dev).to(torch.float8_e4m3fn).t()
            one = torch.ones((), device=dev, dtype=torch.float32)
            try:
                out["fp8_tflops"] = best(lambda: torch._scaled_mm(a, b, scale_a=one, scale_b=one,
                                                                  out_dtype=torch.bfloat16), 2.0 * n ** 3)
            except Exception as e:  # not every build supports it
                out["fp8_tflops"] = None
                out["fp8_note"] = "torch._scaled_mm unavailable: %s" % str(e).splitlines()[0][:120]
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
        torch.cuda.empty_cache()
    out["how"] = "torch.matmul / torch._scaled_mm (cuBLAS / cuBLASLt), square GEMMs, best of 5, CUDA events"
    return out


def fringe_leg(args, torch, corr, dev):
    """Delay-rate fringe search (corr_fringe_search) of one baseline: 256
    sub-integrations x 1024 channels, padded to 512 rate x 8192 lag bins (a
    4x finer lag grid than the channels give), timed per call with CUDA
    events (the call returns when its peak is on the host)."""
    T, K, Nr, Nd = 256, 1024, 512, 8192
    g = torch.Generator(device=dev)
    g.manual_seed(77)
    V = torch.complex(torch.randn((T, K), generator=g, device=dev), torch.randn((T, K), generator=g, device=dev))
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        corr.fringe_search(V, Nr, Nd)
    torch.cuda.synchronize()
    n = 10
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        corr.fringe_search(V, Nr, Nd)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    # algorithmic bytes: V read, lag transforms written and read, map written and read (peak)
    nbytes = 8.0 * (T * K + 2 * T * Nd + 2 * Nr * Nd)
    flops = 5.0 * (T * Nd * np.log2(Nd) + Nd * Nr * np.log2(Nr))  # radix-2 complex FFT count
    return {"workload": "one baseline: %d sub-integrations x %d channels -> %d rate x %d lag bins" % (T, K, Nr, Nd),
            "ms_per_search": ms, "map_points_per_s": Nr * Nd / (ms / 1e3), "hbm_gbs": nbytes / (ms / 1e3) / 1e9,
            "fft_gflops": flops / (ms / 1e3) / 1e9,
            "timing": "CUDA events around %d calls; each call includes its host read of the peak" % n}


def batch_leg(args, torch, corr, dev):
    """96 uneven scans (2-20 stations, 1-16 subbands, 1-2 pols, 128-8192
    channels, 0.5-30 s): all admitted at once and advanced one integration per
    step, every step one CUDA graph over all open scans, chunk lengths from
    the autotuner, FP16 spectra (chunk length and X unit chosen per shape by the autotuner).  Compared with the same scans one
    after another through corr_correlate_device (same precision and chunks),
    and with plain FP32 one after another at the library's default chunks.
    Samples come from a device-resident pool that every station reads at its
    own offset."""
    import synth
    from paper_1502_06894_gb300 import serve
    mix = synth.scan_mix(seed=4, count=args.batch_scans)
    need = max(max(sc.nsamp) * sc.G // 4 for sc in mix)
    pool = serve.ReplayPool(need + (64 << 20), dev, seed=4)
    limit = args.hbm_cap - args.hbm_reserve - pool.nbytes
    tuner = serve.Autotuner(corr, pool, dev, mem_cap=int(limit / len(mix)))
    TC = corr.CORR_PREC_FP16_TC
    t0 = time.perf_counter()
    for sc in mix:
        tuner.choose(sc, TC)
    tune_s = time.perf_counter() - t0
    samples = sum(sc.stations * sc.G * round(sc.fs * sc.tint) * synth.integrations(sc) for sc in mix)

    def jobs(prec):
        return [serve.Job(q, sc, 0.0, precision=prec) for q, sc in enumerate(mix)]

    ex = serve.GpuExecutor(corr, dev, pool, TC, tuner=tuner, copy_results=False)
    sch = serve.Scheduler(ex, args.hbm_cap, args.hbm_reserve, fixed=pool.nbytes)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = sch.run(jobs(TC))
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    t_scan = serve.serial_run(corr, dev, pool, jobs(TC), TC, tuner=tuner)
    t_fp32 = serve.serial_run(corr, dev, pool, jobs(corr.CORR_PREC_FP32), corr.CORR_PREC_FP32)
    del pool
    torch.cuda.empty_cache()
    return {"workload": "cfg4: %d scans, 2-20 stations, 1-16 subbands, 1-2 pols, 128-8192 channels, 0.5-30 s, "
                        "integrations <= 1 s" % len(mix),
            "station_samples": samples, "integrations": sum(synth.integrations(sc) for sc in mix),
            "value": samples / t_batch, "unit": METRIC, "seconds": t_batch,
            "graph_launches": st["steps"], "max_scans_per_graph": st["max_batch"],
            "peak_job_bytes": st["peak_bytes"], "per_scan_tc": {"value": samples / t_scan, "seconds": t_scan},
            "serial_fp32": {"value": samples / t_fp32, "seconds": t_fp32},
            "batched_vs_per_scan": t_scan / t_batch, "batched_tc_vs_serial_fp32": t_fp32 / t_batch,
            "autotune": {"seconds": tune_s, "trials": tuner.trials, "shapes": len(tuner.cache),
                         "chunk_blocks_chosen": sorted(set(v[0] for v in tuner.cache.values())),
                         "x_unit_chosen": {"cuda_cores": sum(1 for v in tuner.cache.values()
                                                             if v[1] == corr.CORR_X_CUDA_CORES),
                                           "tensor_cores": sum(1 for v in tuner.cache.values()
                                                               if v[1] == corr.CORR_X_TENSOR_CORES)}},
            "timing": "wall clock around the whole run, synchronised, handle set-up included",
            "data": "device-resident random 2-bit pool, per-station offsets (replayed chunk)"}


def serve_point(corr, serve, pool, mix, arrivals, cap, reserve, precision):
    """Submit the jobs at their arrival times (seconds from the start) to the
    native server (corr_server_*) and return its statistics."""
    srv = corr.Server(cap, reserve)
    keep = []
    t0 = time.perf_counter()
    for q, (sc, t) in enumerate(zip(mix, arrivals)):
        wait = t - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        views = [pool.view(q * 1024 + s + 1, sc.nsamp[s] * sc.G // 4) for s in range(sc.stations)]
        st = corr.StaticScan(sc, views)
        keep.append(st)
        srv.submit(st, serve.integrations_of(sc), precision)
    if srv.wait(900.0) != corr.CORR_OK:
        raise RuntimeError("served jobs did not finish")
    st = srv.stats()
    srv.close()
    return st


def serve_leg(args, torch, corr, dev):
    """The native continuous-batching server (corr_server_*): jobs drawn from
    the uneven scan mix arrive as a Poisson process and are admitted by HBM
    budget; every step advances all admitted jobs by one integration in one
    CUDA graph (FP16 spectra, X unit by CORR_X_AUTO) and copies every integration to
    pinned host memory.  A sweep over arrival rates gives offered load,
    served load and p50 / p99 latency (arrival to the last integration)."""
    import synth
    from paper_1502_06894_gb300 import serve
    rates = [float(r) for r in args.serve_rates.split(",")]
    mixes, arrs = [], []
    for k, lam in enumerate(rates):
        arr = serve.poisson_arrivals(lam, args.serve_window, seed=5 + k)
        arrs.append(arr)
        mixes.append(synth.scan_mix(seed=50 + k, count=max(1, len(arr))))
    need = max(max(sc.nsamp) * sc.G // 4 for mix in mixes for sc in mix)
    pool = serve.ReplayPool(need + (64 << 20), dev, seed=5)
    points = []
    for lam, mix, arr in zip(rates, mixes, arrs):
        torch.cuda.synchronize()
        st = serve_point(corr, serve, pool, mix, arr, args.hbm_cap - pool.nbytes, args.hbm_reserve,
                         corr.CORR_PREC_FP16_TC)
        offered = sum(sc.stations * sc.G * round(sc.fs * sc.tint) * synth.integrations(sc) for sc in mix)
        points.append({"rate_jobs_per_s": lam, "jobs": len(arr), "offered": offered / args.serve_window,
                       "served": st["station_samples_per_s"], "p50_s": st["p50_s"], "p99_s": st["p99_s"]})
    del pool
    torch.cuda.empty_cache()
    return {"workload": "cfg5 as a sweep: Poisson arrivals for %.1f s per rate, cfg4 shape mix (2-20 stations, "
                        "1-16 subbands, 1-2 pols, 128-8192 channels, 0.5-30 s), HBM cap %.0f GB, reserve %.0f GB"
                        % (args.serve_window, args.hbm_cap / 1e9, args.hbm_reserve / 1e9),
            "unit": METRIC + " (offered, served); seconds (p50, p99)", "server": "native (corr_server_*)",
            "precision": "FP16 spectra, X unit by CORR_X_AUTO (CUDA cores up to 12 stations, tensor cores above)", "points": points,
            "named_window": "the named run (40 jobs/s for 120 s) offers several times the served load at every "
                            "rate above ~5 jobs/s, so its queue (and p99) grows without bound; the sweep shows "
                            "where the latency is the service time",
            "latency": "submission at the arrival time to the end of the last integration's copy to host memory",
            "data": "device-resident random 2-bit pool, per-station offsets (replayed chunk)"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_1502_06894_gb300 import _build
    _build.build()
    from paper_1502_06894_gb300 import corr

    if args.dense_only:
        res, _ = dense_leg(args, torch, corr, dev)
        print(json.dumps({"dense": res}), flush=True)
        return

    scan = make_scan(args.seed + rank, args.duration)
    nint = int(round(scan.duration / scan.tint))
    gen = torch.Generator(device=dev)
    gen.manual_seed(1000 + args.seed + rank)
    dstreams = [device_codes(scan.nsamp[s] * scan.G // 4, gen, dev) for s in range(scan.stations)]
    in_bytes = sum(int(t.numel()) for t in dstreams)
    torch.cuda.synchronize()
    # a dedicated stream: the library's launches and the timing events share it
    stream = torch.cuda.Stream(device=dev)

    out = torch.empty((nint, scan.nbl, scan.G, scan.nchan), dtype=torch.complex64, device=dev)
    wts = torch.empty((nint, scan.nbl), dtype=torch.float64, device=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def device_leg(precision, pipeline=1, unit=0):
        """Time K steps of the device-resident path at one precision (and,
        for FP16 / FP8, one X unit)."""
        c = corr.from_scan(scan, device_streams=dstreams)
        if args.chunk_blocks:
            c.set_chunk_blocks(args.chunk_blocks)
        c.set_precision(precision)
        c.set_x_unit(unit)
        c.set_pipeline(pipeline)
        c.set_stream(stream.cuda_stream)
        c.flush()

        def step():
            c.rewind()
            for i in range(nint):
                rc = c.correlate_device(out[i], wts[i])
                if rc != corr.CORR_OK:
                    raise RuntimeError("correlate_device returned %d" % rc)

        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        c.read_profile()
        c.set_profiling(True)
        clk = Clocks(dev.index)
        barrier()
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1) / args.steps
        prof = c.read_profile()
        shape = c.launch_shape()
        c.close()
        ms = max_over_ranks(ms, dev)
        return ms, prof, clocks, shape

    ms, prof_ovl, clocks, (cb, kz) = device_leg(corr.CORR_PREC_FP32)
    sps = samples_per_step(scan)
    value = replica_value(sps, ws, ms)
    # the same step with F and X in turn on one stream: each kernel's launch
    # time then is its own (with the overlap, F launches share SMs with X), so
    # this leg gives the per-kernel roofline
    ms_seq, prof, clocks_seq, _ = device_leg(corr.CORR_PREC_FP32, pipeline=0)
    # FP16 / FP8 spectra: the library's own choice of X unit (for 10
    # stations the CUDA cores), and the tensor cores forced
    # (each also with F and X in turn, for the per-kernel stage times)
    tc = tc_mma = None
    seq = {}
    if not args.no_tc:
        ms_tc, prof_tc, clocks_tc, _ = device_leg(corr.CORR_PREC_FP16_TC)
        ms_tcm, prof_tcm, clocks_tcm, _ = device_leg(corr.CORR_PREC_FP16_TC, unit=corr.CORR_X_TENSOR_CORES)
        seq["tc"] = device_leg(corr.CORR_PREC_FP16_TC, pipeline=0)[:2]
        seq["tc_mma"] = device_leg(corr.CORR_PREC_FP16_TC, pipeline=0, unit=corr.CORR_X_TENSOR_CORES)[:2]
    fp8 = fp8_mma = None
    if not args.no_fp8:
        ms_f8, prof_f8, clocks_f8, _ = device_leg(corr.CORR_PREC_FP8_TC)
        ms_f8m, prof_f8m, clocks_f8m, _ = device_leg(corr.CORR_PREC_FP8_TC, unit=corr.CORR_X_TENSOR_CORES)
        seq["fp8"] = device_leg(corr.CORR_PREC_FP8_TC, pipeline=0)[:2]
        seq["fp8_mma"] = device_leg(corr.CORR_PREC_FP8_TC, pipeline=0, unit=corr.CORR_X_TENSOR_CORES)[:2]

    # ---- roofline of the dominant kernel ----
    peak_hbm, peak_src = measured_peaks()
    S, G, N, nch = scan.stations, scan.G, scan.N, scan.nchan
    nbl = scan.nbl
    spi = int(round(scan.fs * scan.tint))
    blocks_per_step = sum(-(-(i + 1) * spi // N) - (-(-i * spi // N)) for i in range(nint))
    ss_step = blocks_per_step * S * G * N  # station-samples transformed per step
    steps = args.steps
    f_ms, f_n = prof["fstage"]
    x_ms, x_n = prof["xstage"]
    f_bytes = steps * ss_step * (0.25 + 4.0)
    f_flops = steps * blocks_per_step * S * G * (2.5 * N * np.log2(N))
    x_bytes = steps * (ss_step * 4.0 + (x_n / max(steps, 1)) * kz * nbl * G * nch * 16.0)
    x_flops = steps * blocks_per_step * G * nch * nbl * 8.0
    peak_alu = SM_COUNT * FP32_LANES * 2 * MAX_SM_MHZ * 1e6
    stages = {}
    for name, (tms, n) in prof.items():
        stages[name] = {"ms_per_step": tms / steps, "launches_per_step": n / steps}
    dom = "fstage" if f_ms >= x_ms else "xstage"
    if dom == "fstage":
        d_ms, d_n, d_bytes, d_flops = f_ms, f_n, f_bytes, f_flops
    else:
        d_ms, d_n, d_bytes, d_flops = x_ms, x_n, x_bytes, x_flops
    t_launch = d_ms / 1e3 / max(d_n, 1)
    gbs = d_bytes / max(d_n, 1) / t_launch / 1e9
    tfl = d_flops / max(d_n, 1) / t_launch / 1e12
    hbm_frac = gbs / peak_hbm
    alu_frac = tfl * 1e12 / peak_alu
    if hbm_frac >= alu_frac:
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak_hbm, "unit": "GB/s", "frac": hbm_frac,
                "traffic": None, "peak_source": peak_src}
    else:
        roof = {"bound": "alu", "achieved": tfl, "peak": peak_alu / 1e12, "unit": "TFLOP/s", "frac": alu_frac,
                "traffic": None, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}
    gc = G if G in (16, 32) else 0
    kname = "k_fstage<%d,%d>" % (nch, gc) if dom == "fstage" else "k_xmac_tma<%d>" % S
    traffic = traffic_per_launch(kname)
    roof["traffic"] = traffic
    roof["traffic_over_algorithmic"] = (traffic / (d_bytes / max(d_n, 1))) if traffic else None
    roof.update({"kernel": kname,
                 "bytes_per_launch": d_bytes / max(d_n, 1), "flops_per_launch": d_flops / max(d_n, 1),
                 "launch_ms": t_launch * 1e3, "hbm_frac": hbm_frac, "alu_frac": alu_frac})
    # the F step is bound by instruction issue: its warp instructions per
    # launch (ncu) against the issue ceiling at the SM clock seen under load
    inst = profile_value("instructions.txt", kname)
    roof["warp_instructions"] = inst
    roof["issue_frac"] = issue_frac(inst, t_launch, (clocks or {}).get("sm_mhz") or MAX_SM_MHZ)
    launches = prof_ovl["delay"][1] + prof_ovl["fstage"][1] + prof_ovl["xstage"][1] + 2 * prof_ovl["finalize"][1]
    x_tflops = x_flops / (x_ms / 1e3) / 1e12 if x_ms > 0 else None
    def tc_leg(ms_t, prof_t, clocks_t, dtype, elem_bytes, bound, unit, sq):
        xt_ms, xt_n = prof_t["xstage"]
        ft_ms, ft_n = prof_t["fstage"]
        # reduced-precision spectra: elem_bytes read per station-sample in the X step
        xt_bytes = steps * ss_step * elem_bytes
        return {"value": replica_value(sps, ws, ms_t), "unit": METRIC, "ms_per_step": ms_t, "dtype": dtype,
                "x_unit": unit, "error_bound_rel_rms": bound, "measured_rel_rms": None,
                "xstep_ms_per_step": xt_ms / steps, "fstage_ms_per_step": ft_ms / steps,
                "xstep_tflops": x_flops / (xt_ms / 1e3) / 1e12 if xt_ms > 0 else None,
                "xstep_hbm_gbs": xt_bytes / (xt_ms / 1e3) / 1e9 if xt_ms > 0 else None,
                "xstep_vs_fp32_xstep": (x_ms / xt_ms) if xt_ms > 0 else None,
                "stages": {k: {"ms_per_step": v[0] / steps, "launches_per_step": v[1] / steps}
                           for k, v in prof_t.items()},
                "sequential": {"ms_per_step": sq[0],
                               "stages": {k: {"ms_per_step": v[0] / steps, "launches_per_step": v[1] / steps}
                                          for k, v in sq[1].items()}},
                "clocks": clocks_t}

    auto_unit = "CUDA cores (CORR_X_AUTO: %d stations <= 12)" % S if S <= 12 else "tensor cores (CORR_X_AUTO)"
    if not args.no_tc:
        tc = tc_leg(ms_tc, prof_tc, clocks_tc, "f16 in, f32 accumulate", 2.0, 1e-3, auto_unit, seq["tc"])
        tc_mma = tc_leg(ms_tcm, prof_tcm, clocks_tcm, "f16 in, f32 accumulate", 2.0, 1e-3,
                        "tensor cores (CORR_X_TENSOR_CORES)", seq["tc_mma"])
    if not args.no_fp8:
        fp8 = tc_leg(ms_f8, prof_f8, clocks_f8, "e4m3 in, f32 accumulate", 1.0, 8e-2, auto_unit, seq["fp8"])
        fp8_mma = tc_leg(ms_f8m, prof_f8m, clocks_f8m, "e4m3 in, f32 accumulate", 1.0, 8e-2,
                         "tensor cores (CORR_X_TENSOR_CORES)", seq["fp8_mma"])

    # ---- end to end through the host API ----
    # The inputs live in pinned host memory and every step moves them to the
    # GPU inside the timed region.  Default ("zero-copy"): the stations' pinned
    # buffers are attached with corr_attach_samples_host and the F kernel reads
    # them over NVLink-C2C as it stages each window (each byte crosses once);
    # on this platform a host->device copy occupies the SMs for its whole
    # duration (~211 GB/s), so reading in place lets the transfer hide under
    # the F kernel's arithmetic.  "copy": corr_push_samples_async pieces pushed
    # ahead of the integrations that need them.  Results go back to pinned host
    # memory with corr_correlate.
    e2e = None
    e2e_copy = None
    if not args.no_e2e:
        host = [torch.empty(t.numel(), dtype=torch.uint8, pin_memory=True) for t in dstreams]
        for h, t in zip(host, dstreams):
            h.copy_(t)
        out_h = torch.empty((nint, nbl, G, nch), dtype=torch.complex64, pin_memory=True)
        w_h = torch.empty((nint, nbl), dtype=torch.float64, pin_memory=True)
        d2h = int(out_h[0].numel() * 8 * nint + w_h.numel() * 8)

        def timed(fn, n):
            fn()
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            for _ in range(n):
                fn()
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / n
            return max_over_ranks(dt, dev)

        def correlate_all(cc):
            for i in range(nint):
                rc = cc.correlate_into(out_h[i], w_h[i])
                if rc != corr.CORR_OK:
                    raise RuntimeError("corr_correlate returned %d" % rc)

        c2 = corr.from_scan(scan)
        if args.chunk_blocks:
            c2.set_chunk_blocks(args.chunk_blocks)

        def e2e_zero_copy():
            c2.reset()
            for s in range(S):
                c2.attach_host(s, host[s])
            c2.flush()
            correlate_all(c2)

        ne = max(2, min(args.steps, 5))
        dt = timed(e2e_zero_copy, ne)
        e2e = {"value": replica_value(sps, ws, dt * 1e3), "unit": METRIC, "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": d2h,
               "ms_per_step": dt * 1e3, "steps": ne,
               "mode": "zero-copy: pinned host buffers attached, read by the F kernel over NVLink-C2C"}
        c2.close()

        c3 = corr.from_scan(scan)
        if args.chunk_blocks:
            c3.set_chunk_blocks(args.chunk_blocks)
        for s in range(S):
            c3.reserve(s, host[s].numel())
        pieces = []
        for s in range(S):
            nb = host[s].numel()
            cuts = [((nb * k) // nint) // 4 * 4 for k in range(nint)] + [nb]
            pieces.append([host[s][cuts[k]:cuts[k + 1]] for k in range(nint)])

        def e2e_copy_step():
            c3.reset()
            pushed = 0

            def push_next():
                nonlocal pushed
                if pushed < nint:
                    for s in range(S):
                        c3.push_async(s, pieces[s][pushed])
                    pushed += 1
                    if pushed == nint:
                        c3.flush()
                    return True
                return False

            push_next()
            push_next()
            for i in range(nint):
                push_next()
                while True:
                    rc = c3.correlate_into(out_h[i], w_h[i])
                    if rc == corr.CORR_OK:
                        break
                    if rc != corr.CORR_EAGAIN or not push_next():
                        raise RuntimeError("corr_correlate returned %d" % rc)
            c3.wait_pushes()

        dt = timed(e2e_copy_step, ne)
        e2e_copy = {"value": replica_value(sps, ws, dt * 1e3), "unit": METRIC, "ms_per_step": dt * 1e3, "h2d_bytes_per_step": in_bytes,
                    "mode": "copy: corr_push_samples_async pieces two integrations ahead"}
        c3.close()

    batch = None
    served = None
    dense = None
    dense_sample = None
    fringe = None
    peaks = None
    if rank == 0 and ws == 1:
        # free the single-scan buffers first: the mix brings its own pool
        del out, wts
        torch.cuda.empty_cache()
        if not args.no_dense:
            dense, dense_sample = dense_leg(args, torch, corr, dev)
        if not args.no_fringe:
            fringe = fringe_leg(args, torch, corr, dev)
        if not args.no_peaks:
            peaks = peaks_leg(args, torch, dev)
        if not args.no_batch:
            batch = batch_leg(args, torch, corr, dev)
        if not args.no_serve:
            served = serve_leg(args, torch, corr, dev)

    # ---- CPU oracle on a bounded sample; its visibilities also give the
    #      measured error of every precision on the benchmarked workloads ----
    cpu = None
    measured = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        hs = host_stream_prefix(dstreams, scan)
        r, cores, dt, wmin, ref = cpu_oracle_sample(scan, hs)
        cpu = {"value": r, "unit": METRIC, "cores": cores, "kind": "oracle",
               "sample": "first %.1f s of the scan as one integration, all stations and streams (%.1f s wall)"
                         % (CPU_SAMPLE_S, dt)}
        measured = {"sample": "first %.1f s of the benchmarked scan as one integration, all 16 streams; "
                              "max over the 55 baselines of the relative RMS vs the FP64 oracle" % CPU_SAMPLE_S,
                    **sample_errors(corr, scan, hs, ref)}
        if tc is not None:
            tc["measured_rel_rms"] = measured["fp16"]
            tc_mma["measured_rel_rms"] = measured["fp16_tensor_cores"]
        if fp8 is not None:
            fp8["measured_rel_rms"] = measured["fp8"]
            fp8_mma["measured_rel_rms"] = measured["fp8_tensor_cores"]
        if dense is not None and dense_sample is not None:
            dsc, dprefix = dense_sample
            r2, cores2, dt2, _, dref = cpu_oracle_sample(dsc, dprefix, DENSE_SAMPLE_S, DENSE_SAMPLE_STREAMS)
            derr = sample_errors(corr, dsc, dprefix, dref, DENSE_SAMPLE_S, units=(0,))
            for name in ("fp32", "fp16", "fp8"):
                dense[name]["measured_rel_rms"] = derr[name]
            dense["measured_error_sample"] = ("first %.3f s of the 64-station scan as one integration, streams 0-%d; "
                                              "max over the 2080 baselines; oracle %.1f s on %d cores"
                                              % (DENSE_SAMPLE_S, DENSE_SAMPLE_STREAMS - 1, dt2, cores2))

    if peaks and peaks.get("fp32_tflops"):
        # the F step's flops against the measured FP32 throughput as well
        roof["alu_peak_measured_tflops"] = peaks["fp32_tflops"]
        roof["alu_frac_of_measured"] = roof["flops_per_launch"] / (roof["launch_ms"] / 1e3) / 1e12 / peaks["fp32_tflops"]
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "stations": S, "subbands": scan.nsub, "pols": scan.npol,
                           "nchan": nch, "fft": N, "duration_s": scan.duration, "tint_s": scan.tint,
                           "station_samples_per_step": sps, "input_bytes": in_bytes,
                           "l2": "inputs %.1f GB > 129 MB L2 (no flush needed)" % (in_bytes / 1e9),
                           "chunk_blocks": cb, "x_partials": kz,
                           "parallelism": "replicas x%d" % ws},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "measured_rel_rms": measured,
                "clocks": clocks, "stages": stages,
                "schedule": {"value": "two streams: X of chunk c overlaps F of chunk c+1, delay blocks one "
                                      "integration ahead",
                             "roofline_and_stages": "F and X in turn on one stream (each launch timed alone)",
                             "sequential_ms_per_step": ms_seq,
                             "overlapped_stages": {k: {"ms_per_step": v[0] / args.steps,
                                                       "launches_per_step": v[1] / args.steps}
                                                   for k, v in prof_ovl.items()}},
                "xstep_tflops": x_tflops, "tc": tc, "tc_tensor_cores": tc_mma, "fp8": fp8,
                "fp8_tensor_cores": fp8_mma, "e2e_copy": e2e_copy,
                "dense": dense, "fringe": fringe, "batch": batch, "serve": served, "peaks": peaks}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
