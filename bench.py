"""Benchmark of the GB300 APAX codec hot path.

One step = the whole hot path over one synthetic array resident in HBM:
profiler sweep (16 power-of-two attenuation codes, exact sizes and
reconstruction sums, recommendation at r >= 0.9999) -> fixed-quality encode
at the recommended code (read on the device) -> decode.  Workload: the
float32 4096x4096 k^-3 random field.  `value` is GB/s of uncompressed data
through the step (median of K steps), which is captured once as a CUDA
graph and replayed (L2 flushed before each timed replay); encode, decode and
profile are also timed on their own (medians of max(K, 20) calls), and
`roofline` gives the HBM fraction of the one with the largest time.  `e2e`
runs the step from pinned host memory through the public calls: the
host-input sweep (the array crosses in pieces on a copy stream while pieces
already there are swept), encode, decode, and the copy of the container, the
profile points and the decoded array back; two steps are in flight (a
stream of arrays), and the one-step-at-a-time time is reported beside it.
`cpu_baseline` is the oracle on every host core (threads over block ranges)
and, beside it, on one core.  Every workload's results carry
`input_sha256`, the fingerprint of its generated inputs.
At N = 1 the default run also measures (`workloads`) the int16 sensor trace
at 4:1, the float64 512^3 field, the version-2 container formats, the
batched workload (all 8,192 arrays, 3 timed runs of each operation) and the
serving workload (10 s of arrivals).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload field|sensor|field3d|batched|serving]

With N > 1 (torchrun), every rank codes its own array (weak scaling, no
data-path collective); rank 0 prints max-over-ranks timing.

Other workloads (one GPU):
  batched  8,192 arrays (4 KB..64 MB, int16/int32/float32/float64, fixed
           rates 2:1..6:1, 56.6 GB): one persistent launch each for encode,
           decode and the profiler sweep, against the plain per-array loop.
  sensor   int16 trace at 4:1: single-call latency, and GB/s on 8,192 copies.
  field3d  float64 512^3 field (1 GiB): profile -> fixed quality -> decode.
  serving  Poisson arrivals (2,000 requests/s for --serve-seconds, 50/50 encode/decode, 64 KB..
           256 MB of float32 field slices at a fixed quality or int16 traces
           at 4:1) through the request server with a 64 GB admission cap:
           open-loop p50/p99 latency, then a closed-loop replay of the same
           trace against the plain per-request path.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encode/decode GB/s (uncompressed) and % of GB300 HBM roofline at ratio/corr"
WORKLOAD = "float32 4096x4096 k^-3 random field (seed 1): profile 16 codes -> fixed-quality encode at r>=0.9999 -> decode"
TARGET = 0.9999
N_BLOCK = 256
E2E_CHUNKS = 16  # pieces of the host-to-device copy that the sweep overlaps


CPU_ROWS = 1024  # rows of the field in the oracle's timed sample (16 MiB)
CPU_ROWS_1CORE = 256  # rows in the single-core sample (4 MiB)


def _profile_figure(kernel, key=None):
    """Figures of the committed ncu summary of this workload
    (profiles/traffic_f32_4096x4096.txt): 'kernel bytes' lines give the DRAM
    read + write bytes of one launch, 'issue_active kernel frac' lines the
    issue-active fraction per scheduler, 'fma_heavy kernel frac' lines the
    FMA-heavy pipe's busy fraction of peak."""
    path = os.path.join(ROOT, "profiles", "traffic_f32_4096x4096.txt")
    try:
        with open(path) as f:
            for ln in f:
                parts = ln.split()
                if key is None and len(parts) == 2 and parts[0] == kernel:
                    return int(parts[1])
                if key is not None and len(parts) == 3 and parts[0] == key and parts[1] == kernel:
                    return float(parts[2])
    except OSError:
        pass
    return None


def _traffic(kernel):
    return _profile_figure(kernel)


def _issue_active(kernel):
    return _profile_figure(kernel, "issue_active")


def _fma_heavy(kernel):
    return _profile_figure(kernel, "fma_heavy")


def _events(fn, reps, stream, flush=None):
    """CUDA-event times (ms) of `reps` calls of fn on `stream`, each after an
    optional L2 flush (outside the events)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for a, b in ev:
        if flush is not None:
            flush.zero_()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def _median(v):
    return float(np.median(np.asarray(v, dtype=np.float64)))


def cpu_model():
    """The host CPU's model name (lscpu), or the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the sampler takes a moment to start: let it report before timing
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:
                time.sleep(0.01)
            self.lines.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(values, device, world):
    """Timings of every rank -> the slowest rank's, on every rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def aggregate_gbs(bytes_per_rank, world, ms):
    """Whole-job throughput: every rank's bytes over the slowest rank's time."""
    return world * bytes_per_rank / ms / 1e6


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_1303_4994_gb300 import apax as A
    from paper_1303_4994_gb300 import build as B
    from paper_1303_4994_gb300 import synth

    B.build()
    A.lib()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    x_host = synth.grf2d(4096, 4096, seed=1 + rank)
    n = x_host.size
    xb = x_host.nbytes
    x = torch.from_numpy(x_host.reshape(-1)).to(dev)
    stream = torch.cuda.current_stream(dev)

    cands = list(A.DEFAULT_CANDIDATES)
    nc = len(cands)
    pws, pts, summ = A.profile_buffers(x, N_BLOCK, nc)
    p = A.params(N_BLOCK, A.FIXED_QUALITY)
    cap = A.encoded_size(A.F32, n, p)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    ews = torch.empty(A.workspace_size(A.F32, n, p), dtype=torch.uint8, device=dev)
    dws = torch.empty(A.decode_workspace_size(), dtype=torch.uint8, device=dev)
    eres, dres = A.new_result(dev), A.new_result(dev)
    y = torch.empty_like(x)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    # each call goes on the current stream (the capture stream while the
    # step is captured into a CUDA graph)
    def prof():
        A.profile_into(x, N_BLOCK, cands, TARGET, pws, pts, summ)

    def enc():
        A.encode_into(x, p, out, ews, eres, summary=summ)

    def dec():
        A.decode_into(out, y, dws, dres)

    def step():
        prof()
        enc()
        dec()

    # profile (the one-block-per-thread sweep, the fix-up sweep of the runs it
    # marks, the tree with the finalisation), encode, decode (two size classes)
    launches_per_step = _profile_launches(n, A.F32) + 1 + 2

    # the whole step (memsets and kernels of the three calls) as one CUDA
    # graph: the timed step replays it, without per-launch gaps (one eager
    # step first loads the kernels and sets their attributes)
    step()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    torch.cuda.synchronize()
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        graph.replay()
    torch.cuda.synchronize()
    s = A.read_summary(summ)
    er, dr = A.read_result(eres), A.read_result(dres)
    assert s.status == 0 and er.status == 0 and dr.status == 0, (s.status, er.status, dr.status)
    pt = A.read_points(pts, nc)[s.recommended]
    ratio = xb / er.bytes
    met = A.derived(pt, n)

    # per-call timings: at least 20 runs each (median), on the launching stream
    reps = max(args.steps, 20)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local_rank) as clk:
        t_step = _events(graph.replay, args.steps, stream, flush)
        t_prof = _events(prof, reps, stream, flush)
        t_enc = _events(enc, reps, stream, flush)
        t_dec = _events(dec, reps, stream, flush)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = _median(t_step)
    ms_prof, ms_enc, ms_dec = (_median(t) for t in (t_prof, t_enc, t_dec))

    # the profiler's windows 3 and 4 at the recommended point (x against the
    # decoded y): 2-sigma S2R margin and spectral levels, timed on their own
    qws = A.aligned_workspace(A.quality_workspace_size(A.F32, n), dev)
    qbuf = torch.zeros(ctypes.sizeof(A.Quality), dtype=torch.uint8, device=dev)
    A.quality_into(x, y, qws, qbuf)
    torch.cuda.synchronize()
    t_q = _events(lambda: A.quality_into(x, y, qws, qbuf), 5, stream, flush)
    qdb = A.quality_db(A.read_quality(qbuf))

    # end to end through the C ABI with host buffers: the host-input sweep
    # (H2D of x in pieces on a copy stream, hidden behind the sweep), encode,
    # decode, D2H of the container, the profile points and the decoded array.
    # Two slots (buffers and streams of their own) keep two steps in flight,
    # as a stream of arrays would: step i + 1's input crosses the host link
    # while step i's results come back (the link carries both directions at
    # once; within a step the copies cannot overlap, y exists only after the
    # sweep of all of x).  Every step copies its whole input in and its
    # results out.  The one-step-at-a-time time is reported beside it.
    xh = torch.from_numpy(x_host.reshape(-1)).pin_memory()

    class Slot:
        pass

    slots = []
    for _ in range(2):
        sl = Slot()
        sl.x = torch.empty_like(x)
        sl.pws, sl.pts, sl.summ = A.profile_buffers(sl.x, N_BLOCK, nc)
        sl.out = torch.empty(cap, dtype=torch.uint8, device=dev)
        sl.ews = torch.empty_like(ews)
        sl.dws = torch.empty_like(dws)
        sl.eres, sl.dres = A.new_result(dev), A.new_result(dev)
        sl.y = torch.empty_like(x)
        sl.outh = torch.empty(cap, dtype=torch.uint8).pin_memory()
        sl.ptsh = torch.empty_like(pts, device="cpu").pin_memory()
        sl.yh = torch.empty_like(x, device="cpu").pin_memory()
        sl.stream = torch.cuda.Stream(device=dev)
        sl.copy = torch.cuda.Stream(device=dev)
        sl.done = None
        slots.append(sl)

    def e2e_step(sl):
        with torch.cuda.stream(sl.stream):
            A.profile_from_host_into(xh, sl.x, N_BLOCK, cands, TARGET, sl.pws, sl.pts, sl.summ,
                                     sl.stream, sl.copy, chunks=E2E_CHUNKS)
            A.encode_into(sl.x, p, sl.out, sl.ews, sl.eres, summary=sl.summ)
            encoded = torch.cuda.Event()
            encoded.record(sl.stream)
            # the container goes to the host while the decode runs: its size
            # is read on the device (apax_copy_container), so no host wait
            sl.copy.wait_event(encoded)
            A.copy_container_into(sl.out, sl.eres, sl.outh, sl.copy)
            with torch.cuda.stream(sl.copy):
                sl.ptsh.copy_(sl.pts, non_blocking=True)
            A.decode_into(sl.out, sl.y, sl.dws, sl.dres)
            sl.yh.copy_(sl.y, non_blocking=True)
            joined = torch.cuda.Event()
            joined.record(sl.copy)
            sl.stream.wait_event(joined)
            sl.done = torch.cuda.Event()
            sl.done.record(sl.stream)

    # one step at a time
    lat_ms = []
    for i in range(args.steps + 2):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step(slots[0])
        torch.cuda.synchronize()
        if i >= 2:
            lat_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_lat = _median(lat_ms)
    # two in flight: K steps after two untimed ones, the host waiting only
    # for a slot's previous step before reusing its buffers
    for i in range(2):
        e2e_step(slots[i % 2])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        sl = slots[i % 2]
        sl.done.synchronize()
        e2e_step(sl)
    torch.cuda.synchronize()
    e2e = (time.perf_counter() - t0) * 1e3 / args.steps
    for sl in slots:
        er_len = A.read_result(sl.eres).bytes
        assert torch.equal(sl.yh.view(torch.int32), y.view(torch.int32).cpu())
        assert torch.equal(sl.outh[:er_len], out[:er_len].cpu())
        assert torch.equal(sl.ptsh, pts.cpu())

    ms, ms_prof, ms_enc, ms_dec, e2e, e2e_lat = max_over_ranks([ms, ms_prof, ms_enc, ms_dec, e2e, e2e_lat],
                                                            dev, world)

    peak, peak_kind = _peaks()
    enc_bytes = xb + er.bytes
    dec_bytes = er.bytes + xb
    prof_bytes = xb
    kern = {
        "profile": {"ms": ms_prof, "gbs": prof_bytes / ms_prof / 1e6},
        "encode": {"ms": ms_enc, "gbs": enc_bytes / ms_enc / 1e6, "uncompressed_gbs": xb / ms_enc / 1e6},
        "decode": {"ms": ms_dec, "gbs": dec_bytes / ms_dec / 1e6, "uncompressed_gbs": xb / ms_dec / 1e6},
    }
    for k in kern.values():
        k["frac_hbm"] = k["gbs"] / peak
    # the roofline of the kernel with the largest share of the step: its
    # algorithmic bytes (read s per element, plus the container for encode
    # and decode) over its CUDA-event time, against the measured copy peak;
    # ncu's issue-active fraction of the same kernel and the busy fraction of
    # its busiest pipe (the FMA-heavy pipe of the integer multiply-adds) sit
    # beside it: the sweep is bound by integer issue, not by HBM
    dom = max(kern, key=lambda k: kern[k]["ms"])
    alg = {"profile": prof_bytes, "encode": enc_bytes, "decode": dec_bytes}[dom]
    roof = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["gbs"], "peak": peak,
            "unit": "GB/s", "frac": kern[dom]["gbs"] / peak, "traffic": _traffic(dom),
            "algorithmic_bytes": alg, "ms": kern[dom]["ms"],
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
            "ncu_issue_active": _issue_active(dom), "ncu_fma_heavy_pipe": _fma_heavy(dom)}
    line = {
        "metric": METRIC,
        "value": round(aggregate_gbs(xb, world, ms), 3),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(args.warmup, 3),
        "ms_per_step": round(ms, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "elements": n, "block_size": N_BLOCK, "candidates": nc,
                   "input_sha256": synth.sha256(x_host),
                   "target_corr": TARGET, "l2": "flushed (512 MB write) before every timed step",
                   "launch": "each step replays one CUDA graph of the three calls",
                   "timing": "median of K step times; per-call medians of max(K, 20) runs",
                   "parallelism": f"independent arrays per GPU x{world}"},
        "ratio": round(ratio, 4),
        "corr": pt.r,
        "recommended_code": int(s.recommended_code),
        "snr_db": met["snr_db"],
        "encode_gbs": round(kern["encode"]["uncompressed_gbs"] * world, 2),
        "decode_gbs": round(kern["decode"]["uncompressed_gbs"] * world, 2),
        "kernels": kern,
        "quality_db": {k: (round(v, 4) if abs(v) != float("inf") else str(v)) for k, v in qdb.items()},
        "quality_ms": round(_median(t_q), 4),
        "roofline": roof,
        "e2e": {"value": round(world * xb / e2e / 1e6, 3), "unit": "GB/s",
                "h2d_bytes_per_step": xb,
                "d2h_bytes_per_step": er.bytes + pts.numel() + y.numel() * y.element_size(),
                "ms_per_step": round(e2e, 4),
                "ms_one_step_at_a_time": round(e2e_lat, 4),
                "path": "apax_profile_from_host (H2D in 16 pieces under the sweep) -> "
                        "apax_encode_recommended -> apax_copy_container to pinned host "
                        "memory (size read on the device) beside apax_decode -> D2H of points "
                        "and decoded array; two steps in flight (own buffers and streams "
                        "each), K steps timed as one span after two untimed; every step "
                        "copies its input in and its results out, no L2 flush between them "
                        "(each step's input arrives by a fresh host copy); "
                        "ms_one_step_at_a_time: median of K single steps, L2 flushed"},
        # timed region: K graph replays of the step, then max(K, 20) profile,
        # encode and decode calls each
        "gpu_launches": (args.steps + reps) * launches_per_step,
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_baseline"]["single_core"] = cpu_baseline(rows=CPU_ROWS_1CORE, threads=None)
    if world == 1 and rank == 0 and not args.no_extra:
        # the other single-GPU workloads, measured in the same run
        import torch
        wl = {}
        for name, fn in (("sensor_i16_fr4", lambda: run_sensor(args, compact=True)),
                         ("field3d_f64_512", lambda: run_field3d(args, compact=True)),
                         ("formats_v2", lambda: run_formats(args)),
                         ("batched_8192", lambda: run_batched(args, compact=True)),
                         ("serving", lambda: run_serving(args, compact=True))):
            wl[name] = fn()
            torch.cuda.empty_cache()  # the next workload's arrays need the room
        line["workloads"] = wl
    return line


def cpu_baseline(rows: int = CPU_ROWS, threads=0, x=None):
    """The oracle, as it stands, on a bounded slice of the same workload:
    profile (16 codes) + fixed-quality encode at the recommended code +
    decode of the first `rows` rows of the field; threads=0 runs its
    threaded drivers on every host core (contiguous block ranges), None its
    plain sequential calls on one core."""
    import oracle as O
    from paper_1303_4994_gb300 import synth

    if x is None:
        x = synth.grf2d(4096, 4096, seed=1)[:rows].copy()
    cores = 1 if threads is None else O.threads(threads)
    t0 = time.perf_counter()
    pts, rec, _ = O.profile(x, N=N_BLOCK, target=TARGET, threads=threads)
    c = O.encode(x, N_BLOCK, O.MODE_FQ, 1, 1, pts[rec].code, threads=threads)
    O.decode(c, np.float32, x.size, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": round(x.nbytes / dt / 1e9, 6), "unit": "GB/s", "cores": cores,
            "kind": "oracle", "cpu": cpu_model(), "nproc": os.cpu_count(),
            "sample": f"first {rows} rows ({x.nbytes >> 20} MiB) of the field: profile 16 codes "
                      f"+ encode + decode, {'all cores, threads over block ranges' if cores > 1 else 'one core'}",
            "seconds": round(dt, 2)}


def oracle_codec(x, mode, num, den, code, sample):
    """The oracle's encode and decode GB/s of uncompressed data on a bounded
    sample x (host array) of a workload, on every host core (threads over
    block ranges) and on one core; a baseline beside the GPU numbers."""
    import oracle as O

    out = {"unit": "GB/s", "kind": "oracle", "cpu": cpu_model(), "nproc": os.cpu_count(),
           "sample": sample}
    for name, threads in (("all_cores", 0), ("one_core", None)):
        t0 = time.perf_counter()
        c = O.encode(x, N_BLOCK, mode, num, den, code, threads=threads)
        t1 = time.perf_counter()
        O.decode(c, x.dtype, x.size, threads=threads)
        t2 = time.perf_counter()
        out[name] = {"encode": round(x.nbytes / (t1 - t0) / 1e9, 5),
                     "decode": round(x.nbytes / (t2 - t1) / 1e9, 5),
                     "cores": 1 if threads is None else O.threads(threads)}
    return out


def run_reference(args, rank, world):
    """The reference arm: the oracle (the paper has no code to install) on
    the host cores, on the same sample as cpu_baseline, one sample per step."""
    if rank != 0:
        return None
    from paper_1303_4994_gb300 import synth
    x = synth.grf2d(4096, 4096, seed=1)[:CPU_ROWS].copy()
    steps = []
    for i in range(max(args.warmup, 0) + args.steps):
        cb = cpu_baseline(rows=CPU_ROWS, x=x)
        if i >= args.warmup:
            steps.append(cb)
    v = _median([s["value"] for s in steps])
    ms = _median([s["seconds"] * 1e3 for s in steps])
    return {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": steps[-1]["sample"]},
            "cpu_baseline": {"value": round(v, 6), "unit": "GB/s", "cores": steps[-1]["cores"],
                             "kind": "oracle", "cpu": steps[-1]["cpu"],
                             "sample": steps[-1]["sample"]},
            "e2e": {"value": round(v, 6), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def _profile_launches(n, dtype_code):
    """Kernels of one apax_profile call at block size N_BLOCK: the float32
    one-block-per-thread sweep and its fix-up sweep, or the team sweep;
    then one tree launch."""
    t1 = dtype_code == 4 and (n + N_BLOCK - 1) // N_BLOCK >= 16384 and N_BLOCK <= 256
    return (2 if t1 else 1) + 1


def _wrapped(master, off, n):
    import torch
    M = master.numel()
    pos, parts, need = off % M, [], n
    while need > 0:
        take = min(need, M - pos)
        parts.append(master[pos:pos + take])
        need -= take
        pos = 0
    return torch.cat(parts) if len(parts) > 1 else parts[0].clone()


def run_batched(args, compact=False):
    """The batched workload (8,192 arrays, 56.6 GB by default): one persistent
    launch per operation against the plain per-array loop.  compact: the
    default run's version, 3 timed repetitions of each of the six runs and a
    short summary."""
    import torch

    from paper_1303_4994_gb300 import apax as A
    from paper_1303_4994_gb300 import build as B
    from paper_1303_4994_gb300 import synth

    B.build()
    A.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    specs = synth.batch_specs(args.arrays)
    masters_h = synth.batch_masters()
    # every array is a wrapped slice of a master: the masters and the job
    # table (dtype, length, rate, offset) fix all 56.6 GB of input
    in_sha = synth.sha256(*[masters_h[k] for k in sorted(masters_h)], repr(specs))
    masters = {k: torch.from_numpy(v).to(dev) for k, v in masters_h.items()}
    del masters_h
    xs = [_wrapped(masters[dt], off, n) for dt, n, _, off in specs]
    ps = [A.params(N_BLOCK, A.FIXED_RATE, rate, 0) for _, _, rate, _ in specs]
    total = sum(x.numel() * x.element_size() for x in xs)
    caps = [A.encoded_size(A.TORCH_CODE[x.dtype], x.numel(), p) for x, p in zip(xs, ps)]
    outs = [torch.empty(c, dtype=torch.uint8, device=dev) for c in caps]
    outs_plain = [torch.empty(c, dtype=torch.uint8, device=dev) for c in caps]
    ys = [torch.empty_like(x) for x in xs]
    k = len(xs)
    res = torch.zeros(16 * k, dtype=torch.uint8, device=dev)
    dres = torch.zeros(16 * k, dtype=torch.uint8, device=dev)
    ejobs = A.encode_jobs(xs, ps, outs, res)
    djobs = A.decode_jobs(outs, ys, [N_BLOCK] * k, dres)
    eplan = A.Batch(ejobs, A.aligned_workspace(A.batch_encode_workspace_size(ejobs)))
    dplan = A.Batch(djobs, A.aligned_workspace(A.batch_decode_workspace_size(djobs)))
    # profiler sweep of every array (16 codes) in one launch
    nc = 16
    pts = [torch.zeros(A.POINT_BYTES * nc, dtype=torch.uint8, device=dev) for _ in xs]
    sums = [torch.zeros(A.SUMMARY_BYTES, dtype=torch.uint8, device=dev) for _ in xs]
    pjobs = A.profile_jobs(xs, [N_BLOCK] * k, [list(A.DEFAULT_CANDIDATES)] * k, [TARGET] * k,
                           pts, sums)
    pplan = A.Batch(pjobs, A.aligned_workspace(A.batch_profile_workspace_size(pjobs)))
    for plan in (eplan, dplan, pplan):
        plan.tune(reps=1, stream=stream)
    wsz = max(A.workspace_size(A.TORCH_CODE[x.dtype], x.numel(), p) for x, p in zip(xs, ps))
    ws = torch.empty(wsz, dtype=torch.uint8, device=dev)
    dws = torch.empty(A.decode_workspace_size(), dtype=torch.uint8, device=dev)
    pws = torch.empty(max(A.profile_workspace_size(A.TORCH_CODE[x.dtype], x.numel(), N_BLOCK, nc)
                          for x in xs), dtype=torch.uint8, device=dev)
    r1 = A.new_result(dev)

    def plain_enc():
        for x, p, o in zip(xs, ps, outs_plain):
            A.encode_into(x, p, o, ws, r1, stream)

    def plain_dec():
        for o, y in zip(outs_plain, ys):
            A.decode_into(o, y, dws, r1, stream)

    def plain_prof():
        for x, pt, sm in zip(xs, pts, sums):
            A.profile_into(x, N_BLOCK, list(A.DEFAULT_CANDIDATES), TARGET, pws, pt, sm, stream)

    def timed(fn, reps):
        return _median(_events(fn, reps, stream))

    # each batched operation is one persistent launch, captured once in a CUDA
    # graph and timed as graph replays
    graphs = {}
    for name, plan in (("batched_encode", eplan), ("batched_decode", dplan),
                       ("batched_profile", pplan)):
        plan.run(stream)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.run()  # on the capture stream
        graphs[name] = g
    runs = {"batched_encode": graphs["batched_encode"].replay, "plain_encode": plain_enc,
            "batched_decode": graphs["batched_decode"].replay, "plain_decode": plain_dec,
            "batched_profile": graphs["batched_profile"].replay, "plain_profile": plain_prof}
    reps = 3 if compact else args.steps
    for fn in runs.values():
        for _ in range(2 if compact else max(args.warmup, 3)):
            fn()
    torch.cuda.synchronize()
    with Clocks(0) as clk:
        ms = {name: timed(fn, reps) for name, fn in runs.items()}
    # the batched containers are the plain loop's, byte for byte
    graphs["batched_encode"].replay()
    plain_enc()
    torch.cuda.synchronize()
    same = all(torch.equal(a, b) for a, b in zip(outs, outs_plain))
    st = A.read_results(res, k)
    assert all(r.status == 0 for r in st)
    comp = sum(r.bytes for r in st)
    gbs = {name: total / t / 1e6 for name, t in ms.items()}
    peak, peak_kind = _peaks()
    step_ms = ms["batched_encode"] + ms["batched_decode"]
    if compact:
        return {"workload": f"batched: {k} arrays 4 KB..64 MB ({total / 1e9:.1f} GB), "
                            "int16/int32/float32/float64, fixed rate 2:1/3:1/4:1/6:1, N=256 "
                            "(seed 3); each batched operation one graph-captured persistent launch; "
                            "medians of 3 runs of each",
                "input_sha256": in_sha,
                "gbs_uncompressed": {n: round(v, 2) for n, v in gbs.items()},
                "batched_vs_plain": {op: round(ms["plain_" + op] / ms["batched_" + op], 3)
                                     for op in ("encode", "decode", "profile")},
                "hbm_frac_batched_decode": round((total + comp) / ms["batched_decode"] / 1e6 / peak, 4),
                "ratio": round(total / comp, 4),
                "containers_identical_to_plain": bool(same), "clocks": clk.summary()}
    return {
        "metric": METRIC, "value": round(total / step_ms / 1e6, 3), "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(step_ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "mixed",
        "data": "synthetic",
        "config": {"workload": f"batched: {k} arrays 4 KB..64 MB, int16/int32/float32/float64, "
                               "fixed rate 2:1/3:1/4:1/6:1, N=256 (seed 3)",
                   "bytes": total, "l2": "inputs larger than L2", "input_sha256": in_sha},
        "ratio": round(total / comp, 4),
        "gbs": {n: round(v, 2) for n, v in gbs.items()},
        "ms": {n: round(v, 3) for n, v in ms.items()},
        "batched_vs_plain": {op: round(ms["plain_" + op] / ms["batched_" + op], 3)
                             for op in ("encode", "decode", "profile")},
        "containers_identical_to_plain": bool(same),
        "configs_tuned": {"encode": eplan.config, "decode": dplan.config, "profile": pplan.config},
        "roofline": {"bound": "hbm", "kernel": "batched decode",
                     "achieved": (total + comp) / ms["batched_decode"] / 1e6, "peak": peak,
                     "unit": "GB/s",
                     "frac": (total + comp) / ms["batched_decode"] / 1e6 / peak,
                     "traffic": None, "peak_source": f"{peak_kind} hbm_gbs"},
        "gpu_launches": reps * (3 + k + 2 * k + sum(_profile_launches(x.numel(), A.TORCH_CODE[x.dtype])
                                                    for x in xs)),
        "clocks": clk.summary(),
    }


def run_sensor(args, compact=False):
    """int16 sensor trace at 4:1: single-call latency of the 262,144-sample
    trace, and throughput on a 4 GiB array of 8,192 copies (cold L2)."""
    import torch

    from paper_1303_4994_gb300 import apax as A
    from paper_1303_4994_gb300 import build as B
    from paper_1303_4994_gb300 import synth

    B.build()
    A.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    p = A.params(N_BLOCK, A.FIXED_RATE, (4, 1), 0)
    th = synth.sensor_trace()
    in_sha = synth.sha256(th)  # the replica is 8,192 copies of it
    t = torch.from_numpy(th).to(dev)

    def bufs(x):
        cap = A.encoded_size(A.I16, x.numel(), p)
        return (torch.empty(cap, dtype=torch.uint8, device=dev),
                torch.empty(A.workspace_size(A.I16, x.numel(), p), dtype=torch.uint8, device=dev),
                torch.empty(A.decode_workspace_size(), dtype=torch.uint8, device=dev),
                torch.empty_like(x), A.new_result(dev), A.new_result(dev))

    def timed(fn, reps):
        return _median(_events(fn, max(reps, 20), stream))

    out, ews, dws, y, er, dr = bufs(t)
    for _ in range(max(args.warmup, 3)):
        A.encode_into(t, p, out, ews, er, stream)
        A.decode_into(out, y, dws, dr, stream)
    torch.cuda.synchronize()
    lat_enc = timed(lambda: A.encode_into(t, p, out, ews, er, stream), max(args.steps, 20))
    lat_dec = timed(lambda: A.decode_into(out, y, dws, dr, stream), max(args.steps, 20))
    assert A.read_result(er).status == 0 and A.read_result(dr).status == 0
    xr = t.repeat(8192)
    out, ews, dws, y, er, dr = bufs(xr)
    for _ in range(max(args.warmup, 3)):
        A.encode_into(xr, p, out, ews, er, stream)
        A.decode_into(out, y, dws, dr, stream)
    torch.cuda.synchronize()
    # the same encode with the PREDICT search (its own container)
    pp = A.params(N_BLOCK, A.FIXED_RATE, (4, 1), 0, A.SEARCH_PREDICT)
    outp = torch.empty_like(out)
    erp = A.new_result(dev)
    for _ in range(max(args.warmup, 3)):
        A.encode_into(xr, pp, outp, ews, erp, stream)
    torch.cuda.synchronize()
    with Clocks(0) as clk:
        ms_enc = timed(lambda: A.encode_into(xr, p, out, ews, er, stream), args.steps)
        ms_dec = timed(lambda: A.decode_into(out, y, dws, dr, stream), args.steps)
        ms_encp = timed(lambda: A.encode_into(xr, pp, outp, ews, erp, stream), args.steps)
    xb, cb = xr.numel() * 2, A.read_result(er).bytes
    assert A.read_result(er).status == 0 and A.read_result(dr).status == 0
    assert A.read_result(erp).status == 0 and A.read_result(erp).bytes == cb
    peak, peak_kind = _peaks()
    enc_gbs, dec_gbs = (xb + cb) / ms_enc / 1e6, (xb + cb) / ms_dec / 1e6
    ocodec = oracle_codec(th, A.FIXED_RATE, 4, 1, 0,
                          "the whole 262,144-sample trace (512 KB), fixed rate 4:1, BISECT")
    if compact:
        return {"workload": "int16 sensor trace (262,144 samples, seed 0), fixed rate 4:1, N=256; "
                            "4 GiB = 8,192 copies for throughput",
                "input_sha256": in_sha,
                "oracle_codec": ocodec,
                "single_call_us": {"encode": round(lat_enc * 1e3, 2), "decode": round(lat_dec * 1e3, 2)},
                "replica_gbs_uncompressed": {"encode_bisect": round(xb / ms_enc / 1e6, 2),
                                             "encode_predict": round(xb / ms_encp / 1e6, 2),
                                             "decode": round(xb / ms_dec / 1e6, 2)},
                "hbm_frac": {"encode_bisect": round(enc_gbs / peak, 4),
                             "encode_predict": round((xb + cb) / ms_encp / 1e6 / peak, 4),
                             "decode": round(dec_gbs / peak, 4)},
                "ratio": round(xb / cb, 4), "clocks": clk.summary()}
    return {
        "metric": METRIC, "value": round(xb / (ms_enc + ms_dec) / 1e6, 3), "unit": "GB/s",
        "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": round(ms_enc + ms_dec, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i16", "data": "synthetic",
        "config": {"workload": "int16 sensor trace (262,144 samples, seed 0), fixed rate 4:1, N=256; "
                               "throughput on 8,192 copies (4 GiB)", "l2": "inputs larger than L2",
                   "input_sha256": in_sha},
        "oracle_codec": ocodec,
        "single_call_us": {"encode": round(lat_enc * 1e3, 2), "decode": round(lat_dec * 1e3, 2)},
        "single_call_gbs": {"encode": round(t.numel() * 2 / lat_enc / 1e6, 2),
                            "decode": round(t.numel() * 2 / lat_dec / 1e6, 2)},
        "replica_gbs_uncompressed": {"encode": round(xb / ms_enc / 1e6, 2),
                                     "encode_predict": round(xb / ms_encp / 1e6, 2),
                                     "decode": round(xb / ms_dec / 1e6, 2)},
        "roofline": {"bound": "hbm", "encode_frac": enc_gbs / peak, "decode_frac": dec_gbs / peak,
                     "encode_predict_frac": (xb + cb) / ms_encp / 1e6 / peak,
                     "peak": peak, "unit": "GB/s", "peak_source": f"{peak_kind} hbm_gbs"},
        "ratio": round(xb / cb, 4),
        "clocks": clk.summary(),
    }


def run_field3d(args, compact=False):
    """float64 512^3 k^-4 field with blobs (1 GiB), whole array in one call:
    profile (16 codes, r >= 0.99999) -> fixed quality at the recommended code
    -> decode."""
    import torch

    from paper_1303_4994_gb300 import apax as A
    from paper_1303_4994_gb300 import build as B
    from paper_1303_4994_gb300 import synth

    B.build()
    A.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    xh = synth.field3d(args.field3d_n, seed=2).reshape(-1)
    in_sha = synth.sha256(xh)
    x = torch.from_numpy(xh).to(dev)
    n, xb = x.numel(), x.numel() * 8
    target = 0.99999
    nc = 16
    pws, pts, summ = A.profile_buffers(x, N_BLOCK, nc)
    p = A.params(N_BLOCK, A.FIXED_QUALITY)
    out = torch.empty(A.encoded_size(A.F64, n, p), dtype=torch.uint8, device=dev)
    ews = torch.empty(A.workspace_size(A.F64, n, p), dtype=torch.uint8, device=dev)
    dws = torch.empty(A.decode_workspace_size(), dtype=torch.uint8, device=dev)
    er, dr = A.new_result(dev), A.new_result(dev)
    y = torch.empty_like(x)

    def prof():
        A.profile_into(x, N_BLOCK, list(A.DEFAULT_CANDIDATES), target, pws, pts, summ, stream)

    def enc():
        A.encode_into(x, p, out, ews, er, stream, summary=summ)

    def dec():
        A.decode_into(out, y, dws, dr, stream)

    def timed(fn, reps):
        return _median(_events(fn, max(reps, 20), stream))

    for _ in range(max(args.warmup, 3)):
        prof()
        enc()
        dec()
    torch.cuda.synchronize()
    sm, r = A.read_summary(summ), A.read_result(er)
    assert sm.status == 0 and r.status == 0 and A.read_result(dr).status == 0
    pt = A.read_points(pts, nc)[sm.recommended]
    with Clocks(0) as clk:
        ms = {k: timed(f, args.steps) for k, f in (("profile", prof), ("encode", enc), ("decode", dec))}
    peak, peak_kind = _peaks()
    step = sum(ms.values())
    code = int(pt.code)
    ocodec = oracle_codec(xh[:1 << 21], A.FIXED_QUALITY, 1, 1, code,
                          f"first 2,097,152 elements (16 MiB) of the field, fixed quality at code {code}")
    if compact:
        return {"workload": f"float64 {args.field3d_n}^3 k^-4 field + 4 blobs (seed 2, 1 GiB): "
                            "profile 16 codes -> fixed quality at r>=0.99999 -> decode",
                "input_sha256": in_sha,
                "oracle_codec": ocodec,
                "gbs_step_uncompressed": round(xb / step / 1e6, 2),
                "ms": {k: round(v, 3) for k, v in ms.items()},
                "gbs_uncompressed": {k: round(xb / v / 1e6, 2) for k, v in ms.items()},
                "hbm_frac": {"profile": round(xb / ms["profile"] / 1e6 / peak, 4),
                             "encode": round((xb + r.bytes) / ms["encode"] / 1e6 / peak, 4),
                             "decode": round((xb + r.bytes) / ms["decode"] / 1e6 / peak, 4)},
                "ratio": round(xb / r.bytes, 4), "corr": pt.r,
                "recommended_code": int(sm.recommended_code), "clocks": clk.summary()}
    return {
        "metric": METRIC, "value": round(xb / step / 1e6, 3), "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"float64 {args.field3d_n}^3 k^-4 field + 4 blobs (seed 2): profile 16 "
                               "codes -> fixed quality at r>=0.99999 -> decode, one call each",
                   "bytes": xb, "l2": "inputs larger than L2", "input_sha256": in_sha},
        "oracle_codec": ocodec,
        "ms": {k: round(v, 3) for k, v in ms.items()},
        "gbs_uncompressed": {k: round(xb / v / 1e6, 2) for k, v in ms.items()},
        "hbm_frac": {"encode": (xb + r.bytes) / ms["encode"] / 1e6 / peak,
                     "decode": (xb + r.bytes) / ms["decode"] / 1e6 / peak},
        "ratio": round(xb / r.bytes, 4), "corr": pt.r, "recommended_code": int(sm.recommended_code),
        "peak_source": f"{peak_kind} hbm_gbs", "clocks": clk.summary(),
    }


def run_formats(args):
    """Container version 2 (BFPE groups of 8, the sum stream) against
    version 1: the float32 4096x4096 field at fixed quality, code 2048 (the
    code the profiler recommends for it), and 1,024 copies of the int16
    Nyquist-band trace (512 MiB) lossless (code 0).  Bytes and device time of
    one encode and one decode call per format."""
    import torch

    from paper_1303_4994_gb300 import apax as A
    from paper_1303_4994_gb300 import build as B
    from paper_1303_4994_gb300 import synth

    B.build()
    A.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    names = {0: "v1", A.FORMAT_GROUP8: "group8", A.FORMAT_SUM_STREAM: "sum",
             A.FORMAT_GROUP8 | A.FORMAT_SUM_STREAM: "group8_sum"}

    def timed(fn):
        return _median(_events(fn, max(args.steps, 20), stream))

    def one(x, dc, code):
        xb = x.numel() * x.element_size()
        res = {}
        for fmt, name in names.items():
            p = A.params(N_BLOCK, A.FIXED_QUALITY, (1, 1), code, fmt=fmt)
            out = torch.empty(A.encoded_size(dc, x.numel(), p), dtype=torch.uint8, device=dev)
            ews = torch.empty(A.workspace_size(dc, x.numel(), p), dtype=torch.uint8, device=dev)
            dws = torch.empty(A.decode_workspace_size(), dtype=torch.uint8, device=dev)
            y = torch.empty_like(x)
            er, dr = A.new_result(dev), A.new_result(dev)
            for _ in range(max(args.warmup, 3)):
                A.encode_into(x, p, out, ews, er, stream)
                A.decode_into(out, y, dws, dr, stream)
            torch.cuda.synchronize()
            r = A.read_result(er)
            assert r.status == 0 and A.read_result(dr).status == 0
            assert torch.equal(y.view(torch.uint8), y.view(torch.uint8))
            ms_e = timed(lambda: A.encode_into(x, p, out, ews, er, stream))
            ms_d = timed(lambda: A.decode_into(out, y, dws, dr, stream))
            res[name] = {"ratio": round(xb / r.bytes, 4),
                         "encode_gbs_uncompressed": round(xb / ms_e / 1e6, 2),
                         "decode_gbs_uncompressed": round(xb / ms_d / 1e6, 2)}
        return res

    fh, nh = synth.grf2d(4096, 4096, seed=1).reshape(-1), synth.nyquist_trace()
    field = torch.from_numpy(fh).to(dev)
    out = {"workload": "float32 4096x4096 field (seed 1), fixed quality code 2048, N=256; "
                       "int16 Nyquist-band trace (sensor trace x (-1)^i, seed 0), 1,024 copies, "
                       "code 0 (lossless), N=256",
           "input_sha256": {"field": synth.sha256(fh), "nyquist_trace": synth.sha256(nh)},
           "field_f32_code2048": one(field, A.F32, 2048)}
    del field
    tr = torch.from_numpy(nh).to(dev).repeat(1024)
    out["nyquist_i16_lossless"] = one(tr, A.I16, 0)
    return out


def run_serving(args, compact=False):
    """Poisson arrivals at 2,000 requests/s for --serve-seconds (the default
    run: 10 s): open loop (latency) and closed loop (throughput) through the
    request server, against the plain per-request path."""
    import torch

    from paper_1303_4994_gb300 import apax as A
    from paper_1303_4994_gb300 import build as B
    from paper_1303_4994_gb300 import synth

    B.build()
    A.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    seconds = 10.0 if compact else args.serve_seconds
    trace = synth.serving_trace(seconds)
    # device-resident payload pools (float32 field, int16 trace), 4 GB each
    fh, th = synth.grf2d(4096, 4096, seed=1).reshape(-1), synth.sensor_trace(1 << 25, seed=0)
    # the requests are slices of the pools (16 and 64 copies of these)
    in_sha = synth.sha256(fh, th, repr(trace))
    field = torch.from_numpy(fh).to(dev)
    pool = {"float32": field.repeat(16), "int16": torch.from_numpy(th).to(dev).repeat(64)}
    del th
    # the profiler's choice for the field (fixed quality at r >= 0.9999)
    pts, summ = A.profile(field, N_BLOCK, A.DEFAULT_CANDIDATES, TARGET)
    code = int(summ.recommended_code)
    params = {"float32": A.params(N_BLOCK, A.FIXED_QUALITY, (1, 1), code),
              "int16": A.params(N_BLOCK, A.FIXED_RATE, (4, 1), 0)}
    # decode requests use pre-encoded containers at 64 log-spaced sizes
    sizes = np.unique(np.exp(np.linspace(np.log(64 << 10), np.log(256 << 20), 64)).astype(np.int64))
    pre = {}
    for dt in ("float32", "int16"):
        es = 4 if dt == "float32" else 2
        for nb in sizes:
            n = int(nb) // es
            pre[(dt, int(nb))] = (A.encode(pool[dt][:n], N_BLOCK, params[dt].mode,
                                           (params[dt].rate_num, params[dt].rate_den),
                                           params[dt].atten_code), n)
    reqs = []
    for t, op, dt, nb, off in trace:
        es = 4 if dt == "float32" else 2
        if op == "encode":
            n = nb // es
            o = off % (pool[dt].numel() - n)
            reqs.append((t, op, dt, pool[dt][o:o + n], n, nb))
        else:
            j = int(np.clip(np.searchsorted(sizes, nb), 0, len(sizes) - 1))
            c, n = pre[(dt, int(sizes[j]))]
            reqs.append((t, op, dt, c, n, n * es))
    arena = A.aligned_workspace(64 << 30)
    torch.cuda.synchronize()

    def serve(open_loop, depth):
        srv = A.Server(arena, slots=4, max_batch=256)
        lat, done_bytes, first, last = [], 0, None, 0.0
        i, outstanding = 0, 0
        t0 = time.perf_counter()
        while i < len(reqs) or outstanding:
            now = time.perf_counter() - t0
            while i < len(reqs) and (reqs[i][0] <= now if open_loop else outstanding < depth):
                t, op, dt, buf, n, nb = reqs[i]
                if op == "encode":
                    srv.submit_encode(i, buf, params[dt])
                else:
                    srv.submit_decode(i, buf, getattr(torch, dt), n, N_BLOCK)
                i += 1
                outstanding += 1
            for c in srv.poll():
                assert c.status == 0, c.status
                outstanding -= 1
                lat.append(c.t_done - c.t_submit)
                done_bytes += reqs[c.id][5]
                first = c.t_submit if first is None else min(first, c.t_submit)
                last = max(last, c.t_done)
                srv.release(c.out)
        st = srv.stats()
        srv.close()
        return lat, done_bytes / (last - first) / 1e9, st

    lat, gbs_open, st_open = serve(True, 0)
    lat_c, gbs_closed, st_closed = serve(False, 1024)
    # the plain per-request path: one call per request, one stream
    ws = torch.empty(max(A.workspace_size(A.TORCH_CODE[getattr(torch, dt)], r[4], params[dt])
                         for r in reqs for dt in [r[2]]), dtype=torch.uint8, device=dev)
    dws = torch.empty(A.decode_workspace_size(), dtype=torch.uint8, device=dev)
    r1 = A.new_result(dev)
    out_e = torch.empty(max(A.encoded_size(A.TORCH_CODE[getattr(torch, r[2])], r[4], params[r[2]])
                            for r in reqs), dtype=torch.uint8, device=dev)
    out_d = torch.empty(max(r[5] for r in reqs), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t, op, dt, buf, n, nb in reqs:
        if op == "encode":
            A.encode_into(buf, params[dt], out_e, ws, r1, stream)
        else:
            A.decode_into(buf, out_d[:nb].view(getattr(torch, dt)), dws, r1, stream)
    torch.cuda.synchronize()
    plain_gbs = sum(r[5] for r in reqs) / (time.perf_counter() - t0) / 1e9
    total = sum(r[5] for r in reqs)
    if compact:
        return {"workload": f"serving: Poisson 2000 req/s for {seconds:g} s ({len(reqs)} requests, "
                            f"{total / 1e9:.1f} GB), 50/50 encode/decode, 64 KB..256 MB float32 "
                            f"(fixed quality, code {code}) / int16 (4:1) (seed 4)",
                "input_sha256": in_sha,
                "open_loop": {"gbs": round(gbs_open, 3), "offered_gbs": round(total / seconds / 1e9, 3),
                              "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                              "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3)},
                "closed_loop_gbs": round(gbs_closed, 3), "plain_per_request_gbs": round(plain_gbs, 3),
                "served_vs_plain": round(gbs_closed / plain_gbs, 3)}
    return {
        "metric": METRIC, "value": round(gbs_closed, 3), "unit": "GB/s", "n_gpus": 1,
        "steps": 1, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "mixed", "data": "synthetic",
        "config": {"workload": f"serving: Poisson 2000 req/s for {seconds:g} s, 50/50 "
                               "encode/decode, 64 KB..256 MB float32 (fixed quality, code "
                               f"{code}) / int16 (4:1), 64 GB admission cap (seed 4)",
                   "requests": len(reqs), "bytes": total, "slots": 4, "max_batch": 256,
                   "input_sha256": in_sha},
        "open_loop": {"gbs": round(gbs_open, 3), "offered_gbs": round(total / seconds / 1e9, 3),
                      "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                      "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3),
                      "steps": st_open["steps"], "arena_peak_gb": round(st_open["arena_peak"] / 1e9, 3)},
        "closed_loop": {"gbs": round(gbs_closed, 3),
                        "p50_ms": round(float(np.percentile(lat_c, 50)) * 1e3, 3),
                        "p99_ms": round(float(np.percentile(lat_c, 99)) * 1e3, 3),
                        "steps": st_closed["steps"]},
        "plain_per_request_gbs": round(plain_gbs, 3),
        "served_vs_plain": round(gbs_closed / plain_gbs, 3),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the sensor and float64 field workloads of the default run")
    ap.add_argument("--workload", default="field",
                    choices=["field", "batched", "serving", "sensor", "field3d"])
    ap.add_argument("--field3d-n", type=int, default=512)
    ap.add_argument("--arrays", type=int, default=8192)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    args = ap.parse_args()
    if args.workload != "field" and args.impl == "ours":
        import torch
        torch.cuda.set_device(0)
        line = {"batched": run_batched, "serving": run_serving, "sensor": run_sensor,
                "field3d": run_field3d}[args.workload](args)
        print(json.dumps(line))
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
