"""Benchmark of the GB300 channelizer (arXiv 1411.0436 hot path).

One step = one vspec_execute over one dump of the workload: dual-pol PFB,
131072 channels, 8 taps, Hann-windowed sinc, 4096 spectra of seeded synthetic
int8 input resident in HBM (2.15 GB; the largest single-GPU workload, the
precision-stress one on which the tensor-core and FP32 forms are compared). The metric is the real-time dual-polarisation
bandwidth, S * N / t in GHz (complex sampling: one complex sample per
polarisation per second of time is one hertz of bandwidth).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 the script runs under torchrun, one rank per GPU; every rank
channelizes its own beam (independent input, no data exchange), so the work
scales weakly. Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
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

from paper_1411_0436_gb300 import workloads  # noqa: E402

METRIC = "Dual-pol real-time bandwidth (GHz) & % HBM roofline, TC-FP16 vs FP32 FFT"
CONFIG_NAME = "c4"
WORKLOADS = {
    "c1": "single-pol PFB, 1024 channels, 8 taps, Hann-windowed sinc, 64 spectra, tone at bin 123.4",
    "c2": ("dual-pol PFB, 32768 channels, 8 taps, Hann-windowed sinc, 1000 spectra per dump, "
           "int8 Gaussian sigma=20 with X/Y correlation 0.3 and two tones"),
    "c3": "dual-pol direct FFT, 524288 channels, 256 spectra per dump, int8 Gaussian sigma=20",
    "c4": ("dual-pol PFB, 131072 channels, 8 taps, Hann-windowed sinc, 4096 spectra per dump, "
           "sigma=4 with a tone 40 dB above the per-channel noise floor"),
}
WORKLOAD = WORKLOADS[CONFIG_NAME]
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0
SM_MAX_MHZ = 2070  # maximum SM clock of the GB300


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def source_hash() -> str:
    """Hash of the device-code sources (the kernels an ncu capture measured):
    every line with its // comment and surrounding blanks removed, so that a
    comment-only edit keeps the captures valid."""
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_1411_0436_gb300", "csrc", "*.cuh")))
    for f in files:
        with open(f, encoding="utf-8") as fh:
            code = [line.split("//", 1)[0].strip() for line in fh]
        h.update(os.path.basename(f).encode())
        h.update("\n".join(c for c in code if c).encode())
    return h.hexdigest()[:16]


def _traffic(config: str, kernel: str, spectra_per_launch: float):
    """DRAM bytes per launch from the committed ncu summary of this workload,
    if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    ent = d.get(config, {}).get(kernel)
    if not ent or ent.get("source_hash") != source_hash():
        return None
    return float(ent["dram_bytes_per_spectrum"]) * spectra_per_launch


def beam_seed(rank: int, config: str = CONFIG_NAME) -> int:
    """Seed of rank `rank`'s beam: every rank channelizes independent input."""
    return workloads.config_seed(config) + 7919 * rank


def reduce_max(value: float, dist=None, device=None) -> float:
    """Maximum of `value` over all ranks (the job time is the slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_ghz(world: int, steps: int, nspectra: int, nchan: int, max_ms: float) -> float:
    """Real-time bandwidth of the whole job: every rank's spectra over the max time."""
    return world * steps * nspectra * nchan / (max_ms * 1e-3) / 1e9


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"vspec_clocks_gpu{self.gpu}_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        lines = []
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_rate(bank, x, budget_s: float, nthreads: int):
    """Time the oracle on a bounded sample of the workload (about budget_s of
    CPU work): repeated runs over the first spectra of the same input.
    Returns GHz, spectra per run, runs, seconds."""
    import oracle
    oracle.build()
    n = bank.nchan
    t0 = time.perf_counter()
    oracle.channelize(x, n, bank.ntaps, bank.npol, 4, bank.mode, bank.window, nthreads=nthreads)
    per = max((time.perf_counter() - t0) / 4, 1e-9)
    s = int(max(1, min(bank.nspectra, budget_s / per)))
    runs, dt = 0, 0.0
    while runs == 0 or (dt < budget_s and runs < 100):
        t0 = time.perf_counter()
        oracle.channelize(x, n, bank.ntaps, bank.npol, s, bank.mode, bank.window, nthreads=nthreads)
        dt += time.perf_counter() - t0
        runs += 1
    return runs * s * n / dt / 1e9, s, runs, dt


def _window_sinc(n: int, taps: int, mode: int, window: int) -> np.ndarray:
    """FIR weights h[t, n] of the channelizer (§4's polyphase filter bank):
    a windowed sinc of length taps*n with zeros every n samples, or the bare
    window in direct mode. Written out here for the cuFFT comparison only."""
    L = taps * n if mode == workloads.PFB else n
    i = np.arange(L, dtype=np.float64)
    if window == workloads.WIN_HANN:
        w = 0.5 - 0.5 * np.cos(2 * np.pi * i / (L - 1))
    elif window == workloads.WIN_HAMMING:
        w = 0.54 - 0.46 * np.cos(2 * np.pi * i / (L - 1))
    else:
        w = np.ones(L)
    if mode == workloads.PFB:
        w = w * np.sinc((i - (L - 1) / 2) / n)
    return w.reshape(-1, n)


def run_cufft_comparison(bank, d_in, dev, stream, flush, steps: int):
    """The GPU comparison: the same dump through PyTorch ops and cuFFT
    (torch.fft.fft): int8 -> complex64, the FIR as P scaled adds, one batched
    FFT per chunk of spectra, detection and the sum over spectra, all FP32.
    Returns its rate and its accumulated spectrum."""
    import torch
    n, S, npol = bank.nchan, bank.nspectra, bank.npol
    P = bank.ntaps if bank.mode == workloads.PFB else 1
    h = torch.tensor(_window_sinc(n, P, bank.mode, bank.window), dtype=torch.float32, device=dev)
    frames = d_in.view(torch.int8)[: (S + P - 1) * n * npol * 2].view(S + P - 1, n, npol, 2)
    chunk = max(1, min(S, (1 << 28) // (n * npol)))

    def step():
        acc = torch.zeros(4 if npol == 2 else 1, n, dtype=torch.float32, device=dev)
        for s0 in range(0, S, chunk):
            c = min(chunk, S - s0)
            x = frames[s0: s0 + c + P - 1].float().permute(0, 2, 1, 3).contiguous()
            x = torch.view_as_complex(x)                       # [c+P-1, npol, n]
            y = h[0] * x[0:c]
            for t in range(1, P):
                y = y + h[t] * x[t: t + c]
            Y = torch.fft.fft(y, dim=-1)
            X0 = Y[:, 0]
            acc[0] += (X0.real ** 2 + X0.imag ** 2).sum(0)
            if npol == 2:
                X1 = Y[:, 1]
                acc[1] += (X1.real ** 2 + X1.imag ** 2).sum(0)
                xy = X0 * X1.conj()
                acc[2] += xy.real.sum(0)
                acc[3] += xy.imag.sum(0)
        return acc

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush.fill_(7)
        a.record(stream)
        out = step()
        b.record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    out = out.t().contiguous().cpu().numpy().astype(np.float64)
    return {"value": S * n / (ms * 1e-3) / 1e9, "unit": "GHz", "ms_per_step": ms, "steps": steps,
            "what": "PyTorch int8->complex64, FIR as P scaled adds, torch.fft.fft (cuFFT), detection, sum; FP32"}, out


def run_reference(args, rank: int):
    """The reference arm: the FP64 oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    bank = workloads.CONFIGS[CONFIG_NAME][0]
    x = workloads.generate(bank, workloads.config_seed(CONFIG_NAME))
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    n = bank.nchan
    t0 = time.perf_counter()
    oracle.channelize(x, n, bank.ntaps, bank.npol, 2, bank.mode, bank.window, nthreads=threads)
    per_spec = (time.perf_counter() - t0) / 2
    step_budget = max(0.05, min(1.0, 150.0 / max(1, args.steps + args.warmup)))
    s = int(max(1, min(bank.nspectra, step_budget / max(per_spec, 1e-9))))
    for _ in range(args.warmup):
        oracle.channelize(x, n, bank.ntaps, bank.npol, s, bank.mode, bank.window, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.channelize(x, n, bank.ntaps, bank.npol, s, bank.mode, bank.window, nthreads=threads)
    dt = time.perf_counter() - t0
    value = args.steps * s * n / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GHz",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nchan": n, "ntaps": bank.ntaps, "npol": bank.npol,
                   "nspectra_per_step": s},
        "cpu_baseline": {"value": value, "unit": "GHz", "cores": threads, "kind": "oracle",
                         "sample": f"first {s} spectra of the {CONFIG_NAME} input per step"},
        "e2e": {"value": value, "unit": "GHz", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank: int, world: int, local_rank: int):
    import torch
    from paper_1411_0436_gb300.vspec import Plan

    dist = None
    if world > 1:
        import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    config = args.config
    bank = workloads.CONFIGS[config][0]
    if args.spectra:  # a shorter dump of the same workload (profiling captures)
        import dataclasses
        bank = dataclasses.replace(bank, nspectra=min(args.spectra, bank.nspectra))
    # each rank is an independent beam: its own seeded input
    x = workloads.generate(bank, beam_seed(rank, config))
    nsub = max(1, args.nsub)
    if nsub > 1:  # sub-band input [time][sub][pol][re, im]: independent seeded bands
        x = np.ascontiguousarray(np.stack([x] + [workloads.generate(bank, beam_seed(rank, config) + 31 * b)
                                                 for b in range(1, nsub)], axis=1))
        args.no_variants = args.no_cpu_baseline = args.no_e2e = True
    in_bytes = x.nbytes
    n, S = bank.nchan, bank.nspectra
    plan = Plan(n, bank.ntaps, bank.npol, bank.mode, bank.window, args.plan_flags, nsub=nsub)
    plan_desc = plan.describe()  # decomposition and kernel forms, for the JSON line
    d_in = torch.from_numpy(x.view(np.uint8).reshape(-1)).to(dev)
    acc = torch.zeros(plan.out_floats, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step_device():
        plan.execute(d_in, S, acc, stream)

    # warm-up
    for _ in range(args.warmup):
        flush.fill_(1)
        step_device()
    torch.cuda.synchronize()

    gpu_index = local_rank
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local_rank])
        except (ValueError, IndexError):
            pass
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.2)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)            # L2 flush: 256 MiB written between steps
        starts[i].record(stream)
        step_device()
        ends[i].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
    total_ms = sum(step_ms)
    median_ms = statistics.median(step_ms)

    # second timed pass of the same steps with the library's per-launch event
    # records on (vspec_plan_set_profiling): per-kernel durations for the
    # roofline, kept out of the headline because the extra events add a
    # little time between launches
    prof_steps = max(3, min(args.steps, 200))
    plan.set_profiling(True)
    for i in range(prof_steps):
        flush.fill_(i & 0xFF)
        step_device()
    torch.cuda.synchronize()
    stats = plan.kernel_stats()
    plan.set_profiling(False)
    clk = clocks.stop()

    total_ms = reduce_max(total_ms, dist, dev)
    value = whole_job_ghz(world, args.steps, S, n * nsub, total_ms)

    # dominant kernel: live CUDA-event times
    peak, peak_kind = _peaks()
    per_spec_bytes = (n * bank.npol * 2 + 2.0 * n * 16 / S) * nsub  # int8 input once + accumulator RMW per dump
    dom = max(stats, key=lambda r: r[3])
    name, launches, spectra, kms = dom
    # (a sub-band call's launches each count the spectra of one band)
    achieved = (spectra * per_spec_bytes / nsub) / (kms * 1e-3) / 1e9
    spl = spectra / max(1, launches)
    traffic = _traffic(config, name, spl) if nsub == 1 else None
    path_bytes = args.steps * S * per_spec_bytes
    kernels = {r[0]: {"launches": r[1], "total_ms": round(r[3], 4),
                      "share": round(r[3] / max(1e-9, sum(q[3] for q in stats)), 4)} for r in stats}
    gpu_launches = int(round(sum(r[1] for r in stats) / prof_steps * args.steps))
    # FP32 arithmetic of the method (conventional count per complex sample:
    # 4P FIR + 5 log2 N FFT + detection/accumulation) against the CUDA-core peak
    taps_eff = bank.ntaps if bank.mode == workloads.PFB else 1
    flop_per_sample = 4 * taps_eff + 5 * int(np.log2(n)) + (8 if bank.npol == 2 else 4)
    flop_per_spec = flop_per_sample * n * bank.npol * nsub
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = nsm * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    alu_achieved = spectra * flop_per_spec / nsub / (kms * 1e-3) / 1e12

    # end to end through vspec_execute_host: pinned host input, chunked copies
    # overlapped with the compute on plan-owned streams, result read back to
    # pinned host memory, all inside the timed region
    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(x.view(np.uint8).reshape(-1)).pin_memory()
        h_out = torch.empty(plan.out_floats, dtype=torch.float32).pin_memory()
        e2e_steps = max(3, min(args.steps, 50))
        for _ in range(2):
            plan.execute_host(h_in, S, h_out, stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            plan.execute_host(h_in, S, h_out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = reduce_max(e0.elapsed_time(e1), dist, dev)
        e2e = {"value": whole_job_ghz(world, e2e_steps, S, n, ems), "unit": "GHz",
               "h2d_bytes_per_step": int(in_bytes), "d2h_bytes_per_step": int(plan.out_floats * 4),
               "steps": e2e_steps, "api": "vspec_execute_host (staged copies overlapped with compute)"}
        # the same loop with the pinned input read by the kernels directly
        from paper_1411_0436_gb300.vspec import HOST_MAPPED, HOST_STAGED
        plan.set_host_mode(HOST_MAPPED)
        plan.execute_host(h_in, S, h_out, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(e2e_steps):
            plan.execute_host(h_in, S, h_out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        sms = reduce_max(e0.elapsed_time(e1), dist, dev)
        plan.set_host_mode(HOST_STAGED)
        e2e["mapped_input_value"] = whole_job_ghz(world, e2e_steps, S, n, sms)

    # TC-FP16 vs FP32: the same dump through the tensor-core plan and through
    # the FP32 two-kernel plan (rank 0 only), with their errors against the
    # oracle when the CPU baseline runs
    variants = None
    if rank == 0 and world == 1 and not args.no_variants and bank.npol == 2 and config in ("c2", "c4"):
        from paper_1411_0436_gb300.vspec import PLAN_TENSOR, PLAN_TWO_KERNEL
        variants = {}
        vsteps = max(3, min(args.steps, 50))
        from paper_1411_0436_gb300.vspec import NEVER
        from paper_1411_0436_gb300.vspec import PLAN_KAHAN
        from paper_1411_0436_gb300.vspec import PLAN_RING, PLAN_TENSOR_INT8
        cands = [("tensor_core", PLAN_TENSOR, None), ("tensor_core_int8", PLAN_TENSOR_INT8, None),
                 ("fp32_two_kernel", PLAN_TWO_KERNEL, None), ("fp32_kahan", PLAN_KAHAN, None),
                 ("fp32_ring", PLAN_RING, None)]
        if n <= 32768:  # the one-pass cluster kernel on every call length
            cands.append(("fp32_fused_cluster", 0, {"two_kernel_from": NEVER, "assist_permille": 0}))
        for key, flags, tuning in cands:
            vp = Plan(n, bank.ntaps, bank.npol, bank.mode, bank.window, flags)
            if tuning:
                vp.tune(**tuning)
            vacc = torch.zeros(vp.out_floats, dtype=torch.float32, device=dev)
            for _ in range(3):
                vp.execute(d_in, S, vacc, stream)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(vsteps)]
            for a, b in ev:
                flush.fill_(3)
                a.record(stream)
                vp.execute(d_in, S, vacc, stream)
                b.record(stream)
            torch.cuda.synchronize()
            vms = sum(a.elapsed_time(b) for a, b in ev) / vsteps
            vp.dump(vacc, None, stream)  # clears the accumulator (and a compensated plan's compensation)
            vp.execute(d_in, S, vacc, stream)
            torch.cuda.synchronize()
            variants[key] = {"value": S * n / (vms * 1e-3) / 1e9, "unit": "GHz", "ms_per_step": vms,
                             "out": vacc.cpu().numpy().astype(np.float64).reshape(n, 4),
                             "flags": flags}
            vp.close()
        acc.zero_()
        plan.execute(d_in, S, acc, stream)
        torch.cuda.synchronize()
        variants["fp32_default"] = {"value": value, "unit": "GHz", "ms_per_step": total_ms / args.steps,
                                    "out": acc.cpu().numpy().astype(np.float64).reshape(n, 4)}

    # the cuFFT comparison (rank 0 at N=1), with its spectrum's distance
    # from ours normalised like the parity metric
    cufft = None
    if rank == 0 and world == 1 and not args.no_variants:
        cufft, cout = run_cufft_comparison(bank, d_in, dev, stream, flush, max(3, min(args.steps, 20)))
        cufft["speedup_of_ours"] = value / cufft["value"]

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        ghz, s_used, runs, dt = _oracle_rate(bank, x, 12.0, threads)
        cpu = {"value": ghz, "unit": "GHz", "cores": threads, "kind": "oracle",
               "sample": f"first {s_used} of {S} spectra of the same input, {runs} runs, {dt:.1f} s"}
        ghz1, s1, runs1, dt1 = _oracle_rate(bank, x, 5.0, 1)
        cpu["one_core"] = {"value": ghz1, "cores": 1,
                           "sample": f"first {s1} of {S} spectra, {runs1} runs, {dt1:.1f} s"}
        acc.zero_()
        plan.execute(d_in, S, acc, stream)
        torch.cuda.synchronize()
        ours_out = acc.cpu().numpy().astype(np.float64).reshape(n, -1)
        # errors against the FP64 oracle over the whole dump, normalised
        # as in the parity tests (auto terms by their RMS, cross terms by
        # the geometric mean of the two auto RMS)
        import oracle
        ref = oracle.channelize(x, n, bank.ntaps, bank.npol, S, bank.mode, bank.window, nthreads=threads)
        ref = ref.reshape(n, -1)
        rms = np.sqrt(np.mean(ref ** 2, axis=0))
        scale = (np.array([rms[0], rms[1], np.sqrt(rms[0] * rms[1]), np.sqrt(rms[0] * rms[1])])
                 if bank.npol == 2 else rms)
        for v in (variants or {}).values():
            v["max_err_norm_rms"] = float(np.max(np.abs(v["out"] - ref) / scale))
        if cufft:
            cufft["max_err_norm_rms"] = float(np.max(np.abs(cout.reshape(n, -1) - ref) / scale))
        # the FP32 criterion: |G - O| <= 1e-5 * scale + r(N) * own value, with
        # r(N) = (log2(N) / 4 + 2) * 2^-24: FP32 rounding of the transform
        # (a quarter unit per radix-2 level), detection, summation and the
        # stored result, which bind channels far above the RMS (tones)
        own = np.abs(ref) if bank.npol == 1 else np.concatenate(
            [np.abs(ref[:, :2]), np.repeat(np.sqrt(np.abs(ref[:, :1] * ref[:, 1:2])), 2, axis=1)], axis=1)
        rtol = (np.log2(n) / 4 + 2) * 2.0 ** -24
        allowed = 1e-5 * scale + rtol * own
        parity = {"max_err_norm_rms": float(np.max(np.abs(ours_out - ref) / scale)),
                  "tolerance_use": float(np.max(np.abs(ours_out - ref) / allowed)),
                  "against": "FP64 CPU oracle, whole dump",
                  "criterion": "|G-O| <= 1e-5*RMS + (log2(N)/4 + 2)*2^-24*|O| per channel (tolerance_use <= 1)"}
        allowed_tc = 1e-3 * scale + rtol * own  # the tensor-core form's bound: 1e-3 of the RMS
        for v in (variants or {}).values():
            tc_form = bool(v.get("flags", 0) & 10)  # VSPEC_PLAN_TENSOR or VSPEC_PLAN_TENSOR_INT8
            v["tolerance_use"] = float(np.max(np.abs(v["out"] - ref) / (allowed_tc if tc_form else allowed)))
            v["tolerance"] = "1e-3*RMS + r(N)*|O|" if tc_form else "1e-5*RMS + r(N)*|O|"
    if variants:
        for v in variants.values():
            v.pop("out", None)
        variants["tc_speedup_over_fp32"] = (variants["tensor_core"]["value"] /
                                            variants["fp32_default"]["value"])
        variants["tc_int8_speedup_over_fp32"] = (variants["tensor_core_int8"]["value"] /
                                                 variants["fp32_default"]["value"])
        variants["ring_speedup_over_fp32"] = (variants["fp32_ring"]["value"] /
                                              variants["fp32_default"]["value"])

    plan.close()
    # the batched multi-beam workload (rank 0 at N=1), as an extra key
    batched = None
    if rank == 0 and world == 1 and not args.no_variants:
        batched = measure_batch(max(3, min(args.steps, 50)), 3)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GHz", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[config], "name": config, "nchan": n, "ntaps": bank.ntaps,
                       "npol": bank.npol, "nspectra": S, "nsub": nsub, "input_bytes": int(in_bytes),
                       "l2": "flushed between steps (256 MiB write outside the timed interval)",
                       "parallelism": f"replicas x{world} (independent beams)"},
            "ms_per_step_median": median_ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": name,
                         "peak_source": peak_kind,
                         "algorithmic_bytes_per_spectrum": per_spec_bytes,
                         "timed": f"per-launch events over a second pass of {prof_steps} steps"},
            "alu_roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s",
                             "frac": alu_achieved / alu_peak, "kernel": name,
                             "flop_per_complex_sample": flop_per_sample,
                             "peak_source": f"{nsm} SMs x 128 FP32 lanes x 2 flop x {SM_MAX_MHZ} MHz"},
            "path_roofline": {"bound": "hbm", "achieved": path_bytes / (total_ms * 1e-3) / 1e9,
                              "peak": peak, "unit": "GB/s",
                              "frac": path_bytes / (total_ms * 1e-3) / 1e9 / peak,
                              "what": "whole path: algorithmic bytes of every step over the mean step time"},
            "path_alu_roofline": {"bound": "alu",
                                  "achieved": args.steps * S * flop_per_spec / (total_ms * 1e-3) / 1e12,
                                  "peak": alu_peak, "unit": "TFLOP/s",
                                  "frac": args.steps * S * flop_per_spec / (total_ms * 1e-3) / 1e12 / alu_peak,
                                  "what": "whole path: the method's FP32 flops over the mean step time"},
            "kernels": kernels,
            "plan": plan_desc,
            "gpu_launches": gpu_launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "tc_vs_fp32": variants,
            "cufft_comparison": cufft,
            "batched_c5": batched,
            "parity": parity,
            "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")} | {"samples": clk["samples"]},
            "complex_gsps": 2 * value,
        }
        print(json.dumps(line), flush=True)


def measure_batch(steps: int, warmup: int) -> dict:
    """The batched multi-beam workload (eight banks, 1024..524288 channels,
    PFB and direct alternating, uneven integrations) as one CUDA-graph launch
    per step after the autotuner has picked each bank's plan form, four-step
    split and launch shape."""
    import torch
    from paper_1411_0436_gb300.vspec import Batch
    dev = torch.device("cuda", 0)
    banks = workloads.CONFIGS["c5"]
    xs = [workloads.generate(b, workloads.config_seed("c5", i)) for i, b in enumerate(banks)]
    batch = Batch([(b.nchan, b.ntaps, b.npol, b.mode, b.window) for b in banks])
    d_in = [torch.from_numpy(x.view(np.uint8).reshape(-1)).to(dev) for x in xs]
    accs = [torch.zeros(batch.out_floats(i), dtype=torch.float32, device=dev) for i in range(len(banks))]
    ns = [b.nspectra for b in banks]
    stream = torch.cuda.current_stream(dev)
    flags = batch.autotune(d_in, ns, accs, stream, reps=3)
    batch_shapes = [dict(batch.bank_tuning(i)[1], col_len=batch.bank_shape(i)[0], tile_cols=batch.bank_shape(i)[1])
                    for i in range(len(flags))]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def timed() -> float:
        for _ in range(warmup):
            flush.fill_(1)
            batch.execute(d_in, ns, accs, stream)
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(i & 0xFF)
            starts[i].record(stream)
            batch.execute(d_in, ns, accs, stream)
            ends[i].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in zip(starts, ends))

    # the autotuner's choice of form (per-bank kernels in one graph, or one
    # persistent launch over all banks) is the value; both are reported
    chosen = "persistent" if batch.persistent else "graph"
    samples = sum(b.nspectra * b.nchan for b in banks)
    forms = {}
    for form in (chosen, "graph" if chosen == "persistent" else "persistent"):
        try:
            batch.set_persistent(form == "persistent")
            ms = timed()
            batch.check()
            forms[form] = {"value": steps * samples / (ms * 1e-3) / 1e9, "unit": "GHz", "ms_per_step": ms / steps}
        except Exception as e:  # a bank the persistent kernel has no body for
            forms[form] = {"unavailable": str(e)}
    total_ms = forms[chosen]["ms_per_step"] * steps
    value = forms[chosen]["value"]
    persistent = dict(forms.get("persistent", {}),
                      what="one cooperative launch: kernel-A tiles, rows and folds of all banks as tickets")
    in_bytes = sum(x.nbytes for x in xs)
    peak, peak_kind = _peaks()
    achieved = steps * sum(b.nbytes + 2 * b.nchan * 16 for b in banks) / (total_ms * 1e-3) / 1e9
    batch.close()
    return {"value": value, "unit": "GHz", "steps": steps, "ms_per_step": total_ms / steps,
            "workload": "8 dual-pol banks 1024..524288 channels, PFB-8/direct alternating, "
                        "2048..64 spectra, one CUDA-graph launch per step (the autotuner's form)",
            "input_bytes": int(in_bytes), "bank_flags": flags, "bank_shapes": batch_shapes,
            "persistent": persistent, "form": chosen, "graph": forms.get("graph"),
            "path_roofline": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                              "peak_source": peak_kind}}


def run_batch(args):
    """--config c5: the batched workload as the bench line."""
    r = measure_batch(args.steps, args.warmup)
    print(json.dumps({
        "metric": METRIC + " (batched multi-beam workload)", "value": r["value"], "unit": "GHz",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": r["workload"], "input_bytes": r["input_bytes"], "bank_flags": r["bank_flags"],
                   "bank_shapes": r["bank_shapes"],
                   "l2": "flushed between steps (256 MiB write outside the timed interval)"},
        "path_roofline": r["path_roofline"], "form": r["form"], "persistent": r["persistent"], "graph": r["graph"],
    }), flush=True)


def run_sweep(args):
    """Real-time bandwidth against FFT length and accumulation length (the
    shape of the paper's Fig. 3, §5): 8-tap PFB and direct FFT, N = 2^10 ..
    2^20, a = 1, 10, 100, 1000 spectra per call, device-resident input, and
    the host-copy loop of §4 through vspec_execute_host where the input fits a
    1 GiB pinned buffer. Inputs are random int8 drawn on the device (timing
    only). One JSON line per case."""
    import torch
    from paper_1411_0436_gb300.vspec import Plan, VspecError
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    pinned = torch.empty(1 << 30, dtype=torch.uint8).pin_memory()
    for mode, taps in ((workloads.PFB, 8), (workloads.DIRECT, 1)):
        for e in range(10, 21):
            n = 1 << e
            try:
                plan = Plan(n, taps, 2, mode, workloads.WIN_HANN if mode == workloads.PFB else workloads.WIN_RECT)
            except VspecError as err:
                print(json.dumps({"sweep": True, "mode": "pfb" if mode == workloads.PFB else "direct",
                                  "nchan": n, "unsupported": str(err)}), flush=True)
                continue
            for a in (1, 10, 100, 1000):
                nbytes = (a + taps - 1) * n * 4
                if nbytes > (6 << 30):
                    continue
                d_in = torch.randint(-127, 128, (nbytes,), dtype=torch.int8, device=dev)
                acc = torch.zeros(plan.out_floats, dtype=torch.float32, device=dev)
                reps = max(3, min(20, int(2e8 // (a * n))))
                for _ in range(2):
                    plan.execute(d_in, a, acc, stream)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
                for t0, t1 in ev:
                    flush.fill_(5)
                    t0.record(stream)
                    plan.execute(d_in, a, acc, stream)
                    t1.record(stream)
                torch.cuda.synchronize()
                ms = sum(t0.elapsed_time(t1) for t0, t1 in ev) / reps
                line = {"sweep": True, "mode": "pfb" if mode == workloads.PFB else "direct", "nchan": n,
                        "spectra_per_call": a, "ghz_device": a * n / (ms * 1e-3) / 1e9, "ms_device": ms}
                if nbytes <= pinned.numel():
                    pinned[:nbytes].copy_(d_in.view(torch.uint8).cpu())
                    h_out = torch.empty(plan.out_floats, dtype=torch.float32).pin_memory()
                    plan.execute_host(pinned, a, h_out, stream)
                    torch.cuda.synchronize()
                    t0 = torch.cuda.Event(enable_timing=True)
                    t1 = torch.cuda.Event(enable_timing=True)
                    t0.record(stream)
                    for _ in range(reps):
                        plan.execute_host(pinned, a, h_out, stream)
                    t1.record(stream)
                    torch.cuda.synchronize()
                    hms = t0.elapsed_time(t1) / reps
                    line["ghz_with_copies"] = a * n / (hms * 1e-3) / 1e9
                print(json.dumps(line), flush=True)
                del d_in
            plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the tensor-core and two-kernel comparison runs")
    ap.add_argument("--sweep", action="store_true",
                    help="bandwidth against FFT length and accumulation length (Fig. 3 shape)")
    ap.add_argument("--plan-flags", type=int, default=0,
                    help="VSPEC_PLAN_* flags of the timed plan (profiling other plan forms; 0: the default)")
    ap.add_argument("--nsub", type=int, default=1,
                    help="sub-band mode: NSUB bands of the workload interleaved per sample (vspec_plan_create_sb); "
                         "the rate counts every band; no variants, CPU baseline or end-to-end run")
    ap.add_argument("--spectra", type=int, default=0,
                    help="channelize only the first SPECTRA spectra of the dump (smaller profiling captures)")
    ap.add_argument("--config", choices=["c1", "c2", "c3", "c4", "c5"], default=CONFIG_NAME,
                    help="c4: the 131072-channel PFB dump (default); c1, c2, c3: the other single-bank "
                         "workloads; c5: the batched multi-beam workload")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.sweep:
        if rank == 0:
            run_sweep(args)
        return
    if args.config == "c5":
        if rank == 0:
            run_batch(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
