#!/usr/bin/env python3
"""Benchmark: brute-force dedispersion of one Apertif-like beam per GPU.

Workload (one step = one full forward pass, Algorithm 1, over one beam):
1024 channels from 1420 MHz at 0.29296875 MHz, 50 us sampling, 2048 DM
trials from 0 in steps of 0.25, 20,000 output samples (one second) -- the
Apertif setup of Table 2.  Input: seeded synthetic N(0,1) float32 (or
round(N(128,16)) uint8 with --dtype u8) with 3 injected dispersed pulses.

Prints one JSON line.  ``value`` is DM-trial x samples per second over all
ranks (each rank dedisperses its own beam: weak scaling, no collective on the
data path).  ``roofline`` reports the dominant kernel against the roof that
binds it; ``e2e`` measures the same metric through dd_forward_host with
host buffers (copies inside the timed region); ``cpu_baseline`` times the
oracle on a bounded sample of the same workload on this host's cores.

--impl reference times the oracle itself as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1601_01165_gb300 import synth  # noqa: E402

METRIC = "dedispersed DM-trial·samples/s and achieved HBM GB/s (fraction of roofline), 1 GB300"
UNIT = "DM-trial·samples/s"
L2_BYTES = 129 * 1024 * 1024
FP32_LANES_PER_SM = 128
# int32 lanes per SM: 128 on the integer (ALU) pipe plus 128 on the FMA pipe,
# which also runs integer multiply-adds (a probe measured 251 int32 adds per
# clock per SM); the uint8 path's roof counts one int32 add per 8-bit add
INT32_LANES_PER_SM = 256
SM_MAX_MHZ_NOMINAL = 2070.0

# DRAM traffic per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum),
# keyed by (setup name, output samples, kernel config, dtype); valid only while
# the kernel source hash matches.
NCU_TRAFFIC = {
    # fwd_tmw9_kernel<0>: 111.1 MB read + 123.0 MB written
    ("apertif", 20000, "tmw9_f32_d9_t4096", "f32"): {"bytes": 234_030_848, "hash": "e4f86a4a09fcbaf3"},
    # fwd_u8pk_kernel<8,1,4,24,3>: 32.7 MB read + 111.9 MB written
    ("apertif", 20000, "u8pk_w8x1_d4_c24_st3", "u8"): {"bytes": 144_604_928, "hash": "e4f86a4a09fcbaf3"},
}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), float(m.get("sm_max_mhz", SM_MAX_MHZ_NOMINAL)), "measured"
    except Exception:
        return 6800.0, SM_MAX_MHZ_NOMINAL, "fallback"


def _kernel_hash():
    """Hash of the code the forward kernels are built from, comments and blank
    space removed (the traffic figures are tied to it)."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1601_01165_gb300", "csrc")
    for name in ("fwd_kernels.cu", "fwd_tmw6.cu", "fwd_tmw9.cu", "ptx.cuh", "dd_internal.h"):
        with open(os.path.join(csrc, name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


class NvmlSampler:
    """SM clock, power and clock-event reasons read through NVML (libnvidia-ml,
    ctypes) every 5 ms while `active`, so that even a timed region of a few
    tens of milliseconds gets samples.  Reads only; changes no setting."""

    # nvmlClocksEventReasons bits
    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, uuid: str):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) != 0:
            raise RuntimeError(f"no NVML device {uuid}")
        try:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.rows = []
        self.active = False
        self.done = threading.Event()
        self.thread = None

    def _sample(self):
        ct = self.ct
        sm, mx, mw, rs = ct.c_uint(), ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        ok = self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(sm)) == 0      # NVML_CLOCK_SM
        ok = ok and self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ct.byref(mx)) == 0
        pw = self.lib.nvmlDeviceGetPowerUsage(self.h, ct.byref(mw)) == 0
        rok = self.reasons_fn(self.h, ct.byref(rs)) == 0
        if ok:
            self.rows.append((float(sm.value), float(mx.value), mw.value / 1e3 if pw else None,
                              int(rs.value) if rok else None))

    def _run(self):
        while not self.done.is_set():
            if self.active:
                self._sample()
            time.sleep(0.005)

    def start(self):
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def stop(self):
        self.active = False
        self.done.set()
        if self.thread:
            self.thread.join(timeout=2)
        self.lib.nvmlShutdown()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0, "source": "nvml"}
        reasons = set()
        for r in self.rows:
            if r[3] is not None:
                reasons.update(n for n, bit in self.REASONS.items() if r[3] & bit)
        power = [r[2] for r in self.rows if r[2] is not None]
        return {"sm_mhz": statistics.median(r[0] for r in self.rows), "sm_max_mhz": max(r[1] for r in self.rows),
                "reasons": sorted(reasons), "samples": len(self.rows),
                "power_w_max": max(power) if power else None, "source": "nvml, 5 ms"}


def clock_sampler(dev):
    """NVML sampler of the device (by UUID), else the nvidia-smi one."""
    import torch
    uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    try:
        return NvmlSampler(uuid)
    except Exception:
        return ClockSampler(uuid)


class ClockSampler:
    """nvidia-smi sampler (every 50 ms) for SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, ident):
        self.index = ident
        self.rows = []
        self.proc = None
        self.active = False
        self.ready = threading.Event()

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            self.ready.set()
            return
        threading.Thread(target=self._read, daemon=True).start()
        self.ready.wait(timeout=10)

    def _read(self):
        for line in self.proc.stdout:
            self.ready.set()
            if self.active:
                self.rows.append([v.strip() for v in line.split(",")])

    def stop(self):
        self.active = False
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    "source": "nvidia-smi, 50 ms"}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, n in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows),
                "power_w_max": max((float(r[2]) for r in self.rows if _isnum(r[2])), default=None),
                "source": "nvidia-smi, 50 ms"}


def _pct(xs, q):
    ys = sorted(xs)
    return ys[min(len(ys) - 1, int(round(q / 100 * (len(ys) - 1))))]


def _host_cpu():
    """Host CPU model and core count (the CPU baselines run there)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model, "cores": os.cpu_count()}


def _isnum(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(setup, dtype, target_s=12.0, seed=0):
    """Time the oracle (as it stands, single thread) on a bounded sample of the workload:
    a subset of DM trials spread over the whole range, every channel, all samples."""
    import oracle
    oracle.build()
    d = oracle.delay_table(*setup.plan_args()[:7])
    n_in = setup.n_out + int(d.max())
    x = (synth.noise_u8 if dtype == "u8" else synth.noise_f32)(seed, setup.channels, n_in)
    fwd = (lambda dd: oracle.forward_u8(dd, x, setup.n_out)) if dtype == "u8" else \
        (lambda dd: oracle.forward_f32(dd, x, setup.n_out))
    t = time.perf_counter()
    fwd(d[:1])
    per_row = max(time.perf_counter() - t, 1e-4)
    rows = int(max(1, min(setup.n_dm, target_s / per_row)))
    idx = np.linspace(0, setup.n_dm - 1, rows).astype(np.int64)
    sub = np.ascontiguousarray(d[idx])
    t = time.perf_counter()
    fwd(sub)
    el = time.perf_counter() - t
    return {"value": rows * setup.n_out / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{rows} of {setup.n_dm} DM trials (evenly spaced) x {setup.n_out} samples x "
                      f"{setup.channels} channels, {dtype}, single-threaded C oracle, {el:.1f} s"}


def cpu_baseline_parallel(setup, dtype, target_s=8.0, seed=0):
    """The multi-threaded CPU baseline (the paper's CPU comparison): tune threads,
    DM chunk and time block on a small sample, then time a bounded sample of the
    workload on all host cores.  float32 only (the uint8 path is timed as float)."""
    import oracle
    oracle.build()
    d = oracle.delay_table(*setup.plan_args()[:7])
    n_in = setup.n_out + int(d.max())
    x = synth.noise_f32(seed, setup.channels, n_in)
    all_threads = oracle.cpu_threads()
    probe = np.ascontiguousarray(d[np.linspace(0, setup.n_dm - 1, 4 * all_threads).astype(np.int64)])
    best = None
    for threads in sorted({all_threads, max(1, all_threads // 2)}):
        for dm_chunk in (1, 4):
            for t_block in (1024, 4096):
                t = time.perf_counter()
                oracle.forward_f32_parallel(probe, x, setup.n_out, None, threads, dm_chunk, t_block)
                el = time.perf_counter() - t
                if best is None or el < best[0]:
                    best = (el, threads, dm_chunk, t_block)
    _, threads, dm_chunk, t_block = best
    per_row = best[0] / len(probe)
    rows = int(max(1, min(setup.n_dm, target_s / per_row)))
    idx = np.linspace(0, setup.n_dm - 1, rows).astype(np.int64)
    sub = np.ascontiguousarray(d[idx])
    t = time.perf_counter()
    oracle.forward_f32_parallel(sub, x, setup.n_out, None, threads, dm_chunk, t_block)
    el = time.perf_counter() - t
    return {"value": rows * setup.n_out / el, "unit": UNIT, "cores": threads, "kind": "openmp",
            "tuned": {"threads": threads, "dm_chunk": dm_chunk, "t_block": t_block},
            "sample": f"{rows} of {setup.n_dm} DM trials (evenly spaced) x {setup.n_out} samples x "
                      f"{setup.channels} channels, float32 summed in fp64, {el:.1f} s on {threads} threads "
                      f"of {os.cpu_count()} host cores"}


def run_reference(args, setup):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    d = oracle.delay_table(*setup.plan_args()[:7])
    n_in = setup.n_out + int(d.max())
    x = (synth.noise_u8 if args.dtype == "u8" else synth.noise_f32)(0, setup.channels, n_in)
    fwd = (lambda dd: oracle.forward_u8(dd, x, setup.n_out)) if args.dtype == "u8" else \
        (lambda dd: oracle.forward_f32(dd, x, setup.n_out))
    t = time.perf_counter()
    fwd(d[:1])
    per_row = max(time.perf_counter() - t, 1e-4)
    budget_per_step = 150.0 / max(1, args.steps + args.warmup)
    rows = int(max(1, min(setup.n_dm, budget_per_step / per_row)))
    rng = np.random.default_rng(1)
    for _ in range(args.warmup):
        fwd(np.ascontiguousarray(d[rng.choice(setup.n_dm, rows, replace=False)]))
    t = time.perf_counter()
    for _ in range(args.steps):
        fwd(np.ascontiguousarray(d[rng.choice(setup.n_dm, rows, replace=False)]))
    el = time.perf_counter() - t
    value = rows * setup.n_out * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.dtype == "f32" else "int64", "data": "synthetic",
        "config": _config(setup, args, None, None),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: {rows} random DM trials of {setup.n_dm} x {setup.n_out} "
                                   f"samples x {setup.channels} channels, single-threaded C oracle"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(setup, args, cfg_name, l2_note):
    return {"workload": f"{setup.name}-like single beam per GPU: {setup.channels} ch from {setup.f_low_mhz} MHz x "
                        f"{setup.chan_bw_mhz} MHz, t_samp {setup.t_samp_s * 1e6:.0f} us, {setup.n_dm} DM trials "
                        f"step {setup.dm_step}, {setup.n_out} output samples",
            "dtype": args.dtype, "kernel_config": cfg_name, "l2": l2_note,
            "parallelism": f"beams: one per GPU x {args.gpus}"}


def _sm_count(dev) -> int:
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def _rotating_inputs(plan, setup, dtype, dev, seed, make_host=None):
    """Input buffers of the plan's padded stride, enough of them that the
    bytes rotated through exceed twice the L2 (so every launch reads cold)."""
    import torch
    d = plan.delays()
    stride = plan.padded_in_stride()
    elem = 1 if dtype == "u8" else 4
    in_bytes = setup.channels * stride * elem
    n_buf = max(2, int(np.ceil(2 * L2_BYTES / in_bytes)) + 1)
    host_x, _ = _make_input(setup, dtype, seed, plan.n_in, stride, d)
    xs = [torch.from_numpy(host_x).to(dev) for _ in range(n_buf)]
    return host_x, xs, n_buf, in_bytes


def _time_launches(fn, n_buf, steps, warmup, stream):
    """Warm-up, then `steps` launches bracketed by CUDA events on `stream`;
    returns the per-launch times (ms) and the total (ms)."""
    import torch
    for k in range(warmup):
        fn(k % n_buf)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for k in range(steps):
        fn(k % n_buf)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    return [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)], ev[0].elapsed_time(ev[steps])


def _roofline(setup, plan, dtype, avg_ms, sms, sm_max, peak_kind, hbm_gbs, cfg_name):
    """The dominant kernel against the add roof (float: FP32 lanes; uint8:
    int32 lanes), with the HBM fraction of its compulsory bytes beside it."""
    elem = 1 if dtype == "u8" else 4
    adds = setup.adds
    compulsory = setup.channels * plan.n_in * elem + setup.n_dm * setup.n_out * 4 + 4 * setup.n_dm * setup.channels
    lanes = INT32_LANES_PER_SM if dtype == "u8" else FP32_LANES_PER_SM
    add_peak = sms * lanes * sm_max * 1e6 / 1e12      # T adds/s
    achieved_alu = adds / (avg_ms / 1e3) / 1e12
    achieved_hbm = compulsory / (avg_ms / 1e3) / 1e9
    kh = _kernel_hash()
    tr = NCU_TRAFFIC.get((setup.name, setup.n_out, cfg_name, dtype))
    traffic = tr["bytes"] if tr and tr.get("hash") == kh else None
    lane_note = (f"{lanes} int32 lanes (128 ALU + 128 FMA pipe), one int32 add per 8-bit add" if dtype == "u8"
                 else f"{lanes} FP32 lanes, 1 add = 1 op (Eq. 2 counts one add per input sample)")
    return {"bound": "alu", "achieved": achieved_alu, "peak": add_peak,
            "unit": "TFLOP/s" if dtype == "f32" else "Tops", "frac": achieved_alu / add_peak,
            "traffic": traffic,
            "peak_note": f"{sms} SMs x {lane_note}, {sm_max:.0f} MHz ({peak_kind} max clock)",
            "per_launch_ops": adds, "avg_launch_ms": avg_ms,
            "hbm": {"achieved_gbs": achieved_hbm, "peak_gbs": hbm_gbs, "frac": achieved_hbm / hbm_gbs,
                    "compulsory_bytes": compulsory, "peak_kind": peak_kind,
                    "ncu_traffic_gbs": None if traffic is None else traffic / (avg_ms / 1e3) / 1e9,
                    "ncu_traffic_frac": None if traffic is None else traffic / (avg_ms / 1e3) / 1e9 / hbm_gbs},
            # Eq. 2's accounting: every add reads its own input sample (no reuse);
            # an effective rate for comparison with the paper's figures, not bytes moved
            "eq2_effective_gbs": elem * adds / (avg_ms / 1e3) / 1e9}


def _extra_config(setup, dtype, steps, warmup, dev, sms, sm_max, peak_kind, hbm_gbs):
    """One more configuration timed like the headline (cold L2, CUDA events)."""
    import torch
    from paper_1601_01165_gb300 import binding as dd
    plan = dd.Plan.from_setup(setup, dtype)
    _, xs, n_buf, in_bytes = _rotating_inputs(plan, setup, dtype, dev, 0)
    out = torch.empty((setup.n_dm, setup.n_out), dtype=plan.out_dtype, device=dev)
    stream = torch.cuda.current_stream()
    launch_ms, total_ms = _time_launches(lambda k: plan.forward(xs[k], out=out), n_buf, steps, warmup, stream)
    if plan.device_status() != 0:
        raise RuntimeError(f"device status nonzero ({setup.name} {dtype})")
    avg = statistics.fmean(launch_ms)
    res = {"workload": f"{setup.name}-like beam, {setup.channels} ch, {setup.n_dm} DM trials, {setup.n_out} samples",
           "dtype": dtype, "kernel_config": plan.selected, "value": setup.n_dm * setup.n_out / (total_ms / steps / 1e3),
           "unit": UNIT, "ms_per_step": total_ms / steps, "steps": steps,
           "l2": f"{n_buf} rotating input buffers ({n_buf * in_bytes / 2**20:.0f} MiB > 2x L2)",
           "roofline": _roofline(setup, plan, dtype, avg, sms, sm_max, peak_kind, hbm_gbs, plan.selected)}
    del xs, out
    plan.close()
    torch.cuda.empty_cache()
    return res


def _streamed_vs_plain(steps, warmup, dev):
    """Section 4.2's real-time form on the Apertif-like uint8 beam: 1 s chunks
    through dd_stream_push (the max-delay tail stays on the device; only the
    new second is sent) against the plain per-beam launch of the same second
    (dd_forward over n_out = 1 s, whose input must carry the tail again).
    Timed on the device (inputs resident, rotating > 2x L2) and end to end
    from pinned host memory (chunk in, result out, copies timed)."""
    import torch
    from paper_1601_01165_gb300 import binding as dd
    s = synth.APERTIF
    n = s.n_out
    plan = dd.Plan.from_setup(s, "u8")
    st = dd.Stream(plan, n)
    chunk_bytes = s.channels * n
    n_chunks = max(2, int(np.ceil(2 * L2_BYTES / chunk_bytes)) + 1)
    chunks = [torch.from_numpy(synth.noise_u8(100 + k, s.channels, n)).to(dev) for k in range(n_chunks)]
    out_s = torch.empty((s.n_dm, n), dtype=torch.int32, device=dev)
    _, xs, n_buf, in_bytes = _rotating_inputs(plan, s, "u8", dev, 1)
    out_p = torch.empty((s.n_dm, n), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    k_steps = max(5, min(steps, 20))
    st_ms, st_total = _time_launches(lambda k: st.push(chunks[k], out=out_s), n_chunks, k_steps, warmup, stream)
    pl_ms, pl_total = _time_launches(lambda k: plan.forward(xs[k], out=out_p), n_buf, k_steps, warmup, stream)
    # end to end over consecutive seconds from pinned host memory (chunk in,
    # result out, the same output bytes both ways).  The streamed form runs
    # as a real-time pipeline does: second k + 1 is copied in while second k
    # is dedispersed and second k - 1 copied out (a copy-in stream, the push
    # stream, two copy-out streams; two buffers each; the pushes stay in order
    # on one stream).  The plain form calls
    # dd_forward_host once per second (it pipelines time chunks inside the
    # call and returns with the result in host memory).
    h_chunk = torch.from_numpy(synth.noise_u8(7, s.channels, n)).pin_memory()
    h_beam = torch.from_numpy(np.ascontiguousarray(synth.noise_u8(7, s.channels, plan.n_in))).pin_memory()
    h_outs = [torch.empty((s.n_dm, n), dtype=torch.int32, pin_memory=True) for _ in range(2)]
    d_chunks = [torch.empty((s.channels, n), dtype=torch.uint8, device=dev) for _ in range(2)]
    d_outs = [out_s, torch.empty((s.n_dm, n), dtype=torch.int32, device=dev)]
    s_in, s_run = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    s_outs = [torch.cuda.Stream(device=dev) for _ in range(2)]   # copy-outs alternate, as in dd_forward_host
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_run = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def e2e_stream(seconds):
        for k in range(seconds):
            b = k & 1
            if k >= 2:
                s_in.wait_event(ev_run[b])      # the push of second k - 2 has read this chunk buffer
            with torch.cuda.stream(s_in):
                d_chunks[b].copy_(h_chunk, non_blocking=True)
                ev_in[b].record(s_in)
            s_run.wait_event(ev_in[b])
            if k >= 2:
                s_run.wait_event(ev_out[b])     # second k - 2's result has left this output buffer
            st.push(d_chunks[b], out=d_outs[b], stream=s_run)
            ev_run[b].record(s_run)
            s_out = s_outs[b]
            s_out.wait_event(ev_run[b])
            with torch.cuda.stream(s_out):
                h_outs[b].copy_(d_outs[b], non_blocking=True)
                ev_out[b].record(s_out)
        for so in s_outs:
            so.synchronize()

    def e2e_plain(seconds):
        for _ in range(seconds):
            plan.forward_host(h_beam, out=h_outs[0])

    def wall(fn):
        fn(2)
        torch.cuda.synchronize()
        t = time.perf_counter()
        fn(k_steps)
        return (time.perf_counter() - t) / k_steps * 1e3

    e2e_s, e2e_p = wall(e2e_stream), wall(e2e_plain)
    units = s.n_dm * n
    res = {"workload": f"apertif-like uint8 beam, 1 s chunks of {n} samples, {s.n_dm} DM trials",
           "streamed_ms_per_chunk": st_total / k_steps, "plain_ms_per_second": pl_total / k_steps,
           "streamed_value": units / (st_total / k_steps / 1e3), "plain_value": units / (pl_total / k_steps / 1e3),
           "device_speedup_streamed_vs_plain": pl_total / st_total,
           "e2e_streamed_ms": e2e_s, "e2e_plain_ms": e2e_p, "e2e_speedup_streamed_vs_plain": e2e_p / e2e_s,
           "h2d_bytes_streamed": chunk_bytes, "h2d_bytes_plain": s.channels * plan.n_in,
           "note": "the streamed form sends only the new second and pipelines consecutive seconds; the plain "
                   "launch re-sends the max-delay overlap with every second (Section 2.1: n_in = n_out + "
                   "max_delay) and returns with each second's result; on the device alone both run the "
                   "same kernel (the stream adds two device copies: chunk behind the tail, new tail)",
           "unit": UNIT, "steps": k_steps}
    st.close()
    plan.close()
    torch.cuda.empty_cache()
    return res


def _serving_summary(beams, chunks, seed, kernel_ms_u8):
    """A short real-time serving run (Section 4.2 / 5.1): Apertif-like uint8
    beams delivering 1 s chunks on their own timers, continuous batching with
    HBM-budget admission; plus the beams-in-real-time count implied by the
    kernel time of one beam-second."""
    from paper_1601_01165_gb300.serve import BeamSpec, Server, beam_bytes
    base = synth.APERTIF
    rng = np.random.default_rng(seed)
    specs = [BeamSpec(f"beam{b}", base, "u8", chunk_len=base.n_out, n_chunks=chunks,
                      period_s=base.n_out * base.t_samp_s, phase_s=float(rng.uniform(0, 1)))
             for b in range(beams)]
    cache = {}

    def source(sp, k):
        key = k % 4
        if key not in cache:
            cache[key] = synth.noise_u8(seed + key, base.channels, base.n_out)
        return cache[key]

    budget = beams * beam_bytes(specs[0]) + 1
    rep = Server(budget).run(specs, source)
    return {"workload": f"{beams} apertif-like uint8 beams x {chunks} chunks of 1 s, random phases, "
                        f"HBM budget {budget / 2**30:.1f} GiB",
            "chunks": rep["chunks"], "latency_p50_s": rep["latency_p50_s"], "latency_p99_s": rep["latency_p99_s"],
            "latency_max_s": rep["latency_max_s"], "deadline_s": specs[0].period_s,
            "deadline_misses": rep["deadline_misses"], "peak_beams": rep["peak_beams"],
            "beams_realtime_kernel_bound": int(1000.0 / kernel_ms_u8) if kernel_ms_u8 else None,
            "beams_realtime_note": "one beam-second is one forward over 20,000 samples; the kernel-bound count is "
                                   "1 s / that kernel time (the paper's Section 5.1 sizing: 9 beams per HD7970)"}


def run_ours(args, setup):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_1601_01165_gb300 import binding as dd

    plan = dd.Plan.from_setup(setup, args.dtype)
    if args.config:
        plan.select(args.config)
    cfg_name = plan.selected
    elem = 1 if args.dtype == "u8" else 4
    host_x, xs, n_buf, in_bytes = _rotating_inputs(plan, setup, args.dtype, dev, rank)
    out = torch.empty((setup.n_dm, setup.n_out), dtype=plan.out_dtype, device=dev)
    stream = torch.cuda.current_stream()

    for k in range(args.warmup):
        plan.forward(xs[k % n_buf], out=out)
    torch.cuda.synchronize()
    if plan.device_status() != 0:
        raise RuntimeError("device status nonzero after warm-up")

    sampler = clock_sampler(dev)
    sampler.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.active = True
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        plan.forward(xs[k % n_buf], out=out)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    sampler.active = False
    if ws > 1:
        torch.distributed.barrier()
    sampler.stop()
    launch_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    # warm L2: the same input buffer every launch (reported beside the cold-L2 headline)
    warm_ms = None
    if rank == 0 or ws == 1:
        kw = max(5, min(args.steps, 20))
        for _ in range(3):
            plan.forward(xs[0], out=out)
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0.record(stream)
        for _ in range(kw):
            plan.forward(xs[0], out=out)
        w1.record(stream)
        torch.cuda.synchronize()
        warm_ms = w0.elapsed_time(w1) / kw
    total_ms = ev[0].elapsed_time(ev[args.steps])
    if ws > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    units = setup.n_dm * setup.n_out * args.steps * ws
    value = units / (total_ms / 1e3)

    # end to end through the host-buffer entry point (pinned host memory, copies timed)
    e2e = None
    if not args.no_e2e:
        hx = torch.from_numpy(np.ascontiguousarray(host_x[:, :plan.n_in])).pin_memory()
        hout = torch.empty((setup.n_dm, setup.n_out), dtype=plan.out_dtype, pin_memory=True)
        plan.forward_host(hx, out=hout)
        ke = max(3, min(args.steps, 10))
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            plan.forward_host(hx, out=hout)
        el = time.perf_counter() - t0
        if ws > 1:
            t = torch.tensor([el], device=dev, dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": setup.n_dm * setup.n_out * ke * ws / el, "unit": UNIT,
               "h2d_bytes_per_step": int(setup.channels * plan.n_in * elem),
               "d2h_bytes_per_step": int(setup.n_dm * setup.n_out * 4), "steps": ke}

    if plan.device_status() != 0:
        raise RuntimeError("device status nonzero after timed region")
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    hbm_gbs, sm_max, peak_kind = _peaks()
    sms = _sm_count(dev)
    avg_ms = statistics.fmean(launch_ms)
    roof = _roofline(setup, plan, args.dtype, avg_ms, sms, sm_max, peak_kind, hbm_gbs, cfg_name)
    clocks = sampler.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": _config(setup, args, cfg_name,
                          f"{n_buf} rotating input buffers ({n_buf * in_bytes / 2**20:.0f} MiB > 2x L2)"),
        "roofline": roof, "e2e": e2e, "gpu_launches": args.steps, "clocks": clocks,
        "kernel_source_hash": _kernel_hash(),
        "launch_ms": {"min": min(launch_ms), "p10": _pct(launch_ms, 10), "median": statistics.median(launch_ms),
                      "p90": _pct(launch_ms, 90), "max": max(launch_ms), "warm_l2_mean": warm_ms},
    }
    del xs, out
    plan.close()
    torch.cuda.empty_cache()
    # the other configurations of the headline metric, timed the same way (default run only)
    if ws == 1 and not args.no_extra and args.n_out is None and args.workload == "apertif" and \
            args.dtype == "f32" and not args.config:
        ke = max(5, min(args.steps, 20))
        extra = {"apertif_u8": _extra_config(synth.APERTIF, "u8", ke, args.warmup, dev, sms, sm_max, peak_kind,
                                             hbm_gbs),
                 "lofar_f32": _extra_config(synth.LOFAR, "f32", ke, args.warmup, dev, sms, sm_max, peak_kind,
                                            hbm_gbs)}
        extra["streamed_vs_plain_u8"] = _streamed_vs_plain(ke, args.warmup, dev)
        extra["serving_u8"] = _serving_summary(args.serve_beams, 2, args.seed,
                                               extra["apertif_u8"]["ms_per_step"])
        line["extra"] = extra
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(setup, args.dtype)
        line["cpu_baseline_parallel"] = cpu_baseline_parallel(setup, args.dtype)
        line["cpu_baseline"]["host"] = line["cpu_baseline_parallel"]["host"] = _host_cpu()
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batched(args):
    """64 uneven beams (Section 5.1: many beams per device): the batch (one
    CUDA-graph launch: persistent launches per configuration group, each
    taking its beams' tiles longest first, and single launches for the other
    beams, spread over internal streams) against 64 plain launches of the same
    plans, first with each plan's default configuration, then after
    dd_batch_tune has tuned each distinct setup once and timed each persistent
    group against its beams' own launches (both forms then run the tuned
    kernels); also the same graph with one launch per beam and with every
    group persistent."""
    import torch
    from paper_1601_01165_gb300 import binding as dd
    torch.cuda.set_device(0)
    beams = synth.batched_setups(args.seed, args.beams)
    plans, xs, outs = [], [], []
    g = torch.Generator(device="cuda").manual_seed(args.seed)
    for s, dt in beams:
        p = dd.Plan.from_setup(s, dt)
        x = torch.empty((s.channels, p.padded_in_stride()), dtype=p.in_dtype, device="cuda")
        if dt == "u8":
            x.copy_(torch.randint(0, 256, x.shape, generator=g, device="cuda", dtype=torch.int32).to(torch.uint8))
        else:
            x.normal_(generator=g)
        plans.append(p)
        xs.append(x)
        outs.append(torch.empty((s.n_dm, s.n_out), dtype=p.out_dtype, device="cuda"))
    batch = dd.Batch(plans)
    stream = torch.cuda.Stream()
    units = sum(s.n_dm * s.n_out for s, _ in beams)
    adds = sum(s.adds for s, _ in beams)

    def timed(fn, k):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            stream.synchronize()
            ev0.record(stream)
            for _ in range(k):
                fn()
            ev1.record(stream)
        stream.synchronize()
        return ev0.elapsed_time(ev1) / k

    def run_batch():
        batch.run(xs, outs, stream=stream)

    def run_plain():
        for p, x, o in zip(plans, xs, outs):
            p.forward(x, out=o, stream=stream)

    def solo_sum():
        """Sum of each beam's own launch time (each timed alone)."""
        tot = 0.0
        for p, x, o in zip(plans, xs, outs):
            tot += timed(lambda: p.forward(x, out=o, stream=stream), 3)
        return tot

    ms_batch_def = timed(run_batch, args.steps)
    ms_plain_def = timed(run_plain, args.steps)
    t0 = time.perf_counter()
    n_setups = batch.tune(budget_s=args.tune_budget)
    tune_s = time.perf_counter() - t0
    ms_batch = timed(run_batch, args.steps)     # persistent groups where tuning measured them faster
    batch.set_persistent(0)                     # the same graph with one launch per beam
    ms_batch_per_beam = timed(run_batch, args.steps)
    batch.set_persistent(2)                     # every group that can be persistent
    ms_batch_all_persistent = timed(run_batch, args.steps)
    batch.set_persistent(1)
    ms_plain = timed(run_plain, args.steps)
    ms_solo = solo_sum()
    # the batch's results equal the per-beam launches (checked on every beam)
    with torch.cuda.stream(stream):
        run_batch()
        ref = [p.forward(x, stream=stream) for p, x in zip(plans, xs)]
    stream.synchronize()
    same = all(torch.equal(o, r) for o, r in zip(outs, ref))
    line = {"metric": METRIC, "workload": "batched", "value": units / (ms_batch / 1e3), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch,
            "plain_launches_ms": ms_plain, "speedup_vs_plain": ms_plain / ms_batch,
            "default_configs": {"batch_ms": ms_batch_def, "plain_launches_ms": ms_plain_def,
                                "speedup_vs_plain": ms_plain_def / ms_batch_def},
            "tuned_over_default_batch": ms_batch_def / ms_batch, "setups_tuned": n_setups, "tune_s": tune_s,
            "graph_one_launch_per_beam_ms": ms_batch_per_beam,
            "graph_every_group_persistent_ms": ms_batch_all_persistent,
            "batch_over_one_launch_per_beam": ms_batch_per_beam / ms_batch,
            "sum_of_solo_launch_ms": ms_solo, "batch_over_solo_sum": ms_batch / ms_solo,
            "beams": len(beams), "adds_per_step": adds, "batch_equals_plain": same, "gpu_launches": args.steps,
            "config": {"workload": f"{len(beams)} uneven beams (channels 32/256/1024, DMs 256/1024/4096, "
                                   f"10k-200k samples, Apertif/LOFAR grids, mixed uint8/float32), seed {args.seed}; "
                                   f"tuning budget {args.tune_budget} s per setup"}}
    print(json.dumps(line), flush=True)
    return 0 if same else 1


def run_autograd(args):
    """The differentiable configuration: learnable per-channel weights on the
    Apertif-like float beam, dedispersion -> 8-sample boxcar -> -max S/N loss,
    backward to the weights (the adjoint of Algorithm 1 and the per-channel
    dot products).  One step = forward + loss + backward; the value counts
    the forward's DM-trial samples per second of whole steps."""
    import torch
    from paper_1601_01165_gb300 import binding as dd
    from paper_1601_01165_gb300.autograd import boxcar_snr_loss, dedisperse
    torch.cuda.set_device(0)
    setup = synth.APERTIF
    plan = dd.Plan.from_setup(setup, "f32")
    g = torch.Generator(device="cuda").manual_seed(args.seed)
    in_bytes = setup.channels * plan.padded_in_stride() * 4
    n_buf = max(2, -(-2 * L2_BYTES // in_bytes) + 1)
    xs = []
    for _ in range(n_buf):
        x = plan.alloc_input()
        x.normal_(generator=g)
        xs.append(x)
    w = torch.ones(setup.channels, device="cuda", requires_grad=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    parts = [0.0, 0.0, 0.0]
    loss_val = None

    def step(k, timed):
        nonlocal loss_val
        w.grad = None
        if timed:
            ev[0].record()
        out = dedisperse(xs[k % n_buf], w, plan)
        if timed:
            ev[1].record()
        loss = boxcar_snr_loss(out)
        if timed:
            ev[2].record()
        loss.backward()
        if timed:
            ev[3].record()
            torch.cuda.synchronize()
            for j in range(3):
                parts[j] += ev[j].elapsed_time(ev[j + 1])
        loss_val = loss

    for k in range(args.warmup):
        step(k, False)
    torch.cuda.synchronize()
    # whole steps back to back (no synchronisation inside the timed region)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        step(k, False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # the parts, each step synchronised (reported beside the back-to-back time)
    kp = min(args.steps, 10)
    for k in range(kp):
        step(k, True)
    if plan.device_status() != 0:
        raise RuntimeError("device status nonzero after timed region")
    gw = w.grad
    line = {"metric": METRIC, "workload": "autograd", "value": setup.n_dm * setup.n_out / (ms / 1e3), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "forward_ms": parts[0] / kp, "loss_ms": parts[1] / kp, "backward_ms": parts[2] / kp,
            "loss": float(loss_val.item()), "grad_w_finite": bool(torch.isfinite(gw).all().item()),
            "config": {"workload": f"apertif-like beam ({setup.channels} ch, {setup.n_dm} DM trials, {setup.n_out} "
                                   f"samples, float32), learnable channel weights, 8-sample boxcar -max S/N loss, "
                                   f"backward to the weights; {n_buf} rotating inputs > 2x L2",
                       "kernel_config": plan.selected}}
    print(json.dumps(line), flush=True)
    return 0


def run_dm_sweep(args):
    """Auto-tuning across the number of DM trials (Section 4.3, Figs. 3-4): for
    2, 4, ..., 4096 trials on the Apertif grid, and for perfect data reuse
    (dm_step = 0, every delay zero, Section 4.2), time every configuration of
    the plan, keep the fastest, and compare it with the generic one-trial-per-
    thread kernel (Section 5's "generic" code).  Fig. 3's analogue: for every
    case, the distribution of throughput over all configurations timed (a
    histogram of GFLOP/s, one add = one floating-point operation as the paper
    counts), with the tuned and generic values and their ratio."""
    import tempfile
    import torch
    from paper_1601_01165_gb300 import binding as dd
    torch.cuda.set_device(0)
    rows, winners, hists = [], {}, {}
    cases = [(n, synth.APERTIF.dm_step) for n in [2 ** k for k in range(1, 13)]] + [(2048, 0.0)]
    with tempfile.TemporaryDirectory() as tmp:
        for dtype in ("f32", "u8"):
            for n_dm, step in cases:
                s = synth.APERTIF.replace(n_dm=n_dm, dm_step=step)
                plan = dd.Plan.from_setup(s, dtype)
                db = os.path.join(tmp, f"{dtype}_{n_dm}_{step}.jsonl")
                name, ms = plan.tune(budget_s=0.0, db_path=db)
                with open(db) as f:
                    timings = json.loads(f.readline())["timings"]
                generic = min(v for k, v in timings.items() if k.startswith("naive"))
                fam = name.split("_")[0]
                winners[f"{dtype}:{fam}"] = winners.get(f"{dtype}:{fam}", 0) + 1
                gflops = {k: s.adds / (v / 1e3) / 1e9 for k, v in timings.items()}
                vals = np.array(sorted(gflops.values()))
                edges = np.linspace(vals[0], vals[-1], 9) if vals[-1] > vals[0] else np.array([vals[0], vals[0] + 1])
                counts, _ = np.histogram(vals, edges)
                key = f"{dtype}:{n_dm}" + (":perfect-reuse" if step == 0.0 else "")
                hists[key] = {"gflops_bin_edges": [round(float(e), 1) for e in edges],
                              "configs_per_bin": [int(c) for c in counts],
                              "configs": int(len(vals)), "median_gflops": float(np.median(vals)),
                              "tuned_gflops": float(vals[-1]), "generic_gflops": s.adds / (generic / 1e3) / 1e9,
                              "tuned_over_generic": generic / ms, "tuned_config": name}
                rows.append({"dtype": dtype, "n_dm": n_dm, "dm_step": step, "tuned": name, "tuned_ms": ms,
                             "generic_ms": generic, "speedup_vs_generic": generic / ms,
                             "dm_samples_per_s": n_dm * s.n_out / (ms / 1e3), "configs_timed": len(timings)})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
                plan.close()
    units = sum(r["n_dm"] * synth.APERTIF.n_out for r in rows)
    total_ms = sum(r["tuned_ms"] for r in rows)
    line = {"metric": METRIC, "workload": "dm-sweep", "value": units / (total_ms / 1e3), "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "rows": rows, "histogram": hists, "winning_families": winners,
            "config": {"workload": "Apertif grid (1024 ch, 20000 samples), 2..4096 DM trials step 0.25, "
                                   "plus 2048 trials at dm_step 0; float32 and uint8; every configuration timed "
                                   "(median of 5 after 2 warm-ups, warm L2); histogram: GFLOP/s over the "
                                   "configurations of each case, 8 equal bins from slowest to fastest"}}
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """Real-time serving: Apertif-like uint8 beams delivering 1 s chunks on independent timers."""
    import torch
    from paper_1601_01165_gb300.serve import BeamSpec, Server, beam_bytes
    torch.cuda.set_device(0)
    base = synth.APERTIF
    rng = np.random.default_rng(args.seed)
    specs = [BeamSpec(f"beam{b}", base, "u8", chunk_len=base.n_out, n_chunks=args.chunks,
                      period_s=base.n_out * base.t_samp_s, phase_s=float(rng.uniform(0, 1)))
             for b in range(args.beams)]
    cache = {}

    def source(sp, k):
        key = k % 4
        if key not in cache:
            cache[key] = synth.noise_u8(args.seed + key, base.channels, base.n_out)
        return cache[key]

    budget = int(args.budget_gb * 2**30) if args.budget_gb else args.beams * beam_bytes(specs[0]) + 1
    rep = Server(budget).run(specs, source)
    line = {"metric": METRIC, "workload": "serving", "unit": UNIT, "n_gpus": 1,
            "value": rep["throughput_dm_samples_per_s"], "beams": args.beams, "chunks": rep["chunks"],
            "latency_p50_s": rep["latency_p50_s"], "latency_p99_s": rep["latency_p99_s"],
            "latency_max_s": rep["latency_max_s"], "deadline_s": specs[0].period_s,
            "deadline_misses": rep["deadline_misses"], "peak_beams": rep["peak_beams"],
            "peak_bytes": rep["peak_bytes"], "budget_bytes": rep["budget_bytes"],
            "config": {"workload": f"{args.beams} Apertif-like uint8 beams, 1 s chunks ({base.n_out} samples), "
                                   f"{args.chunks} chunks each, random phases, HBM budget {budget / 2**30:.1f} GiB"}}
    print(json.dumps(line), flush=True)
    return 0


def _make_input(setup, dtype, seed, n_in, stride, d):
    x = (synth.noise_u8 if dtype == "u8" else synth.noise_f32)(seed, setup.channels, n_in, stride)
    for i_p, t_p in synth.pulse_sites(seed, setup.n_dm, setup.n_out, 3):
        synth.inject_pulse(x, d[i_p], t_p, 3, 40.0 if dtype == "u8" else 5.0)
    return x, None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--dtype", choices=["f32", "u8"], default="f32")
    ap.add_argument("--config", default=None, help="kernel configuration name (default: plan's choice)")
    ap.add_argument("--workload", choices=["apertif", "lofar", "batched", "serving", "dm-sweep", "autograd"],
                    default="apertif")
    ap.add_argument("--beams", type=int, default=None, help="batched: 64, serving: 40")
    ap.add_argument("--chunks", type=int, default=4, help="serving: chunks per beam")
    ap.add_argument("--budget-gb", type=float, default=None, help="serving: HBM budget")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--n-out", type=int, default=None,
                    help="output samples per beam instead of the setup's (smaller cases for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="default run: skip the uint8, LOFAR, streamed and serving lines beside the headline")
    ap.add_argument("--serve-beams", type=int, default=40, help="beams of the default run's short serving line")
    ap.add_argument("--tune-budget", type=float, default=1.5, help="batched: dd_tune budget per setup (s)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload == "batched":
        args.beams = args.beams or 64
        return run_batched(args)
    if args.workload == "serving":
        args.beams = args.beams or 40
        return run_serving(args)
    if args.workload == "dm-sweep":
        return run_dm_sweep(args)
    if args.workload == "autograd":
        return run_autograd(args)
    setup = synth.APERTIF if args.workload == "apertif" else synth.LOFAR
    if args.n_out:
        setup = setup.replace(n_out=args.n_out)
    if args.impl == "reference":
        return run_reference(args, setup)
    return run_ours(args, setup)


if __name__ == "__main__":
    sys.exit(main())
