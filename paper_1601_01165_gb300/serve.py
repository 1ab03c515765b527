"""Real-time multi-beam serving on one GPU with continuous batching.

Section 4.2 asks for each second of data to be dedispersed in under a second,
and Section 5.1 sizes a many-beam instrument by how many beams one device
keeps in real time.  This module runs that as a service:

* every beam delivers chunks of `chunk_len` samples on its own timer
  (period and phase per beam); a chunk's deadline is its arrival time plus
  one period (the next chunk of the same beam);
* a beam is admitted when its device memory need (plan tables, streaming
  state with the max-delay tail, one input chunk, one output chunk) fits in
  the HBM budget next to the beams already running; beams that do not fit
  wait in arrival order and are admitted as running beams finish and free
  their memory;
* each admitted beam owns a CUDA stream; a ready chunk is copied in from
  page-locked host memory, dedispersed by dd_stream_push (tail kept on the
  device) and copied back, so chunks of different beams overlap on the GPU;
* latency = time the result is back in host memory - chunk arrival.

All compute runs in libdd; this is host-side scheduling only.
"""
from __future__ import annotations

import dataclasses
import heapq
import statistics
import time
from typing import Callable

import numpy as np

from . import binding


@dataclasses.dataclass
class BeamSpec:
    name: str
    setup: object              # synth.Setup (geometry; n_out is ignored)
    dtype: str                 # "u8" or "f32"
    chunk_len: int
    n_chunks: int
    period_s: float            # time between chunks (chunk_len * t_samp for real time)
    phase_s: float = 0.0       # first chunk arrives at start + phase
    keep_output: bool = False  # keep every output chunk on the host (tests)


@dataclasses.dataclass
class ChunkRecord:
    beam: str
    index: int
    t0: int
    arrival: float
    done: float

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class _Active:
    def __init__(self, spec: BeamSpec, torch, device):
        s = spec.setup
        self.spec = spec
        self.plan = binding.Plan(s.channels, s.f_low_mhz, s.chan_bw_mhz, s.t_samp_s, s.dm_first, s.dm_step,
                                 s.n_dm, spec.chunk_len, dtype=spec.dtype)
        self.state = binding.Stream(self.plan, spec.chunk_len)
        self.cuda_stream = torch.cuda.Stream(device=device)
        in_dt = self.plan.in_dtype
        self.d_chunk = torch.empty((s.channels, spec.chunk_len), dtype=in_dt, device=device)
        self.d_out = torch.empty((s.n_dm, spec.chunk_len), dtype=self.plan.out_dtype, device=device)
        self.h_in = torch.empty((s.channels, spec.chunk_len), dtype=in_dt, pin_memory=True)
        self.h_out = torch.empty((s.n_dm, spec.chunk_len), dtype=self.plan.out_dtype, pin_memory=True)
        self.pending = None          # (chunk index, arrival, t0, event)
        self.next_chunk = 0
        self.outputs = []

    def close(self):
        self.state.close()
        self.plan.close()


def beam_bytes(spec: BeamSpec) -> int:
    """Device memory a running beam holds, as the library reports it before
    anything is allocated: the beam's plan (dd_plan_footprint), its stream
    (dd_stream_footprint: the stream's own plan and its two state buffers
    with the max-delay tail) and the server's chunk buffers (one input chunk,
    one output chunk)."""
    s = spec.setup
    geo = (s.channels, s.f_low_mhz, s.chan_bw_mhz, s.t_samp_s, s.dm_first, s.dm_step, s.n_dm)
    elem = 1 if spec.dtype == "u8" else 4
    chunks = s.channels * spec.chunk_len * elem + 4 * s.n_dm * spec.chunk_len
    return (binding.plan_footprint(*geo, dtype=spec.dtype) +
            binding.stream_footprint(*geo, spec.chunk_len, dtype=spec.dtype) + chunks)


class AdmissionError(RuntimeError):
    pass


class Server:
    """Continuous-batching dedispersion server for many beams on one GPU."""

    def __init__(self, hbm_budget_bytes: int, device: int = 0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.budget = int(hbm_budget_bytes)

    def run(self, specs: list[BeamSpec], chunk_source: Callable[[BeamSpec, int], np.ndarray],
            time_scale: float = 1.0, poll_s: float = 2e-4) -> dict:
        """Serve all beams until every chunk is processed; returns a report.

        chunk_source(spec, k) returns chunk k of a beam as a host array
        [channels][chunk_len] (called when the chunk arrives).  time_scale
        stretches (>1) or compresses (<1) all periods and phases.
        """
        torch = self.torch
        need = {sp.name: beam_bytes(sp) for sp in specs}
        for sp in specs:
            if need[sp.name] > self.budget:
                raise AdmissionError(f"beam {sp.name} needs {need[sp.name]} bytes, budget {self.budget}")
        waiting = list(specs)
        active: dict[str, _Active] = {}
        in_use = 0
        peak_in_use = 0
        peak_beams = 0
        records: list[ChunkRecord] = []
        outputs: dict[str, list] = {}
        admitted_at: dict[str, float] = {}
        start = time.perf_counter()
        # per-beam arrival clock starts when the beam is admitted
        arrivals: list[tuple[float, str, int]] = []

        def admit():
            nonlocal in_use, peak_in_use, peak_beams
            newly = []
            while waiting and in_use + need[waiting[0].name] <= self.budget:
                sp = waiting.pop(0)
                with torch.cuda.device(self.device):
                    active[sp.name] = _Active(sp, torch, self.device)
                newly.append(sp)
                in_use += need[sp.name]
                peak_in_use = max(peak_in_use, in_use)
                peak_beams = max(peak_beams, len(active))
            # the admitted beams' clocks start together, once all their resources exist
            now = time.perf_counter()
            for sp in newly:
                admitted_at[sp.name] = now
                for k in range(sp.n_chunks):
                    heapq.heappush(arrivals, (now + (sp.phase_s + k * sp.period_s) * time_scale, sp.name, k))

        admit()
        ready: list[tuple[float, str, int]] = []
        with torch.cuda.device(self.device):
            while active or waiting:
                now = time.perf_counter()
                while arrivals and arrivals[0][0] <= now:
                    ready.append(heapq.heappop(arrivals))
                # launch every ready chunk whose beam has nothing in flight (chunks of a beam stay in order)
                still = []
                for (arr, name, k) in sorted(ready):
                    act = active[name]
                    if act.pending is not None or k != act.next_chunk:
                        still.append((arr, name, k))
                        continue
                    torch.cuda.nvtx.range_push(f"chunk {name}:{k}")
                    host = chunk_source(act.spec, k)
                    h = act.h_in
                    h.copy_(torch.from_numpy(np.ascontiguousarray(host)))
                    with torch.cuda.stream(act.cuda_stream):
                        act.d_chunk.copy_(h, non_blocking=True)
                        _, t0 = act.state.push(act.d_chunk, out=act.d_out, stream=act.cuda_stream)
                        act.h_out.copy_(act.d_out, non_blocking=True)
                        ev = torch.cuda.Event()
                        ev.record(act.cuda_stream)
                    torch.cuda.nvtx.range_pop()
                    act.pending = (k, arr, t0, ev, h)
                    act.next_chunk += 1
                ready = still
                # collect finished chunks
                for name in list(active):
                    act = active[name]
                    if act.pending is not None and act.pending[3].query():
                        k, arr, t0, _, _ = act.pending
                        done = time.perf_counter()
                        records.append(ChunkRecord(name, k, t0, arr, done))
                        if act.spec.keep_output:
                            outputs.setdefault(name, []).append((t0, act.h_out.clone()))
                        act.pending = None
                        if act.next_chunk == act.spec.n_chunks:
                            act.cuda_stream.synchronize()
                            act.close()
                            del active[name]
                            in_use -= need[name]
                            admit()
                if not ready and arrivals and all(a.pending is None for a in active.values()):
                    time.sleep(max(0.0, min(poll_s * 10, arrivals[0][0] - time.perf_counter())))
                else:
                    time.sleep(poll_s)
        elapsed = time.perf_counter() - start
        lat = sorted(r.latency for r in records)
        period = {sp.name: sp.period_s * time_scale for sp in specs}
        misses = sum(1 for r in records if r.latency > period[r.beam])
        units = sum(sp.setup.n_dm * sp.chunk_len * sp.n_chunks for sp in specs)
        return {
            "chunks": len(records),
            "latency_p50_s": statistics.median(lat) if lat else None,
            "latency_p99_s": lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None,
            "latency_max_s": lat[-1] if lat else None,
            "deadline_misses": misses,
            "elapsed_s": elapsed,
            "throughput_dm_samples_per_s": units / elapsed if elapsed > 0 else None,
            "peak_beams": peak_beams,
            "peak_bytes": peak_in_use,
            "budget_bytes": self.budget,
            "admitted_at": admitted_at,
            "records": records,
            "outputs": outputs,
        }
