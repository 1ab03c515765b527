"""Seeded synthetic inputs shaped like the paper's two survey setups.

This module holds no dedispersion arithmetic: it draws noise, places pulses at
sample positions the caller supplies (a delay row computed by whichever side
is under test) and describes observational setups.  Both the CUDA path's tests
and the oracle's tests use it, so the two sides see identical inputs.

Setups follow Table 2 (Section 3): LOFAR (32 channels, 200 kHz sampling,
138 MHz up) and Apertif (1024 channels, 20 kHz sampling, 1420 MHz up), plus a
tiny case for fast checks.  DM trials start at ``dm_first`` and step by
``dm_step`` (Section 3 uses 0.25 from 0).  The output covers ``n_out`` samples,
one second of data for the survey setups (Section 2.1).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Setup:
    name: str
    channels: int
    f_low_mhz: float
    chan_bw_mhz: float
    t_samp_s: float
    dm_first: float
    dm_step: float
    n_dm: int
    n_out: int

    def plan_args(self):
        return (self.channels, self.f_low_mhz, self.chan_bw_mhz, self.t_samp_s,
                self.dm_first, self.dm_step, self.n_dm, self.n_out)

    def replace(self, **kw) -> "Setup":
        return dataclasses.replace(self, **kw)

    @property
    def dm_samples(self) -> int:
        """Output elements (DM trials x samples) one forward pass produces."""
        return self.n_dm * self.n_out

    @property
    def adds(self) -> int:
        """Additions Algorithm 1 performs: d x s x c (Section 2.1)."""
        return self.n_dm * self.n_out * self.channels


TINY = Setup("tiny", 64, 1400.0, 1.0, 1e-3, 0.0, 1.0, 32, 1024)
APERTIF = Setup("apertif", 1024, 1420.0, 0.29296875, 50e-6, 0.0, 0.25, 2048, 20000)
LOFAR = Setup("lofar", 32, 138.0, 0.1953125, 5e-6, 0.0, 0.01, 4096, 200000)
SETUPS = {s.name: s for s in (TINY, APERTIF, LOFAR)}


def noise_f32(seed: int, channels: int, n_in: int, row_stride: int | None = None) -> np.ndarray:
    """i.i.d. N(0, 1) float32, shape [channels][row_stride] (columns >= n_in are 0)."""
    rng = np.random.default_rng(seed)
    stride = n_in if row_stride is None else row_stride
    x = np.zeros((channels, stride), dtype=np.float32)
    x[:, :n_in] = rng.standard_normal((channels, n_in), dtype=np.float32)
    return x


def noise_u8(seed: int, channels: int, n_in: int, row_stride: int | None = None,
             mean: float = 128.0, sd: float = 16.0) -> np.ndarray:
    """round(N(mean, sd)) clipped to [0, 255] as uint8, shape [channels][row_stride]."""
    rng = np.random.default_rng(seed)
    stride = n_in if row_stride is None else row_stride
    x = np.zeros((channels, stride), dtype=np.uint8)
    v = np.rint(rng.normal(mean, sd, size=(channels, n_in)))
    x[:, :n_in] = np.clip(v, 0, 255).astype(np.uint8)
    return x


def inject_pulse(x: np.ndarray, arrival: np.ndarray, t0: int, width: int, amplitude: float) -> None:
    """Add a boxcar pulse in place: x[c][t0 + arrival[c] + k] += amplitude for k < width.

    ``arrival`` is the per-channel sample offset of the pulse (the delay row of
    the pulse's DM, supplied by the caller).  uint8 input saturates at 0/255.
    """
    C = x.shape[0]
    for c in range(C):
        lo = t0 + int(arrival[c])
        if x.dtype == np.uint8:
            seg = x[c, lo:lo + width].astype(np.int32) + int(round(amplitude))
            x[c, lo:lo + width] = np.clip(seg, 0, 255).astype(np.uint8)
        else:
            x[c, lo:lo + width] += np.float32(amplitude)


def pulse_sites(seed: int, n_dm: int, n_out: int, count: int, width: int = 3):
    """Seeded (dm_index, t0) pairs with t0 + width <= n_out, distinct DM indices."""
    rng = np.random.default_rng(seed + 7919)
    dms = rng.choice(n_dm, size=count, replace=False)
    ts = rng.integers(0, n_out - width, size=count)
    return [(int(i), int(t)) for i, t in zip(dms, ts)]


def weights(seed: int | None, channels: int) -> np.ndarray:
    """Per-channel weights: all ones if seed is None, else U(0.5, 1.5)."""
    if seed is None:
        return np.ones(channels, dtype=np.float32)
    rng = np.random.default_rng(seed + 104729)
    return rng.uniform(0.5, 1.5, size=channels).astype(np.float32)


def batched_setups(seed: int, beams: int = 64):
    """Uneven beam setups for one batched launch.

    Channels from {32, 256, 1024}, DM trials from {256, 1024, 4096}, output
    length uniform in [10000, 200000], and either the Apertif-like or the
    LOFAR-like frequency/sampling grid with the grid's total bandwidth kept
    (chan_bw = bandwidth / channels).  Returns a list of (Setup, dtype) with
    dtype 'u8' or 'f32'.
    """
    rng = np.random.default_rng(seed + 31337)
    grids = {
        "apertif": (1420.0, 300.0, 50e-6, 0.25),
        "lofar": (138.0, 6.25, 5e-6, 0.01),
    }
    out = []
    for b in range(beams):
        C = int(rng.choice([32, 256, 1024]))
        n_dm = int(rng.choice([256, 1024, 4096]))
        n_out = int(rng.integers(10000, 200001))
        gname = "apertif" if rng.random() < 0.5 else "lofar"
        f_low, bw, t_samp, step = grids[gname]
        dtype = "u8" if rng.random() < 0.5 else "f32"
        out.append((Setup(f"beam{b}-{gname}", C, f_low, bw / C, t_samp, 0.0, step, n_dm, n_out), dtype))
    return out
