"""Shared helpers for the parity tests (imports the oracle; test-only)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1601_01165_gb300 import synth

# fp32 parity bar: |gpu - oracle| <= FP32_REL * sum_c |w_c * in[c][t + d]| (+ FP32_ABS)
FP32_REL = 1e-5
FP32_ABS = 1e-6


def oracle_table(setup):
    return oracle.delay_table(*setup.plan_args()[:7])


def make_input(setup, dtype, seed, n_in, row_stride=None, pulses=0, d=None, width=3):
    """Seeded input of the setup's shape with optional dispersed pulses (placed with table d)."""
    if dtype == "u8":
        x = synth.noise_u8(seed, setup.channels, n_in, row_stride)
        amp = 40.0
    else:
        x = synth.noise_f32(seed, setup.channels, n_in, row_stride)
        amp = 5.0
    sites = []
    if pulses:
        sites = synth.pulse_sites(seed, setup.n_dm, setup.n_out, pulses, width)
        for i_p, t_p in sites:
            synth.inject_pulse(x, d[i_p], t_p, width, amp)
    return x, sites


def oracle_window(d, x, dtype, i0, i1, t0, n_w, w=None):
    """Oracle output rows [i0, i1) x samples [t0, t0 + n_w) and the fp32 error scale."""
    sub = np.ascontiguousarray(d[i0:i1])
    md = int(sub.max())
    xw = np.ascontiguousarray(x[:, t0:t0 + n_w + md])
    if dtype == "u8":
        return oracle.forward_u8(sub, xw, n_w), None
    ref = oracle.forward_f32(sub, xw, n_w, w)
    scale = oracle.forward_f32(sub, np.abs(xw), n_w, None if w is None else np.abs(w))
    return ref, scale


def assert_parity(got, ref, scale, dtype, where=""):
    got = np.asarray(got)
    if dtype == "u8":
        bad = np.argwhere(got != ref)
        assert bad.size == 0, f"{where}: {len(bad)} integer mismatches, first at {bad[:3].tolist()}: " \
                              f"got {got[tuple(bad[0])]} want {ref[tuple(bad[0])]}"
    else:
        err = np.abs(got.astype(np.float64) - ref)
        lim = FP32_REL * scale + FP32_ABS
        bad = np.argwhere(err > lim)
        assert bad.size == 0, f"{where}: {len(bad)} fp32 mismatches, first at {bad[:3].tolist()}: " \
                              f"err {err[tuple(bad[0])]} lim {lim[tuple(bad[0])]}"
