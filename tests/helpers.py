"""Shared helpers for the parity tests (imports the oracle; test-only)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1601_01165_gb300 import synth

# fp32 parity bar, per output element: |gpu - oracle| <= FP32_REL * sum_c |w_c * in[c][t + d]|,
# the oracle summing in fp64.  No absolute slack: where every term is zero both
# sides are exactly zero.
FP32_REL = 1e-5


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
        lim = FP32_REL * scale
        bad = np.argwhere(err > lim)
        assert bad.size == 0, f"{where}: {len(bad)} fp32 mismatches, first at {bad[:3].tolist()}: " \
                              f"err {err[tuple(bad[0])]} lim {lim[tuple(bad[0])]}"


def full_parity(d, x, dtype, outputs, w=None, n_out=None, rows_per_job=None, workers=None):
    """Compare whole GPU outputs with the oracle, every element.

    ``outputs`` maps a label to a host array [n_dm][n_out] (several kernels'
    outputs of the same input share one oracle pass).  The oracle (single-
    threaded C) runs on blocks of DM rows in a thread pool: ctypes releases
    the GIL, so the blocks run on all host cores.  Returns
    {label: (mismatches, worst error / (FP32_REL * scale) or 0 for integers)}.
    """
    import os
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    n_dm = d.shape[0]
    n_out = next(iter(outputs.values())).shape[1] if n_out is None else n_out
    x = np.ascontiguousarray(x)
    ax = np.abs(x) if dtype != "u8" else None
    aw = None if w is None else np.abs(w)
    workers = workers or max(1, os.cpu_count() or 1)
    if rows_per_job is None:
        # about 64 MB of fp64 per job and per array, and at least 4 jobs per worker
        rows_per_job = max(1, min(n_dm // (4 * workers) or 1, (64 << 20) // (8 * n_out)))
    blocks = [(i0, min(n_dm, i0 + rows_per_job)) for i0 in range(0, n_dm, rows_per_job)]

    def job(blk):
        i0, i1 = blk
        sub = np.ascontiguousarray(d[i0:i1])
        res = {}
        if dtype == "u8":
            ref = oracle.forward_u8(sub, x, n_out)
            for k, got in outputs.items():
                res[k] = (int(np.count_nonzero(got[i0:i1] != ref)), 0.0)
        else:
            ref = oracle.forward_f32(sub, x, n_out, w)
            scale = oracle.forward_f32(sub, ax, n_out, aw)
            lim = FP32_REL * scale
            for k, got in outputs.items():
                err = np.abs(got[i0:i1].astype(np.float64) - ref)
                bad = int(np.count_nonzero(err > lim))
                # lim is 0 only where every term is 0; an error there gives a huge ratio
                res[k] = (bad, float((err / np.maximum(lim, 1e-300)).max()))
        return res

    total = {k: (0, 0.0) for k in outputs}
    with ThreadPoolExecutor(max_workers=workers) as pool:
        for res in pool.map(job, blocks):
            for k, (b, r) in res.items():
                tb, tr = total[k]
                total[k] = (tb + b, max(tr, r))
    return total
