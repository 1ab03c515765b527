"""Oracle for brute-force incoherent dedispersion: test infrastructure only.

This package is the slow, plainly correct CPU statement of what the CUDA
library computes.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library itself never does
and shares no code with it.

Two independent forms live here:

* ``dd_oracle.c`` (compiled by :func:`build` with gcc, loaded with ctypes):
  Eq. 1 for the delay table and Algorithm 1 for the forward sum, plus the
  transpose, the weight gradient and the boxcar S/N loss, all accumulated in
  fp64 / int64.
* ``brute_*`` functions below: the same definitions as pure-Python loops over
  numpy scalars, for tiny inputs only, as a second opinion on the C code.

Beside the oracle, ``cpu_parallel.c`` is the multi-threaded CPU baseline (the
paper's CPU comparison, Section 5): the oracle's fp64 sum with DM trials
spread over the host's cores, used only by ``bench.py``'s CPU-baseline leg
and checked bit for bit against the oracle in the tests.

Each function cites the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_PAR_SRC = os.path.join(_HERE, "cpu_parallel.c")
_PAR_SO = os.path.join(_BUILD, "libcpuparallel.so")
_lock = threading.Lock()
_lib = None
_par = None


def build(force: bool = False) -> str:
    """Compile ``dd_oracle.c`` into ``oracle/_build/liboracle.so`` (plain gcc -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    if force or not os.path.exists(_PAR_SO) or os.path.getmtime(_PAR_SO) < os.path.getmtime(_PAR_SRC):
        tmp = _PAR_SO + f".tmp{os.getpid()}"
        base = ["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _PAR_SRC, "-o", tmp]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:   # no OpenMP: the same code, one thread
            subprocess.check_call(base)
        os.replace(tmp, _PAR_SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, dbl, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            lib.orc_delay_table.argtypes = [i32, dbl, dbl, dbl, dbl, dbl, i32, vp]
            lib.orc_delay_table.restype = ctypes.c_int
            lib.orc_max_delay.argtypes = [vp, i32, i32]
            lib.orc_max_delay.restype = i32
            for name in ("orc_forward_f32", "orc_adjoint_f32", "orc_wgrad_f32"):
                getattr(lib, name).argtypes = [i32, i32, i64, i64, vp, vp, vp, vp]
                getattr(lib, name).restype = ctypes.c_int
            lib.orc_forward_u8.argtypes = [i32, i32, i64, i64, vp, vp, vp]
            lib.orc_forward_u8.restype = ctypes.c_int
            lib.orc_boxcar_snr_loss.argtypes = [i32, i64, vp, vp, vp, vp, vp]
            lib.orc_boxcar_snr_loss.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with oracle code {rc}")


def _load_parallel():
    global _par
    with _lock:
        if _par is None:
            build()
            lib = ctypes.CDLL(_PAR_SO)
            i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
            lib.cpb_max_threads.argtypes = []
            lib.cpb_max_threads.restype = ctypes.c_int
            lib.cpb_forward_f32.argtypes = [i32, i32, i64, i64, vp, vp, vp, vp, i32, i32, i32]
            lib.cpb_forward_f32.restype = ctypes.c_int
            _par = lib
    return _par


# ---------------------------------------------------------------- C-backed API

def delay_table(C: int, f_low: float, chan_bw: float, t_samp: float,
                dm_first: float, dm_step: float, n_dm: int) -> np.ndarray:
    """Eq. 1 (Section 2) in samples, rounded half up: int32 [n_dm][C]."""
    d = np.empty((n_dm, C), dtype=np.int32)
    _check(_load().orc_delay_table(C, f_low, chan_bw, t_samp, dm_first, dm_step, n_dm, _ptr(d)),
           "delay_table")
    return d


def max_delay(d: np.ndarray) -> int:
    """Largest entry of a delay table (lowest channel, highest DM trial)."""
    d = np.ascontiguousarray(d, dtype=np.int32)
    return int(_load().orc_max_delay(_ptr(d), d.shape[1], d.shape[0]))


def forward_f32(d: np.ndarray, x: np.ndarray, n_out: int, w: np.ndarray | None = None) -> np.ndarray:
    """Algorithm 1 (Section 2.1) on float32 input, summed in fp64: [n_dm][n_out] float64."""
    d = np.ascontiguousarray(d, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float32)
    n_dm, C = d.shape
    out = np.empty((n_dm, n_out), dtype=np.float64)
    _check(_load().orc_forward_f32(C, n_dm, n_out, x.shape[1], _ptr(d), _ptr(x), _ptr(w), _ptr(out)),
           "forward_f32")
    return out


def forward_u8(d: np.ndarray, x: np.ndarray, n_out: int) -> np.ndarray:
    """Algorithm 1 (Section 2.1) on uint8 input, summed in int64: [n_dm][n_out] int32."""
    d = np.ascontiguousarray(d, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.uint8)
    n_dm, C = d.shape
    out = np.empty((n_dm, n_out), dtype=np.int32)
    _check(_load().orc_forward_u8(C, n_dm, n_out, x.shape[1], _ptr(d), _ptr(x), _ptr(out)),
           "forward_u8")
    return out


def adjoint_f32(d: np.ndarray, grad_out: np.ndarray, n_in: int, w: np.ndarray | None = None) -> np.ndarray:
    """Transpose of weighted Algorithm 1: grad_in [C][n_in] float64."""
    d = np.ascontiguousarray(d, dtype=np.int32)
    g = np.ascontiguousarray(grad_out, dtype=np.float32)
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float32)
    n_dm, C = d.shape
    gi = np.empty((C, n_in), dtype=np.float64)
    _check(_load().orc_adjoint_f32(C, n_dm, g.shape[1], n_in, _ptr(d), _ptr(g), _ptr(w), _ptr(gi)),
           "adjoint_f32")
    return gi


def wgrad_f32(d: np.ndarray, grad_out: np.ndarray, x: np.ndarray) -> np.ndarray:
    """d/dw of weighted Algorithm 1 contracted with grad_out: [C] float64."""
    d = np.ascontiguousarray(d, dtype=np.int32)
    g = np.ascontiguousarray(grad_out, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    n_dm, C = d.shape
    gw = np.empty((C,), dtype=np.float64)
    _check(_load().orc_wgrad_f32(C, n_dm, g.shape[1], x.shape[1], _ptr(d), _ptr(g), _ptr(x), _ptr(gw)),
           "wgrad_f32")
    return gw


def boxcar_snr_loss(out: np.ndarray, want_grad: bool = True):
    """8-sample boxcar, per-DM S/N, loss = -max S/N.  Returns (loss, grad|None, (i, t))."""
    o = np.ascontiguousarray(out, dtype=np.float64)
    n_dm, n_out = o.shape
    loss = np.zeros(1, dtype=np.float64)
    bi = np.zeros(1, dtype=np.int32)
    bt = np.zeros(1, dtype=np.int64)
    g = np.empty_like(o) if want_grad else None
    _check(_load().orc_boxcar_snr_loss(n_dm, n_out, _ptr(o), _ptr(loss), _ptr(g), _ptr(bi), _ptr(bt)),
           "boxcar_snr_loss")
    return float(loss[0]), g, (int(bi[0]), int(bt[0]))


# ------------------------------------------------- pure-Python second opinion

def brute_delay(C, f_low, chan_bw, t_samp, dm_first, dm_step, n_dm):
    """Eq. 1 with Python floats, one entry at a time (tiny sizes only)."""
    f_h = f_low + (C - 1) * chan_bw
    d = np.zeros((n_dm, C), dtype=np.int64)
    for i in range(n_dm):
        dm = dm_first + i * dm_step
        for c in range(C):
            f = f_low + c * chan_bw
            x = 4150.0 * dm * (1.0 / f ** 2 - 1.0 / f_h ** 2) / t_samp
            d[i, c] = int(np.floor(x + 0.5))
    return d


def brute_forward(d, x, n_out, w=None):
    """Algorithm 1 as literal Python loops (tiny sizes only)."""
    n_dm, C = d.shape
    out = np.zeros((n_dm, n_out), dtype=np.float64 if x.dtype != np.uint8 else np.int64)
    for dm in range(n_dm):
        for s in range(n_out):
            acc = 0
            for c in range(C):
                v = x[c, s + d[dm, c]]
                acc += (float(w[c]) * float(v)) if w is not None else (int(v) if x.dtype == np.uint8 else float(v))
            out[dm, s] = acc
    return out


# ------------------------------------------------- multi-threaded CPU baseline

def cpu_threads() -> int:
    """Threads the multi-threaded baseline uses by default (1 without OpenMP)."""
    return int(_load_parallel().cpb_max_threads())


def forward_f32_parallel(d: np.ndarray, x: np.ndarray, n_out: int, w: np.ndarray | None = None,
                         threads: int = 0, dm_chunk: int = 4, t_block: int = 2048) -> np.ndarray:
    """Algorithm 1 on the host's cores: the oracle's fp64 sums, bit for bit.

    threads = 0 uses every core; DM trials go to threads in chunks of
    ``dm_chunk``; time runs in blocks of ``t_block`` samples."""
    d = np.ascontiguousarray(d, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float32)
    n_dm, C = d.shape
    out = np.empty((n_dm, n_out), dtype=np.float64)
    _check(_load_parallel().cpb_forward_f32(C, n_dm, n_out, x.shape[1], _ptr(d), _ptr(x), _ptr(w), _ptr(out),
                                            threads, dm_chunk, t_block), "forward_f32_parallel")
    return out
