"""ctypes binding over the libdd C ABI (include/dd.h).

Argument marshalling only: every step of the computation runs in libdd's
CUDA kernels.  Tensors are torch tensors on the plan's device (PyTorch serves
for device memory and streams); the current torch stream is passed as the
``cudaStream_t`` unless one is given.  A missing or unloadable libdd raises;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

DD_U8_I32 = 0
DD_F32_F32 = 1
_DTYPES = {"u8": DD_U8_I32, "f32": DD_F32_F32}

STATUS = {0: "DD_OK", 1: "DD_ERR_ARG", 2: "DD_ERR_SHAPE", 3: "DD_ERR_ALIGN", 4: "DD_ERR_NOMEM",
          5: "DD_ERR_CUDA", 6: "DD_ERR_UNSUPPORTED", 7: "DD_ERR_BUDGET", 8: "DD_ERR_STATE"}


class DDError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        self.name = STATUS.get(status, f"status {status}")
        super().__init__(f"{where}: {self.name}: {detail}")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libdd.so (building it first if it is missing and nvcc is present).
    The environment variable DD_LIBRARY may name another build of the library
    (the tests use it for the checked build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("DD_LIBRARY") or _build.LIB
        if not os.path.exists(path):
            if os.environ.get("DD_LIBRARY"):
                raise RuntimeError(f"DD_LIBRARY names a missing file: {path}")
            if not build_if_missing:
                raise RuntimeError(f"libdd.so is not built ({path}); run __graft_entry__.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        _declare(lib)
        _lib = lib
        return lib


def _declare(lib):
    i32, i64, dbl, vp, st = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
    P32, P64, PD = ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(dbl)
    sig = {
        "dd_plan": (st, [ctypes.POINTER(vp), i32, dbl, dbl, dbl, dbl, dbl, i32, i64, st]),
        "dd_plan_dm_range": (st, [ctypes.POINTER(vp), i32, dbl, dbl, dbl, dbl, dbl, i32, i32, i64, st]),
        "dd_delay_table": (st, [i32, dbl, dbl, dbl, dbl, dbl, i32, vp]),
        "dd_delay_table_dm_range": (st, [i32, dbl, dbl, dbl, dbl, dbl, i32, i32, vp]),
        "dd_plan_destroy": (st, [vp]),
        "dd_plan_info": (st, [vp, P64, P32, P64]),
        "dd_plan_delays": (st, [vp, vp]),
        "dd_plan_in_stride": (st, [vp, P64]),
        "dd_plan_num_configs": (st, [vp, P32]),
        "dd_plan_config_name": (ctypes.c_char_p, [vp, i32]),
        "dd_plan_select_config": (st, [vp, i32]),
        "dd_plan_selected_config": (st, [vp, P32]),
        "dd_plan_device_status": (st, [vp, P32]),
        "dd_check_wait_timeout": (st, [vp, i64, vp]),
        "dd_forward": (st, [vp, vp, i64, vp, vp, i64, vp]),
        "dd_forward_host": (st, [vp, vp, i64, vp, vp, i64, vp]),
        "dd_adjoint": (st, [vp, vp, i64, vp, vp, i64, vp, i64, vp, vp]),
        "dd_batch_create": (st, [ctypes.POINTER(vp), ctypes.POINTER(vp), i32]),
        "dd_batch_run": (st, [vp, ctypes.POINTER(vp), P64, ctypes.POINTER(vp), P64, vp]),
        "dd_batch_destroy": (st, [vp]),
        "dd_batch_tune": (st, [vp, dbl, ctypes.c_char_p, P32]),
        "dd_batch_set_persistent": (st, [vp, i32]),
        "dd_stream_create": (st, [ctypes.POINTER(vp), vp, i64]),
        "dd_stream_push": (st, [vp, vp, vp, P64, vp]),
        "dd_stream_reset": (st, [vp, vp]),
        "dd_stream_state_bytes": (st, [vp, P64]),
        "dd_stream_device_bytes": (st, [vp, P64]),
        "dd_plan_footprint": (st, [i32, dbl, dbl, dbl, dbl, dbl, i32, st, P64]),
        "dd_stream_footprint": (st, [i32, dbl, dbl, dbl, dbl, dbl, i32, i64, st, P64]),
        "dd_stream_save": (st, [vp, vp, vp]),
        "dd_stream_restore": (st, [vp, vp, vp]),
        "dd_stream_destroy": (st, [vp]),
        "dd_tune": (st, [vp, dbl, ctypes.c_char_p, PD]),
        "dd_boxcar_snr": (st, [vp, i64, i32, i64, vp, vp, i64, vp]),
        "dd_status_string": (ctypes.c_char_p, [st]),
        "dd_last_error": (ctypes.c_char_p, []),
        "dd_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args


def check(status: int, where: str):
    if status != 0:
        detail = load().dd_last_error()
        raise DDError(status, where, detail.decode() if detail else "")


def _stream_handle(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def delay_table(channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, n_dm, dm_index0=0) -> np.ndarray:
    """Eq. 1 delay table as libdd computes it (host only, no GPU needed): rows
    of trials dm_index0 .. dm_index0 + n_dm - 1 of the DM grid."""
    out = np.empty((n_dm, channels), dtype=np.int32)
    check(load().dd_delay_table_dm_range(channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, dm_index0,
                                         n_dm, out.ctypes.data_as(ctypes.c_void_p)), "dd_delay_table_dm_range")
    return out


def plan_footprint(channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, n_dm, dtype="f32") -> int:
    """Device bytes a plan of this geometry holds (dd_plan_footprint; host only)."""
    n = ctypes.c_int64()
    check(load().dd_plan_footprint(channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, n_dm,
                                   _DTYPES[dtype], ctypes.byref(n)), "dd_plan_footprint")
    return n.value


def stream_footprint(channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, n_dm, chunk_len,
                     dtype="f32") -> int:
    """Device bytes a stream of this geometry holds (dd_stream_footprint; host only)."""
    n = ctypes.c_int64()
    check(load().dd_stream_footprint(channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, n_dm,
                                     int(chunk_len), _DTYPES[dtype], ctypes.byref(n)), "dd_stream_footprint")
    return n.value


def _rows(t, name, dtype, device):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name} must be on {device}, got {t.device}")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be 2-D with unit inner stride")
    return t.stride(0)


class Plan:
    """A dedispersion plan: geometry + delay table (Eq. 1) + kernel choice.

    ``dtype`` is 'f32' (float32 in/out, optional weights) or 'u8' (uint8 in,
    int32 out, unit weights).
    """

    def __init__(self, channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, n_dm, n_out,
                 dtype: str = "f32", dm_index0: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        check(lib.dd_plan_dm_range(ctypes.byref(h), channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step,
                                   dm_index0, n_dm, n_out, _DTYPES[dtype]), "dd_plan_dm_range")
        self._h = h
        self.channels, self.n_dm, self.n_out, self.dtype = channels, n_dm, n_out, dtype
        self.dm_index0 = dm_index0
        self.geometry = (channels, f_low_mhz, chan_bw_mhz, t_samp_s, dm_first, dm_step, n_dm, n_out)
        n_in, md, db = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        check(lib.dd_plan_info(h, ctypes.byref(n_in), ctypes.byref(md), ctypes.byref(db)), "dd_plan_info")
        self.n_in, self.max_delay, self.device_bytes = n_in.value, md.value, db.value
        import torch
        self.device = torch.device("cuda", torch.cuda.current_device())

    @classmethod
    def from_setup(cls, setup, dtype="f32"):
        return cls(*setup.plan_args(), dtype=dtype)

    @classmethod
    def dm_range(cls, setup, i0, i1, dtype="f32"):
        """The plan of trials [i0, i1) of the setup's DM grid: its outputs are
        rows i0 .. i1 - 1 of the full plan's, bit for bit (dd_plan_dm_range)."""
        args = list(setup.plan_args())
        args[6] = i1 - i0  # n_dm
        return cls(*args, dtype=dtype, dm_index0=i0)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dd_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def in_dtype(self):
        import torch
        return torch.uint8 if self.dtype == "u8" else torch.float32

    @property
    def out_dtype(self):
        import torch
        return torch.int32 if self.dtype == "u8" else torch.float32

    def delays(self) -> np.ndarray:
        d = np.empty((self.n_dm, self.channels), dtype=np.int32)
        check(load().dd_plan_delays(self._h, d.ctypes.data_as(ctypes.c_void_p)), "dd_plan_delays")
        return d

    def configs(self):
        lib = load()
        n = ctypes.c_int32()
        check(lib.dd_plan_num_configs(self._h, ctypes.byref(n)), "dd_plan_num_configs")
        return [lib.dd_plan_config_name(self._h, k).decode() for k in range(n.value)]

    def select(self, cfg):
        k = self.configs().index(cfg) if isinstance(cfg, str) else int(cfg)
        check(load().dd_plan_select_config(self._h, k), "dd_plan_select_config")

    @property
    def selected(self) -> str:
        k = ctypes.c_int32()
        check(load().dd_plan_selected_config(self._h, ctypes.byref(k)), "dd_plan_selected_config")
        return self.configs()[k.value]

    def device_status(self) -> int:
        code = ctypes.c_int32()
        st = load().dd_plan_device_status(self._h, ctypes.byref(code))
        if st not in (0, 8):
            check(st, "dd_plan_device_status")
        return code.value

    def check_wait_timeout(self, limit_cycles=2_000_000, stream=None):
        """dd_check_wait_timeout: make a bounded wait expire on the GPU (read the result with device_status)."""
        check(load().dd_check_wait_timeout(self._h, int(limit_cycles), _stream_handle(stream)),
              "dd_check_wait_timeout")

    def alloc_input(self, row_stride=None):
        import torch
        stride = row_stride or self.padded_in_stride()
        return torch.zeros((self.channels, stride), dtype=self.in_dtype, device=self.device)

    def padded_in_stride(self) -> int:
        """Row stride (elements) that every kernel of the plan takes at full speed (dd_plan_in_stride)."""
        n = ctypes.c_int64()
        check(load().dd_plan_in_stride(self._h, ctypes.byref(n)), "dd_plan_in_stride")
        return n.value

    def forward(self, x, w=None, out=None, stream=None):
        """out[i][t] = sum_c w[c] x[c][t + delay(c, i)] on the GPU (Algorithm 1)."""
        import torch
        in_stride = _rows(x, "x", self.in_dtype, self.device)
        if out is None:
            out = torch.empty((self.n_dm, self.n_out), dtype=self.out_dtype, device=self.device)
        out_stride = _rows(out, "out", self.out_dtype, self.device)
        wp = None
        if w is not None:
            if w.dtype != torch.float32 or w.device != self.device or not w.is_contiguous():
                raise ValueError("w must be a contiguous float32 tensor on the plan's device")
            wp = w.data_ptr()
        check(load().dd_forward(self._h, x.data_ptr(), in_stride, wp, out.data_ptr(), out_stride,
                                _stream_handle(stream)), "dd_forward")
        return out

    def forward_host(self, x, w=None, out=None, stream=None):
        """dd_forward_host: host input/weights in, host output back (copies inside the call)."""
        import torch
        if x.device.type != "cpu" or out is not None and out.device.type != "cpu":
            raise ValueError("forward_host takes host tensors")
        in_stride = _rows(x, "x", self.in_dtype, torch.device("cpu"))
        if out is None:
            out = torch.empty((self.n_dm, self.n_out), dtype=self.out_dtype, pin_memory=True)
        out_stride = _rows(out, "out", self.out_dtype, torch.device("cpu"))
        wp = None if w is None else w.data_ptr()
        check(load().dd_forward_host(self._h, x.data_ptr(), in_stride, wp, out.data_ptr(), out_stride,
                                     _stream_handle(stream)), "dd_forward_host")
        return out

    def adjoint(self, grad_out, w=None, x=None, grad_in=True, grad_w=False, stream=None, grad_in_out=None):
        """Transpose of the weighted forward (grad_in) and d/dw (grad_w); returns (grad_in, grad_w).

        grad_in_out, if given, is a [C][>= n_in] float32 tensor that receives grad_in
        (only its first n_in columns are written)."""
        import torch
        go_stride = _rows(grad_out, "grad_out", torch.float32, self.device)
        gi = gw = None
        gi_stride = 0
        if grad_in:
            gi = grad_in_out if grad_in_out is not None else \
                torch.empty((self.channels, self.n_in), dtype=torch.float32, device=self.device)
            gi_stride = _rows(gi, "grad_in", torch.float32, self.device)
        in_stride = 0
        if grad_w:
            if x is None:
                raise ValueError("grad_w needs the forward input x")
            in_stride = _rows(x, "x", torch.float32, self.device)
            gw = torch.empty((self.channels,), dtype=torch.float32, device=self.device)
        wp = None if w is None else w.data_ptr()
        check(load().dd_adjoint(self._h, grad_out.data_ptr(), go_stride, wp,
                                None if gi is None else gi.data_ptr(), gi_stride,
                                None if x is None else x.data_ptr(), in_stride,
                                None if gw is None else gw.data_ptr(), _stream_handle(stream)), "dd_adjoint")
        return gi, gw

    def tune(self, budget_s=0.0, db_path=None):
        ms = ctypes.c_double()
        check(load().dd_tune(self._h, float(budget_s), None if db_path is None else db_path.encode(),
                             ctypes.byref(ms)), "dd_tune")
        return self.selected, ms.value


SNR_FIELDS = ("loss", "snr", "mean", "std", "best_t", "best_row", "valid")


def boxcar_snr(x, grad=False, stream=None):
    """dd_boxcar_snr: 8-sample boxcar S/N over each row of x ([rows][>= cols] float32 CUDA).

    Returns (result, grad_tensor | None, raw) where `result` is a dict read back
    from the device (synchronises the stream) and `raw` the 48-byte device
    buffer (raw.view(torch.float64)[0] is the loss, still on the device)."""
    import torch
    stride = _rows(x, "x", torch.float32, x.device)
    n_rows, n_cols = x.shape
    raw = torch.zeros(48, dtype=torch.uint8, device=x.device)
    g = torch.empty_like(x) if grad else None
    check(load().dd_boxcar_snr(x.data_ptr(), stride, n_rows, n_cols, raw.data_ptr(),
                               None if g is None else g.data_ptr(), 0 if g is None else g.stride(0),
                               _stream_handle(stream)), "dd_boxcar_snr")
    return raw, g


def snr_result(raw) -> dict:
    import struct
    b = bytes(raw.cpu().numpy().tobytes())
    vals = struct.unpack("<4dqii", b)
    return dict(zip(SNR_FIELDS, vals))


class Batch:
    """dd_batch_*: several beams' forward passes in one persistent launch (CUDA graph)."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        check(load().dd_batch_create(ctypes.byref(h), arr, len(self.plans)), "dd_batch_create")
        self._h = h

    def run(self, ins, outs, stream=None):
        n = len(self.plans)
        if len(ins) != n or len(outs) != n:
            raise ValueError("one input and one output per beam")
        for p, x, o in zip(self.plans, ins, outs):
            _rows(x, "input", p.in_dtype, p.device)
            _rows(o, "output", p.out_dtype, p.device)
        vp = ctypes.c_void_p
        i_arr = (vp * n)(*[x.data_ptr() for x in ins])
        o_arr = (vp * n)(*[o.data_ptr() for o in outs])
        is_arr = (ctypes.c_int64 * n)(*[x.stride(0) for x in ins])
        os_arr = (ctypes.c_int64 * n)(*[o.stride(0) for o in outs])
        check(load().dd_batch_run(self._h, i_arr, is_arr, o_arr, os_arr, _stream_handle(stream)), "dd_batch_run")
        return outs

    def tune(self, budget_s: float = 0.0, db_path: str | None = None) -> int:
        """dd_batch_tune: tune each distinct setup once; returns the number of setups tuned."""
        n = ctypes.c_int32()
        check(load().dd_batch_tune(self._h, float(budget_s), db_path.encode() if db_path else None,
                                   ctypes.byref(n)), "dd_batch_tune")
        return n.value

    def set_persistent(self, mode: int = 1):
        """dd_batch_set_persistent: 0 (or False) one launch per beam; 1 (or True, the
        default) persistent launches where dd_batch_tune measured them faster; 2 a
        persistent launch for every group that can have one."""
        mode = int(mode)
        check(load().dd_batch_set_persistent(self._h, mode), "dd_batch_set_persistent")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dd_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stream:
    """dd_stream_*: chunked real-time dedispersion with the overlap tail kept on the device."""

    def __init__(self, plan, chunk_len):
        self.plan = plan
        self.chunk_len = int(chunk_len)
        h = ctypes.c_void_p()
        check(load().dd_stream_create(ctypes.byref(h), plan.handle, self.chunk_len), "dd_stream_create")
        self._h = h

    def push(self, chunk, out=None, stream=None):
        """Dedisperse the next chunk ([C][chunk_len], contiguous); returns (out, t0)."""
        import torch
        p = self.plan
        if chunk.dtype != p.in_dtype or chunk.device != p.device or not chunk.is_contiguous() or \
                tuple(chunk.shape) != (p.channels, self.chunk_len):
            raise ValueError("chunk must be a contiguous [channels][chunk_len] tensor of the plan's type")
        if out is None:
            out = torch.empty((p.n_dm, self.chunk_len), dtype=p.out_dtype, device=p.device)
        if not out.is_contiguous() or tuple(out.shape) != (p.n_dm, self.chunk_len):
            raise ValueError("out must be a contiguous [n_dm][chunk_len] tensor")
        t0 = ctypes.c_int64()
        check(load().dd_stream_push(self._h, chunk.data_ptr(), out.data_ptr(), ctypes.byref(t0),
                                    _stream_handle(stream)), "dd_stream_push")
        return out, t0.value

    def reset(self, stream=None):
        check(load().dd_stream_reset(self._h, _stream_handle(stream)), "dd_stream_reset")

    def state_bytes(self) -> int:
        n = ctypes.c_int64()
        check(load().dd_stream_state_bytes(self._h, ctypes.byref(n)), "dd_stream_state_bytes")
        return n.value

    def device_bytes(self) -> int:
        """Device memory the stream holds (its plan's tables and two state buffers)."""
        n = ctypes.c_int64()
        check(load().dd_stream_device_bytes(self._h, ctypes.byref(n)), "dd_stream_device_bytes")
        return n.value

    def save(self, stream=None) -> bytes:
        buf = ctypes.create_string_buffer(self.state_bytes())
        check(load().dd_stream_save(self._h, buf, _stream_handle(stream)), "dd_stream_save")
        return buf.raw

    def restore(self, state: bytes, stream=None):
        buf = ctypes.create_string_buffer(state, len(state))
        check(load().dd_stream_restore(self._h, buf, _stream_handle(stream)), "dd_stream_restore")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dd_stream_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
