"""dd_boxcar_snr_noalloc: the allocation-free form of the S/N loss.

Callers that cannot allocate device memory while running (a real-time
pipeline whose memory was all reserved at start-up, or a host framework that
owns every allocation) use this entry point; it must give the same answers as
dd_boxcar_snr.  The file is named so that pytest collects it last.  It calls
the C ABI directly and works in a fresh process as well as after the other
tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_ROWS = 65536  # DD_NOALLOC_MAX_ROWS in include/dd.h


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_01165_gb300 import binding
    lib = binding.load()
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    for name in ("dd_boxcar_snr", "dd_boxcar_snr_noalloc"):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        fn.argtypes = [vp, i64, i32, i64, vp, vp, i64, vp]
    return lib


def _block(seed, rows, cols):
    g = torch.Generator(device="cpu").manual_seed(seed)
    x = torch.randn((rows, cols), generator=g)
    x[rows // 3, cols // 2: cols // 2 + 5] += 6.0          # a clear maximum
    return x.cuda()


def _call(lib, name, x):
    res = torch.zeros(48, dtype=torch.uint8, device="cuda")
    grad = torch.empty_like(x)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, name)(x.data_ptr(), x.stride(0), x.shape[0], x.shape[1], res.data_ptr(),
                            grad.data_ptr(), grad.stride(0), stream)
    assert rc == 0, (name, rc, lib.dd_last_error())
    torch.cuda.synchronize()
    return res.cpu(), grad.cpu()


def _fields(raw):
    import struct
    return struct.unpack("<4dqii", bytes(raw.numpy().tobytes()))


def test_noalloc_matches_allocating_entry_point_twice(lib):
    # two calls in a row on different blocks: the shared scratch must not leak
    # state from one call into the next
    for seed, (rows, cols) in ((1, (300, 2000)), (2, (517, 1333))):
        x = _block(seed, rows, cols)
        ref_raw, ref_grad = _call(lib, "dd_boxcar_snr", x)
        got_raw, got_grad = _call(lib, "dd_boxcar_snr_noalloc", x)
        ref, got = _fields(ref_raw), _fields(got_raw)
        assert got[4:] == ref[4:]                                  # best_t, best_row, valid
        np.testing.assert_allclose(got[:4], ref[:4], rtol=1e-12, atol=0)
        np.testing.assert_allclose(got_grad.numpy(), ref_grad.numpy(), rtol=1e-6, atol=1e-9)
        assert got[6] == 1 and got[5] == rows // 3


def test_noalloc_accepts_the_maximum_row_count(lib):
    # exactly DD_NOALLOC_MAX_ROWS rows fill the whole fixed scratch; the
    # maximum sits in the last row, whose scratch entry is the array's last.
    # S/N is measured against each row's own spread, which a pulse widens, so
    # the pulse must be a small part of its row to stand out: with 512 columns
    # its S/N (about 9) is far above the best noise row's (about 5)
    g = torch.Generator(device="cpu").manual_seed(3)
    x = torch.randn((MAX_ROWS, 512), generator=g)
    x[MAX_ROWS - 1, 200:208] += 9.0
    x = x.cuda()
    ref_raw, ref_grad = _call(lib, "dd_boxcar_snr", x)
    got_raw, got_grad = _call(lib, "dd_boxcar_snr_noalloc", x)
    ref, got = _fields(ref_raw), _fields(got_raw)
    assert got[4:] == ref[4:] and got[5] == MAX_ROWS - 1 and got[6] == 1
    np.testing.assert_allclose(got[:4], ref[:4], rtol=1e-12, atol=0)
    np.testing.assert_allclose(got_grad.numpy(), ref_grad.numpy(), rtol=1e-6, atol=1e-9)


def test_noalloc_rejects_too_many_rows(lib):
    x = torch.zeros((1, 16), device="cuda")
    res = torch.zeros(48, dtype=torch.uint8, device="cuda")
    rc = lib.dd_boxcar_snr_noalloc(x.data_ptr(), 16, MAX_ROWS + 1, 16, res.data_ptr(), None, 0, None)
    assert rc == 2  # DD_ERR_SHAPE, rejected before any GPU work
