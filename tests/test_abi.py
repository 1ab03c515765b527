"""C ABI checks that need no GPU: the library loads, exports every entry point
include/dd.h declares, and its host-side logic (Eq. 1 delay table, argument
validation, status names) behaves as documented."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1601_01165_gb300 import binding, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "dd.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(dd_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = binding.load()
    declared = _declared()
    assert len(declared) >= 25
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_status_names():
    lib = binding.load()
    assert b"sm_103a" in lib.dd_version()
    for code, name in binding.STATUS.items():
        assert lib.dd_status_string(code).decode() == name


@pytest.mark.parametrize("setup", [synth.TINY, synth.APERTIF, synth.LOFAR], ids=lambda s: s.name)
def test_library_delay_table_equals_oracle(oracle, setup):
    # the library's Eq. 1 code and the oracle's are written independently
    got = binding.delay_table(*setup.plan_args()[:7])
    want = oracle.delay_table(*setup.plan_args()[:7])
    assert got.dtype == np.int32 and (got == want).all()


@pytest.mark.parametrize("setup", [synth.APERTIF, synth.LOFAR], ids=lambda s: s.name)
def test_delay_table_dm_range_rows_equal_the_full_table(setup):
    """A block of trials [i0, i1) of the DM grid (the rows one GPU computes
    when a beam is split by DM trials) has exactly the full table's rows, for
    blocks on and off the kernels' trial tiles."""
    from paper_1601_01165_gb300.shard import split_dm_range
    args = list(setup.plan_args()[:7])
    full = binding.delay_table(*args)
    blocks = split_dm_range(setup.n_dm, 3, 6) + split_dm_range(setup.n_dm, 7, 1) + [(1, 2), (setup.n_dm - 1, setup.n_dm)]
    for i0, i1 in blocks:
        if i1 == i0:
            continue
        sub = binding.delay_table(*args[:6], i1 - i0, dm_index0=i0)
        assert (sub == full[i0:i1]).all(), (i0, i1)


def test_delay_table_dm_range_argument_errors():
    for i0 in (-1, 2 ** 31 - 2):
        with pytest.raises(binding.DDError) as e:
            binding.delay_table(4, 1400.0, 1.0, 1e-3, 0.0, 1.0, 4, dm_index0=i0)
        assert e.value.name == "DD_ERR_ARG"
    lib = binding.load()
    h = ctypes.c_void_p()
    assert lib.dd_plan_dm_range(ctypes.byref(h), 64, 1400.0, 1.0, 1e-3, 0.0, 1.0, -3, 32, 100, 1) == 1


def test_delay_table_argument_errors():
    for bad in [(0, 1400.0, 1.0, 1e-3, 0.0, 1.0, 4), (4, 0.0, 1.0, 1e-3, 0.0, 1.0, 4),
                (4, 1400.0, -1.0, 1e-3, 0.0, 1.0, 4), (4, 1400.0, 1.0, 0.0, 0.0, 1.0, 4),
                (4, 1400.0, 1.0, 1e-3, -1.0, 1.0, 4), (4, 1400.0, 1.0, 1e-3, 0.0, -0.5, 4),
                (4, 1400.0, 1.0, 1e-3, 0.0, 1.0, 0), (4, float("nan"), 1.0, 1e-3, 0.0, 1.0, 4)]:
        with pytest.raises(binding.DDError) as e:
            binding.delay_table(*bad)
        assert e.value.name == "DD_ERR_ARG"
        assert binding.load().dd_last_error()


def test_delay_overflow_is_an_argument_error():
    # a delay beyond int32 samples must be refused, not wrapped
    with pytest.raises(binding.DDError) as e:
        binding.delay_table(2, 1.0, 1.0e6, 1e-12, 1e6, 1.0, 2)
    assert e.value.name == "DD_ERR_ARG"


def test_plan_validation_before_device_use():
    lib = binding.load()
    h = ctypes.c_void_p()
    assert lib.dd_plan(ctypes.byref(h), 64, 1400.0, 1.0, 1e-3, 0.0, 1.0, 32, 0, 1) == 1   # n_out = 0
    assert lib.dd_plan(ctypes.byref(h), 64, 1400.0, 1.0, 1e-3, 0.0, 1.0, 32, 100, 7) == 1  # bad dtype
    assert lib.dd_plan(None, 64, 1400.0, 1.0, 1e-3, 0.0, 1.0, 32, 100, 1) == 1
    assert lib.dd_plan_destroy(None) == 0
    assert lib.dd_forward(None, None, 0, None, None, 0, None) == 1
    assert lib.dd_batch_destroy(None) == 0 and lib.dd_stream_destroy(None) == 0
