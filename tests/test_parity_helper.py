"""The whole-output parity checker used by the full-size GPU tests, checked on
the CPU: it must pass the oracle's own rounded output and catch single planted
errors (float32 and uint8), whichever row block they fall in."""
import numpy as np

import oracle
from paper_1601_01165_gb300 import synth
from helpers import FP32_REL, full_parity, oracle_table

S = synth.Setup("helper", 48, 1420.0, 2.0, 50e-6, 0.0, 0.25, 37, 700)


def _inputs(dtype):
    d = oracle_table(S)
    n_in = S.n_out + int(d.max())
    x = (synth.noise_u8 if dtype == "u8" else synth.noise_f32)(4, S.channels, n_in, n_in + 5)
    return d, x


def test_float_rounded_oracle_passes_and_planted_errors_fail():
    d, x = _inputs("f32")
    w = synth.weights(4, S.channels)
    ref = oracle.forward_f32(d, x, S.n_out, w)
    scale = oracle.forward_f32(d, np.abs(x), S.n_out, np.abs(w))
    good = ref.astype(np.float32)
    bad1 = good.copy()
    bad1[36, 699] += np.float32(3 * FP32_REL * scale[36, 699])   # last row, last sample
    bad2 = good.copy()
    bad2[0, 0] = -bad2[0, 0] if bad2[0, 0] != 0 else 1.0          # a flipped sign
    res = full_parity(d, x, "f32", {"good": good, "bad1": bad1, "bad2": bad2}, w=w, rows_per_job=5, workers=3)
    assert res["good"][0] == 0 and res["good"][1] <= 1.0
    assert res["bad1"][0] == 1 and res["bad1"][1] > 2.0
    assert res["bad2"][0] == 1


def test_uint8_bit_exact_and_planted_error_fails():
    d, x = _inputs("u8")
    ref = oracle.forward_u8(d, x, S.n_out)
    bad = ref.copy()
    bad[17, 350] += 1
    res = full_parity(d, x, "u8", {"good": ref, "bad": bad}, rows_per_job=4, workers=2)
    assert res["good"] == (0, 0.0)
    assert res["bad"][0] == 1
