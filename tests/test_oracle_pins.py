"""Pins for the oracle: checks against what the paper and the mathematics fix.

None of these tests re-derives an oracle result by calling the oracle's own
code path twice.  They compare it with: a textbook value of the dispersion
delay, exact rational arithmetic, invariants of Eq. 1, the zero-DM special
case of Section 4.3 (every DM trial 0 gives the plain channel sum), impulse
responses, literal pure-Python loops on tiny inputs, linearity, explicit
matrices, closed-form loss values and finite differences.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1601_01165_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                parts = line.split()
                vals[parts[0]] = float(parts[1])
    return vals


def _exact_delay(s, i, c):
    """Eq. 1 in exact rational arithmetic on the double-valued parameters."""
    f = Fraction(s.f_low_mhz + c * s.chan_bw_mhz)
    fh = Fraction(s.f_low_mhz + (s.channels - 1) * s.chan_bw_mhz)
    dm = Fraction(s.dm_first + i * s.dm_step)
    return 4150 * dm * (1 / (f * f) - 1 / (fh * fh)) / Fraction(s.t_samp_s)


def _round_half_up(x: Fraction) -> int:
    return math.floor(x + Fraction(1, 2))


# ----------------------------------------------------------------- delay table

def test_delay_textbook_units(oracle):
    # Lorimer & Kramer: a unit DM delays 1 GHz by about 4.15 ms relative to
    # infinite frequency; Eq. 1 with the paper's 4150 s MHz^2 gives exactly that.
    # Top channel at 1e7 MHz stands in for infinite frequency.
    d = oracle.delay_table(2, 1000.0, 1.0e7, 1e-6, 0.0, 1.0, 3)
    assert d[:, 1].tolist() == [0, 0, 0]              # top channel is the reference
    assert d[:, 0].tolist() == [0, 4150, 8300]        # 4.15 ms per unit DM at 1 us sampling
    d = oracle.delay_table(2, 1000.0, 1.0e7, 1e-4, 2.5, 1.0, 1)
    assert d[0, 0] == 104                             # 2.5 * 4.15 ms / 0.1 ms = 103.75 -> 104
    d = oracle.delay_table(2, 2000.0, 1.0e7, 1e-7, 1.0, 1.0, 1)
    assert d[0, 0] == 10375                           # f^-2 law: doubling f quarters the delay


@pytest.mark.parametrize("setup,stride", [(synth.TINY, 1), (synth.APERTIF, 97), (synth.LOFAR, 211)])
def test_delay_exact_rational(oracle, setup, stride):
    d = oracle.delay_table(setup.channels, setup.f_low_mhz, setup.chan_bw_mhz, setup.t_samp_s,
                           setup.dm_first, setup.dm_step, setup.n_dm)
    rows = sorted(set(range(0, setup.n_dm, stride)) | {setup.n_dm - 1})
    cols = sorted(set(range(0, setup.channels, max(1, setup.channels // 64))) | {0, setup.channels - 1})
    for i in rows:
        for c in cols:
            x = _exact_delay(setup, i, c)
            assert d[i, c] == _round_half_up(x), (i, c, float(x))


@pytest.mark.parametrize("setup", [synth.TINY, synth.APERTIF, synth.LOFAR])
def test_delay_invariants_and_max(oracle, setup):
    d = oracle.delay_table(setup.channels, setup.f_low_mhz, setup.chan_bw_mhz, setup.t_samp_s,
                           setup.dm_first, setup.dm_step, setup.n_dm)
    assert d.shape == (setup.n_dm, setup.channels)
    assert (d[:, -1] == 0).all()                     # f_h has no delay
    assert (d[0] == 0).all()                         # DM trial 0 is 0 pc/cm^3
    assert (np.diff(d, axis=1) <= 0).all()           # lower frequency arrives later
    assert (np.diff(d, axis=0) >= 0).all()           # larger DM delays more
    md = oracle.max_delay(d)
    assert md == d[-1, 0]
    assert md == _round_half_up(_exact_delay(setup, setup.n_dm - 1, 0))
    # linear in DM up to rounding (Eq. 1): d(2i) within 1 of 2 d(i)
    half = setup.n_dm // 2
    assert np.abs(d[2 * np.arange(half)].astype(np.int64) - 2 * d[:half].astype(np.int64)).max() <= 1


def test_delay_max_values(oracle):
    # Maximum delays of the three setups, by exact arithmetic at (last DM, channel 0).
    for s, want in ((synth.TINY, 6), (synth.APERTIF, 6702), (synth.LOFAR, 146874)):
        assert _round_half_up(_exact_delay(s, s.n_dm - 1, 0)) == want
        d = oracle.delay_table(*s.plan_args()[:7])
        assert oracle.max_delay(d) == want


def test_delay_rejects_bad_args(oracle):
    with pytest.raises(oracle.OracleError):
        oracle.delay_table(0, 1400.0, 1.0, 1e-3, 0.0, 1.0, 4)
    with pytest.raises(oracle.OracleError):
        oracle.delay_table(4, -1.0, 1.0, 1e-3, 0.0, 1.0, 4)
    with pytest.raises(oracle.OracleError):
        oracle.delay_table(4, 1400.0, 1.0, 0.0, 0.0, 1.0, 4)


# --------------------------------------------------------------------- forward

def _small_setup(C=7, n_dm=5, n_out=23, dm_step=3.0):
    return synth.Setup("small", C, 400.0, 8.0, 1e-3, 0.0, dm_step, n_dm, n_out)


def test_forward_zero_dm_is_channel_sum(oracle):
    # Section 4.3: with every DM trial 0 the delays vanish and each output row
    # is the plain sum over channels.
    s = synth.APERTIF.replace(n_dm=6, n_out=300, dm_step=0.0)
    d = oracle.delay_table(*s.plan_args()[:7])
    assert (d == 0).all()
    x = synth.noise_f32(3, s.channels, s.n_out)
    out = oracle.forward_f32(d, x, s.n_out)
    want = x.astype(np.float64).sum(axis=0)
    for i in range(s.n_dm):
        np.testing.assert_allclose(out[i], want, rtol=1e-12, atol=1e-9)
    xu = synth.noise_u8(4, s.channels, s.n_out)
    outu = oracle.forward_u8(d, xu, s.n_out)
    wantu = xu.astype(np.int64).sum(axis=0)
    assert (outu == wantu[None, :]).all()


@pytest.mark.parametrize("c0,u0", [(0, 40), (3, 17), (6, 5)])
def test_forward_impulse_response(oracle, c0, u0):
    # A single unit sample at (c0, u0) reaches out[i][t] exactly when
    # t + delay(c0, i) == u0: fixes the direction of the shift and the roles of
    # the channel and DM indices in Algorithm 1.
    s = _small_setup()
    d = oracle.delay_table(*s.plan_args()[:7])
    n_in = s.n_out + oracle.max_delay(d)
    x = np.zeros((s.channels, n_in), dtype=np.float32)
    x[c0, u0] = 1.0
    out = oracle.forward_f32(d, x, s.n_out)
    want = np.zeros_like(out)
    for i in range(s.n_dm):
        t = u0 - d[i, c0]
        if 0 <= t < s.n_out:
            want[i, t] = 1.0
    assert (out == want).all()
    xu = np.zeros_like(x, dtype=np.uint8)
    xu[c0, u0] = 1
    assert (oracle.forward_u8(d, xu, s.n_out) == want.astype(np.int32)).all()


def test_forward_matches_python_loops(oracle):
    s = _small_setup(C=5, n_dm=4, n_out=13)
    d = oracle.delay_table(*s.plan_args()[:7])
    bd = oracle.brute_delay(*s.plan_args()[:7])
    assert (d == bd).all()
    n_in = s.n_out + int(d.max())
    x = synth.noise_f32(11, s.channels, n_in)
    w = synth.weights(5, s.channels)
    np.testing.assert_allclose(oracle.forward_f32(d, x, s.n_out, w), oracle.brute_forward(d, x, s.n_out, w),
                               rtol=1e-13, atol=1e-12)
    xu = synth.noise_u8(12, s.channels, n_in)
    assert (oracle.forward_u8(d, xu, s.n_out) == oracle.brute_forward(d, xu, s.n_out)).all()


def test_forward_linearity(oracle):
    s = _small_setup(C=9, n_dm=6, n_out=50)
    d = oracle.delay_table(*s.plan_args()[:7])
    n_in = s.n_out + int(d.max())
    # integer-valued samples and dyadic coefficients keep a*x + b*y exact in float32
    x = np.rint(8 * synth.noise_f32(1, s.channels, n_in))
    y = np.rint(8 * synth.noise_f32(2, s.channels, n_in))
    a, b = 0.75, -2.5
    lhs = oracle.forward_f32(d, (a * x + b * y).astype(np.float32), s.n_out)
    rhs = a * oracle.forward_f32(d, x, s.n_out) + b * oracle.forward_f32(d, y, s.n_out)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-10)
    xu = (synth.noise_u8(3, s.channels, n_in) // 2).astype(np.uint8)
    yu = (synth.noise_u8(4, s.channels, n_in) // 2).astype(np.uint8)
    su = (xu.astype(np.int32) + yu).astype(np.uint8)
    assert (oracle.forward_u8(d, su, s.n_out).astype(np.int64) ==
            oracle.forward_u8(d, xu, s.n_out).astype(np.int64) + oracle.forward_u8(d, yu, s.n_out)).all()


def test_forward_weights_scale_channels(oracle):
    # Weights multiply each channel's contribution: w = e_c isolates channel c.
    s = _small_setup(C=6, n_dm=3, n_out=20)
    d = oracle.delay_table(*s.plan_args()[:7])
    n_in = s.n_out + int(d.max())
    x = synth.noise_f32(8, s.channels, n_in)
    total = np.zeros((s.n_dm, s.n_out))
    for c in range(s.channels):
        e = np.zeros(s.channels, dtype=np.float32)
        e[c] = 2.0
        part = oracle.forward_f32(d, x, s.n_out, e)
        for i in range(s.n_dm):
            np.testing.assert_array_equal(part[i], 2.0 * x[c, d[i, c]:d[i, c] + s.n_out].astype(np.float64))
        total += part
    np.testing.assert_allclose(total, 2.0 * oracle.forward_f32(d, x, s.n_out), rtol=1e-12, atol=1e-10)


def _physical_arrival(s, dm):
    # arrival sample offset of a pulse of DM `dm` in each channel, from Eq. 1
    fh = s.f_low_mhz + (s.channels - 1) * s.chan_bw_mhz
    f = s.f_low_mhz + np.arange(s.channels) * s.chan_bw_mhz
    return np.floor(4150.0 * dm * (1.0 / f ** 2 - 1.0 / fh ** 2) / s.t_samp_s + 0.5).astype(np.int64)


def test_forward_tiny_pulse(oracle):
    s = synth.TINY
    d = oracle.delay_table(*s.plan_args()[:7])
    n_in = s.n_out + oracle.max_delay(d)
    arrival = _physical_arrival(s, 12.0)
    # width 1: unique maximum 5 * 64 at (DM 12, t 400)
    x = np.zeros((s.channels, n_in), dtype=np.float32)
    synth.inject_pulse(x, arrival, 400, 1, 5.0)
    out = oracle.forward_f32(d, x, s.n_out)
    assert out[12, 400] == 5.0 * 64
    assert (out == out.max()).sum() == 1 and np.unravel_index(out.argmax(), out.shape) == (12, 400)
    # width 3: value 320 at (12, 400..402); (12, 400) is among the maxima
    x = np.zeros((s.channels, n_in), dtype=np.float32)
    synth.inject_pulse(x, arrival, 400, 3, 5.0)
    out = oracle.forward_f32(d, x, s.n_out)
    assert out[12, 400:403].tolist() == [320.0] * 3 and out.max() == 320.0
    # the configured noisy input still peaks on the pulse's DM sweep plateau
    xn = synth.noise_f32(0, s.channels, n_in)
    synth.inject_pulse(xn, arrival, 400, 3, 5.0)
    outn = oracle.forward_f32(d, xn, s.n_out)
    i, t = np.unravel_index(outn.argmax(), outn.shape)
    assert 400 - 2 <= t <= 402 + 2


@pytest.mark.parametrize("setup,dtype", [(synth.APERTIF, "f32"), (synth.APERTIF, "u8"), (synth.LOFAR, "f32")])
def test_forward_pulse_peaks_at_true_dm(oracle, setup, dtype):
    # A dispersed pulse injected into noise peaks at its DM trial and time.
    # Computed on a window of DM trials and samples around each pulse.
    s = setup
    d = oracle.delay_table(*s.plan_args()[:7])
    n_in = s.n_out + oracle.max_delay(d)
    sites = synth.pulse_sites(0, s.n_dm, s.n_out, 3 if s is synth.APERTIF else 2)
    if dtype == "u8":
        x = synth.noise_u8(0, s.channels, n_in)
        amp = 40.0
    else:
        x = synth.noise_f32(0, s.channels, n_in)
        amp = 5.0
    for i_p, t_p in sites:
        synth.inject_pulse(x, _physical_arrival(s, s.dm_first + i_p * s.dm_step), t_p, 3, amp)
    for i_p, t_p in sites:
        i0, i1 = max(0, i_p - 12), min(s.n_dm, i_p + 13)
        t0 = max(0, t_p - 40)
        n_w = min(s.n_out, t_p + 43) - t0
        sub = d[i0:i1]
        xw = np.ascontiguousarray(x[:, t0:t0 + n_w + int(sub.max())])
        if dtype == "u8":
            out = oracle.forward_u8(sub, xw, n_w).astype(np.float64)
            out -= 128.0 * s.channels
        else:
            out = oracle.forward_f32(sub, xw, n_w)
        i, t = np.unravel_index(out.argmax(), out.shape)
        assert i0 + i == i_p, (i_p, t_p, i0 + i, t0 + t)
        assert t_p <= t0 + t <= t_p + 2


def test_forward_rejects_short_input(oracle):
    s = _small_setup()
    d = oracle.delay_table(*s.plan_args()[:7])
    x = np.zeros((s.channels, s.n_out + int(d.max()) - 1), dtype=np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.forward_f32(d, x, s.n_out)


def test_table2_counts():
    # Section 3 / Table 2 / Section 2.1 / Section 5.1 figures from the setup dimensions.
    g = _golden("table2_counts.txt")
    ap, lo = synth.APERTIF, synth.LOFAR
    assert abs(ap.channels * ap.n_out / 1e6 - g["apertif_mflop_per_dm"]) <= 0.5
    assert abs(lo.channels * lo.n_out / 1e6 - g["lofar_mflop_per_dm"]) <= 0.5
    assert abs(450 * ap.channels * ap.n_out * 4 / 1e9 - g["apertif_input_gbs_450"]) <= 1.0
    assert abs(450 * 2000 * ap.n_out * 4 / 1e9 - g["apertif_output_gbs_450"]) <= 0.5
    assert abs(450 * 2000 * ap.channels * ap.n_out / 1e12 - g["apertif_tflops_450x2000"]) <= 0.1
    assert math.floor(1.0 / g["hd7970_seconds_2000dm"]) == g["hd7970_beams_2x_memory"]


# -------------------------------------------------------------- adjoint, wgrad

def _dense_matrix(d, n_out, n_in, w):
    n_dm, C = d.shape
    A = np.zeros((n_dm * n_out, C * n_in))
    for i in range(n_dm):
        for t in range(n_out):
            for c in range(C):
                A[i * n_out + t, c * n_in + t + d[i, c]] += w[c]
    return A


def test_adjoint_is_transpose(oracle):
    s = _small_setup(C=4, n_dm=3, n_out=11)
    d = oracle.delay_table(*s.plan_args()[:7])
    n_in = s.n_out + int(d.max())
    w = synth.weights(3, s.channels)
    A = _dense_matrix(d, s.n_out, n_in, w)
    x = synth.noise_f32(5, s.channels, n_in)
    np.testing.assert_allclose(oracle.forward_f32(d, x, s.n_out, w).ravel(), A @ x.ravel().astype(np.float64),
                               rtol=1e-12, atol=1e-12)
    g = synth.noise_f32(6, s.n_dm, s.n_out)
    np.testing.assert_allclose(oracle.adjoint_f32(d, g, n_in, w).ravel(), A.T @ g.ravel().astype(np.float64),
                               rtol=1e-12, atol=1e-12)


def test_adjoint_dot_product(oracle):
    s = synth.TINY
    d = oracle.delay_table(*s.plan_args()[:7])
    n_in = s.n_out + oracle.max_delay(d)
    w = synth.weights(1, s.channels)
    x = synth.noise_f32(2, s.channels, n_in)
    y = synth.noise_f32(3, s.n_dm, s.n_out)
    lhs = float((oracle.forward_f32(d, x, s.n_out, w) * y.astype(np.float64)).sum())
    rhs = float((x.astype(np.float64) * oracle.adjoint_f32(d, y, n_in, w)).sum())
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs) + 1.0)


def test_wgrad_is_channelwise_contraction(oracle):
    s = _small_setup(C=6, n_dm=4, n_out=30)
    d = oracle.delay_table(*s.plan_args()[:7])
    n_in = s.n_out + int(d.max())
    x = synth.noise_f32(9, s.channels, n_in)
    g = synth.noise_f32(10, s.n_dm, s.n_out)
    gw = oracle.wgrad_f32(d, g, x)
    for c in range(s.channels):
        e = np.zeros(s.channels, dtype=np.float32)
        e[c] = 1.0
        want = float((oracle.forward_f32(d, x, s.n_out, e) * g.astype(np.float64)).sum())
        assert abs(gw[c] - want) <= 1e-12 * (1 + abs(want))


# ------------------------------------------------------------------------ loss

def test_loss_closed_form():
    import oracle as orc
    g = _golden("loss_spike.txt")
    n = int(g["n_out"])
    out = np.zeros((3, n))
    out[1, int(g["spike_t"])] = 1.0
    out[0] = 0.0          # constant rows have no S/N and are skipped
    out[2, :] = 7.0
    loss, grad, (bi, bt) = orc.boxcar_snr_loss(out)
    assert abs(loss - g["loss"]) < 1e-15
    assert (bi, bt) == (1, int(g["best_t"]))
    assert abs(loss + 2.0 / math.sqrt(5.0)) < 1e-15


def test_loss_invariances_and_gradient():
    import oracle as orc
    rng = np.random.default_rng(0)
    out = rng.standard_normal((4, 40))
    loss, grad, best = orc.boxcar_snr_loss(out)
    # S/N is invariant to a per-row offset and a positive per-row scale
    shifted = out * np.array([[2.0], [0.5], [3.0], [1.5]]) + np.array([[1.0], [-4.0], [0.25], [9.0]])
    loss2, _, best2 = orc.boxcar_snr_loss(shifted, want_grad=False)
    assert abs(loss - loss2) < 1e-12 and best == best2
    # central finite differences
    h = 1e-6
    for (i, t) in [(best[0], best[1]), (best[0], best[1] + 3), (best[0], 39), ((best[0] + 1) % 4, 5)]:
        p = out.copy()
        p[i, t] += h
        m = out.copy()
        m[i, t] -= h
        fd = (orc.boxcar_snr_loss(p, False)[0] - orc.boxcar_snr_loss(m, False)[0]) / (2 * h)
        assert abs(fd - grad[i, t]) < 1e-6, (i, t, fd, grad[i, t])


def test_parallel_cpu_baseline_matches_oracle_bit_for_bit():
    """The multi-threaded CPU baseline sums the same fp64 terms in the same
    channel order as the oracle, for any thread count and block sizes."""
    import oracle
    from paper_1601_01165_gb300 import synth
    s = synth.Setup("cpb", 48, 1420.0, 6.25, 50e-6, 0.0, 0.5, 23, 3001)
    d = oracle.delay_table(*s.plan_args()[:7])
    x = synth.noise_f32(4, s.channels, s.n_out + int(d.max()) + 5)
    w = synth.weights(4, s.channels)
    ref = oracle.forward_f32(d, x, s.n_out, w)
    for threads, dm_chunk, t_block in [(0, 1, 64), (1, 4, 2048), (3, 5, 1000), (0, 23, 3001)]:
        got = oracle.forward_f32_parallel(d, x, s.n_out, w, threads, dm_chunk, t_block)
        assert (got == ref).all(), (threads, dm_chunk, t_block)
    assert (oracle.forward_f32_parallel(d, x, s.n_out) == oracle.forward_f32(d, x, s.n_out)).all()
    with pytest.raises(oracle.OracleError):
        oracle.forward_f32_parallel(d, x[:, :s.n_out], s.n_out)     # input too short for the delays


def test_oracle_adjoint_and_weight_gradient_pass_gradcheck():
    """torch.autograd.gradcheck on the oracle path (CPU, fp64 outputs): the
    oracle's transpose and weight gradient are the derivatives of its forward
    sum (the sum is bilinear in (input, weights), so central differences are
    exact up to the float32 rounding of the perturbed inputs)."""
    torch = pytest.importorskip("torch")
    import oracle
    s = synth.Setup("gc", 5, 400.0, 8.0, 1e-3, 0.0, 3.0, 4, 9)
    d = oracle.delay_table(*s.plan_args()[:7])
    n_in = s.n_out + int(d.max())

    class OracleDD(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, w):
            ctx.save_for_backward(x, w)
            return torch.from_numpy(oracle.forward_f32(d, x.numpy(), s.n_out, w.numpy()))

        @staticmethod
        def backward(ctx, g):
            x, w = ctx.saved_tensors
            gx = oracle.adjoint_f32(d, g.numpy(), n_in, w.numpy())
            gw = oracle.wgrad_f32(d, g.numpy(), x.numpy())
            return torch.from_numpy(gx), torch.from_numpy(gw)

    gen = torch.Generator().manual_seed(3)
    x = torch.randn(s.channels, n_in, dtype=torch.float64, generator=gen).float().double().requires_grad_()
    w = torch.rand(s.channels, dtype=torch.float64, generator=gen).float().double().requires_grad_()
    assert torch.autograd.gradcheck(OracleDD.apply, (x, w), eps=1e-3, atol=1e-4, rtol=1e-3)


def test_packed_uint8_decode_is_exact_within_16_bit_lanes():
    """The packed uint8 kernel keeps, per aligned word x = s0 + 2^8 s1 + 2^16 s2
    + 2^24 s3, the sum A of the words modulo 2^32 and the sum B of the odd
    bytes as two 16-bit lanes, and recovers S1, S3 = B's lanes and
    S0 + 2^16 S2 = A - 2^8 S1 - 2^24 S3 (mod 2^32).  Exact while every S_k
    < 2^16: for any 8-bit samples up to 257 channels (257 * 255 = 65535), so
    the kernel's 256-channel periods are safe; checked on random, all-255 and
    all-0 words, and shown to fail at 258 channels of 255."""
    rng = np.random.default_rng(7)

    def decode(words):
        s = np.stack([(words >> (8 * k)) & 0xFF for k in range(4)], axis=1)
        a = int(words.sum()) & 0xFFFFFFFF
        b = int((s[:, 1] | (s[:, 3] << 16)).sum()) & 0xFFFFFFFF
        s1, s3 = b & 0xFFFF, b >> 16
        s02 = (a - (s1 << 8) - (s3 << 24)) & 0xFFFFFFFF
        return [s02 & 0xFFFF, s1, s02 >> 16, s3], [int(v) for v in s.sum(axis=0)]

    for n in (1, 2, 255, 256, 257):
        for kind in ("random", "max", "zero"):
            if kind == "random":
                w = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64)
            else:
                w = np.full(n, 0xFFFFFFFF if kind == "max" else 0, dtype=np.uint64)
            got, want = decode(w)
            assert got == want, (n, kind)
    got, want = decode(np.full(258, 0xFFFFFFFF, dtype=np.uint64))
    assert got != want   # 258 * 255 >= 2^16: a 16-bit lane overflows
