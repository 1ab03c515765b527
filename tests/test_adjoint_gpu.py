"""GPU parity of the adjoint, weight gradient, S/N loss and autograd chain against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1601_01165_gb300 import synth
from helpers import FP32_REL, make_input, oracle_table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_01165_gb300 import binding
    binding.load()
    return binding


ADJ_SETUPS = [
    synth.TINY,
    synth.Setup("adj-ragged", 37, 1420.0, 8.0, 50e-6, 0.0, 0.25, 45, 1001),
    synth.Setup("adj-lofar-cut", 32, 138.0, 0.1953125, 5e-6, 0.0, 0.01, 70, 3001),
    synth.Setup("adj-apertif-cut", 1024, 1420.0, 0.29296875, 50e-6, 3.0, 0.25, 41, 1931),
]


def _tensors(plan, s, seed, weighted=True):
    d = oracle_table(s)
    x, _ = make_input(s, "f32", seed, plan.n_in)
    g = synth.noise_f32(seed + 100, s.n_dm, s.n_out)
    w = synth.weights(seed, s.channels) if weighted else None
    return d, x, g, w


@pytest.mark.parametrize("setup", ADJ_SETUPS, ids=lambda s: s.name)
def test_adjoint_and_wgrad_match_oracle(dd, setup):
    s = setup
    plan = dd.Plan.from_setup(s, "f32")
    d, x, g, w = _tensors(plan, s, 3)
    xt, gt, wt = (torch.from_numpy(a).cuda() for a in (x, g, w))
    gi, gw = plan.adjoint(gt, w=wt, x=xt, grad_in=True, grad_w=True)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    ref = oracle.adjoint_f32(d, g, plan.n_in, w)
    scale = oracle.adjoint_f32(d, np.abs(g), plan.n_in, np.abs(w))
    err = np.abs(gi.cpu().numpy().astype(np.float64) - ref)
    assert (err <= FP32_REL * scale).all(), float((err - FP32_REL * scale).max())
    refw = oracle.wgrad_f32(d, g, x)
    scalew = oracle.wgrad_f32(d, np.abs(g), np.abs(x))
    errw = np.abs(gw.cpu().numpy().astype(np.float64) - refw)
    assert (errw <= FP32_REL * scalew).all(), float((errw - FP32_REL * scalew).max())
    # grad_w alone (transpose into plan scratch) agrees bit for bit with the combined call
    _, gw2 = plan.adjoint(gt, w=wt, x=xt, grad_in=False, grad_w=True)
    assert torch.equal(gw, gw2)


@pytest.mark.parametrize("n_out", [1931, 8192], ids=["ragged", "whole-tiles"])
def test_weight_gradient_alone_on_tmw9_tiles(dd, n_out):
    """grad_w requested alone on a plan and input the 9-trial Tensor-Memory
    forward takes runs on that kernel's tiles: the products of grad_out with
    the input windows, summed per channel in a fixed order.  It matches the
    oracle, the transposed-plan path (the combined call) within the fp32 bar,
    and itself bit for bit.  NaN in the row padding past n_in must not reach
    the sums (samples past the output are masked)."""
    s = synth.Setup(f"wg-{n_out}", 1024, 1420.0, 0.29296875, 50e-6, 3.0, 0.25, 41, n_out)
    plan = dd.Plan.from_setup(s, "f32")
    assert "tmw9_f32_d9_t4096" in plan.configs()
    d = oracle_table(s)
    stride = plan.padded_in_stride()
    x, _ = make_input(s, "f32", 11, plan.n_in, stride)
    x[:, plan.n_in:] = np.nan
    g = synth.noise_f32(12, s.n_dm, s.n_out)
    xt, gt = torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda()
    _, gw = plan.adjoint(gt, x=xt, grad_in=False, grad_w=True)
    _, gw_again = plan.adjoint(gt, x=xt, grad_in=False, grad_w=True)
    _, gw_transposed = plan.adjoint(gt, x=xt, grad_in=True, grad_w=True)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    assert torch.equal(gw, gw_again)
    xs = np.ascontiguousarray(x[:, :plan.n_in])
    refw = oracle.wgrad_f32(d, g, xs)
    scalew = oracle.wgrad_f32(d, np.abs(g), np.abs(xs))
    for got in (gw, gw_transposed):
        errw = np.abs(got.cpu().numpy().astype(np.float64) - refw)
        assert np.isfinite(errw).all()
        assert (errw <= FP32_REL * scalew).all(), float((errw - FP32_REL * scalew).max())


def test_adjoint_full_apertif_sampled(dd):
    """Full Apertif size: a sample of channels checked against the oracle on all DMs."""
    s = synth.APERTIF
    plan = dd.Plan.from_setup(s, "f32")
    d = oracle_table(s)
    g = synth.noise_f32(9, s.n_dm, s.n_out)
    gi, _ = plan.adjoint(torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    got = gi.cpu().numpy()
    cols = [0, 1, 511, 1022, 1023]
    sub = np.ascontiguousarray(d[:, cols])
    ref = oracle.adjoint_f32(sub, g, plan.n_in)
    scale = oracle.adjoint_f32(sub, np.abs(g), plan.n_in)
    err = np.abs(got[cols].astype(np.float64) - ref)
    assert (err <= FP32_REL * scale).all()


def test_dot_product_identity_gpu(dd):
    """<A x, y> = <x, A^T y> with both sides from the GPU (fp32 rounding only)."""
    s = synth.Setup("dot", 256, 1420.0, 1.171875, 50e-6, 0.0, 0.25, 96, 4000)
    plan = dd.Plan.from_setup(s, "f32")
    x = torch.randn((s.channels, plan.padded_in_stride()), device="cuda")
    y = torch.randn((s.n_dm, s.n_out), device="cuda")
    w = torch.rand(s.channels, device="cuda") + 0.5
    ax = plan.forward(x, w)
    aty, _ = plan.adjoint(y, w=w)
    lhs = float((ax.double() * y.double()).sum())
    rhs = float((x[:, :plan.n_in].double() * aty.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * float((ax.abs().double() * y.abs().double()).sum())


def test_boxcar_snr_matches_oracle(dd):
    s = synth.TINY
    plan = dd.Plan.from_setup(s, "f32")
    d = oracle_table(s)
    x, _ = make_input(s, "f32", 0, plan.n_in, plan.padded_in_stride(), pulses=1, d=d)
    out = plan.forward(torch.from_numpy(x).cuda())
    raw, grad = dd.boxcar_snr(out, grad=True)
    torch.cuda.synchronize()
    res = dd.snr_result(raw)
    o = out.cpu().numpy().astype(np.float64)
    loss, g_ref, (bi, bt) = oracle.boxcar_snr_loss(o)
    assert res["valid"] == 1
    assert (res["best_row"], res["best_t"]) == (bi, bt)
    assert abs(res["loss"] - loss) <= 1e-9 * abs(loss)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.abs(g - g_ref).max() <= 1e-6 * np.abs(g_ref).max()


def test_boxcar_snr_constant_rows(dd):
    x = torch.zeros((3, 16), device="cuda")
    x[1, 4] = 1.0
    x[2] = 7.0
    raw, grad = dd.boxcar_snr(x, grad=True)
    res = dd.snr_result(raw)
    assert res["valid"] == 1 and (res["best_row"], res["best_t"]) == (1, 0)
    assert abs(res["loss"] + 2.0 / np.sqrt(5.0)) < 1e-12     # closed form of tests/golden/loss_spike.txt
    raw, _ = dd.boxcar_snr(torch.ones((2, 20), device="cuda"))
    assert dd.snr_result(raw)["valid"] == 0


def test_autograd_chain_matches_oracle(dd):
    """dedisperse -> boxcar S/N loss, backward through dd_adjoint, against the oracle gradient."""
    from paper_1601_01165_gb300.autograd import boxcar_snr_loss, dedisperse
    s = synth.Setup("grad", 128, 1420.0, 2.34375, 50e-6, 0.0, 0.25, 64, 3000)
    plan = dd.Plan.from_setup(s, "f32")
    d = oracle_table(s)
    x_np, _ = make_input(s, "f32", 4, plan.n_in, plan.padded_in_stride(), pulses=1, d=d)
    x = torch.from_numpy(x_np).cuda().requires_grad_(True)
    w = torch.ones(s.channels, device="cuda", requires_grad=True)
    out = dedisperse(x, w, plan)
    loss = boxcar_snr_loss(out)
    loss.backward()
    torch.cuda.synchronize()
    o = out.detach().cpu().numpy().astype(np.float64)
    l_ref, go_ref, _ = oracle.boxcar_snr_loss(o)
    assert abs(float(loss) - l_ref) <= 1e-6 * abs(l_ref)
    go32 = go_ref.astype(np.float32)
    xs = np.ascontiguousarray(x_np[:, :plan.n_in])
    gx_ref = oracle.adjoint_f32(d, go32, plan.n_in, np.ones(s.channels, np.float32))
    gx_scale = oracle.adjoint_f32(d, np.abs(go32), plan.n_in)
    gx = x.grad.cpu().numpy()
    assert (gx[:, plan.n_in:] == 0).all()
    tol = 1e-4 * gx_scale + 1e-6 * np.abs(gx_ref).max()
    assert (np.abs(gx[:, :plan.n_in] - gx_ref) <= tol).all()
    gw_ref = oracle.wgrad_f32(d, go32, xs)
    gw_scale = oracle.wgrad_f32(d, np.abs(go32), np.abs(xs))
    assert (np.abs(w.grad.cpu().numpy() - gw_ref) <= 1e-4 * gw_scale + 1e-6).all()


def test_weight_gradient_finite_differences(dd):
    from paper_1601_01165_gb300.autograd import boxcar_snr_loss, dedisperse
    s = synth.Setup("fd", 64, 1420.0, 4.6875, 50e-6, 0.0, 0.25, 32, 2000)
    plan = dd.Plan.from_setup(s, "f32")
    d = oracle_table(s)
    x_np, _ = make_input(s, "f32", 5, plan.n_in, plan.padded_in_stride(), pulses=1, d=d)
    x = torch.from_numpy(x_np).cuda()
    w = torch.ones(s.channels, device="cuda", requires_grad=True)
    boxcar_snr_loss(dedisperse(x, w, plan)).backward()
    gw = w.grad.double().cpu().numpy()
    h = 1e-2
    for c in (0, 17, 63):
        wp = torch.ones(s.channels, device="cuda")
        wm = torch.ones(s.channels, device="cuda")
        wp[c] += h
        wm[c] -= h
        lp = float(boxcar_snr_loss(plan.forward(x, wp)))
        lm = float(boxcar_snr_loss(plan.forward(x, wm)))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gw[c]) <= 0.05 * abs(gw).max(), (c, fd, gw[c])


def test_adjoint_errors(dd):
    plan = dd.Plan.from_setup(synth.TINY, "u8")
    g = torch.zeros((synth.TINY.n_dm, synth.TINY.n_out), device="cuda")
    with pytest.raises(dd.DDError) as e:
        plan.adjoint(g)
    assert e.value.name == "DD_ERR_UNSUPPORTED"
    plan = dd.Plan.from_setup(synth.TINY, "f32")
    with pytest.raises(dd.DDError) as e:
        plan.adjoint(g, grad_in=False, grad_w=False)
    assert e.value.name == "DD_ERR_ARG"
