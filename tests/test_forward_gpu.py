"""GPU parity of the forward path (Algorithm 1) against the oracle, through the C ABI."""
import numpy as np
import pytest

from paper_1601_01165_gb300 import synth
from helpers import assert_parity, full_parity, make_input, oracle_table, oracle_window

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_01165_gb300 import binding
    binding.load()
    return binding


def _run(dd, setup, dtype, seed=0, weighted=False, cfg=None, pulses=0, row_pad=0):
    plan = dd.Plan.from_setup(setup, dtype)
    d = oracle_table(setup)
    assert plan.n_in == setup.n_out + int(d.max())
    if cfg is not None:
        plan.select(cfg)
    stride = plan.padded_in_stride() + row_pad
    x, sites = make_input(setup, dtype, seed, plan.n_in, stride, pulses, d)
    w = synth.weights(seed, setup.channels) if weighted else None
    xt = torch.from_numpy(x).cuda()
    wt = torch.from_numpy(w).cuda() if w is not None else None
    out = plan.forward(xt, wt)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    return plan, d, x, w, out.cpu().numpy(), sites


def test_plan_delay_table_matches_oracle(dd):
    for s in (synth.TINY, synth.APERTIF, synth.LOFAR):
        plan = dd.Plan.from_setup(s, "f32")
        assert (plan.delays() == oracle_table(s)).all()


def _all_configs(dd, setup, dtype):
    return dd.Plan.from_setup(setup, dtype).configs()


@pytest.mark.parametrize("dtype,weighted", [("f32", False), ("f32", True), ("u8", False)])
def test_tiny_every_config(dd, dtype, weighted):
    s = synth.TINY
    for cfg in _all_configs(dd, s, dtype):
        plan, d, x, w, got, _ = _run(dd, s, dtype, seed=1, weighted=weighted, cfg=cfg)
        ref, scale = oracle_window(d, x, dtype, 0, s.n_dm, 0, s.n_out, w)
        assert_parity(got, ref, scale, dtype, where=f"tiny {dtype} w={weighted} {cfg}")


RAGGED = [
    synth.Setup("ragged-a", 37, 1420.0, 0.29296875 * 1024 / 37, 50e-6, 0.0, 0.25, 3, 1001),
    synth.Setup("ragged-b", 5, 400.0, 8.0, 1e-3, 0.0, 3.0, 1, 17),
    synth.Setup("ragged-c", 130, 1420.0, 2.0, 50e-6, 0.0, 0.5, 45, 2999),
    synth.Setup("zero-dm", 64, 1400.0, 1.0, 1e-3, 0.0, 0.0, 2, 1500),
    synth.Setup("lofar-cut", 32, 138.0, 0.1953125, 5e-6, 0.0, 0.01, 70, 3001),
    synth.Setup("apertif-cut", 1024, 1420.0, 0.29296875, 50e-6, 3.0, 0.25, 41, 1931),
    # one channel: a single chunk in which most copying lanes have nothing to copy
    synth.Setup("one-channel", 1, 1420.0, 1.0, 50e-6, 0.0, 0.25, 7, 1777),
    # a 32-channel chunk and a 1-channel chunk; 70 trials end inside a DM block
    synth.Setup("c33", 33, 1420.0, 300.0 / 33, 50e-6, 0.0, 0.25, 70, 2500),
]


@pytest.mark.parametrize("setup", RAGGED, ids=lambda s: s.name)
@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_ragged_every_config(dd, setup, dtype):
    for cfg in _all_configs(dd, setup, dtype):
        plan, d, x, w, got, _ = _run(dd, setup, dtype, seed=2, weighted=(dtype == "f32"), cfg=cfg)
        ref, scale = oracle_window(d, x, dtype, 0, setup.n_dm, 0, setup.n_out, w)
        assert_parity(got, ref, scale, dtype, where=f"{setup.name} {dtype} {cfg}")


FULL = [(synth.APERTIF, "f32", False), (synth.APERTIF, "f32", True), (synth.APERTIF, "u8", False),
        (synth.LOFAR, "f32", False)]


@pytest.mark.parametrize("setup,dtype,weighted", FULL,
                         ids=["apertif-f32", "apertif-f32-weighted", "apertif-u8", "lofar-f32"])
def test_full_size_every_element(dd, setup, dtype, weighted):
    """Full-size beams against the oracle, every output element: the plan's
    default configuration (the launch the benchmark times) and, for the
    Apertif beam, every other configuration of its menu on the same input.
    Covers every tile seam of every kernel (the float Tensor-Memory kernel's
    4096-sample time tiles and 6-trial groups, the staged kernels' DM blocks
    and time tiles) and the ragged tails.  Bit-exact for uint8; for float32
    within 1e-5 of the sum of the terms' magnitudes, element by element.
    The injected pulses must also peak at their true (DM, time)."""
    n_pulses = 3 if setup is synth.APERTIF else 2
    plan, d, x, w, got, sites = _run(dd, setup, dtype, seed=0, weighted=weighted, pulses=n_pulses)
    outputs = {f"default {plan.selected}": got}
    if setup is synth.APERTIF:
        xt = torch.from_numpy(x).cuda()
        wt = torch.from_numpy(w).cuda() if w is not None else None
        for cfg in plan.configs():
            if cfg == plan.selected:
                continue
            p2 = dd.Plan.from_setup(setup, dtype)
            p2.select(cfg)
            outputs[cfg] = p2.forward(xt, wt).cpu().numpy()
            assert p2.device_status() == 0, cfg
            p2.close()
        del xt
    seams = [t for t in range(4096, setup.n_out, 4096)]
    res = full_parity(d, x, dtype, outputs, w=w, n_out=setup.n_out)
    for name, (bad, worst) in res.items():
        assert bad == 0, (f"{setup.name} {dtype} w={weighted} {name}: {bad} of {setup.n_dm * setup.n_out} "
                          f"outputs outside the bound (worst {worst:.3g} of it); seams at {seams[:3]}...")
    for (i_p, t_p) in sites:
        i0, i1 = max(0, i_p - 12), min(setup.n_dm, i_p + 13)
        ta, tb = max(0, t_p - 40), min(setup.n_out, t_p + 43)
        blk = got[i0:i1, ta:tb].astype(np.float64)
        i, t = np.unravel_index(blk.argmax(), blk.shape)
        assert i0 + i == i_p and t_p <= ta + t <= t_p + 2, (i_p, t_p, i0 + i, ta + t)


def test_strides_and_canary(dd):
    s = synth.Setup("stride", 96, 1420.0, 1.5, 50e-6, 0.0, 0.25, 24, 1234)
    for dtype in ("f32", "u8"):
        plan = dd.Plan.from_setup(s, dtype)
        d = oracle_table(s)
        stride = plan.padded_in_stride() + (64 if dtype == "u8" else 12)
        x, _ = make_input(s, dtype, 5, plan.n_in, stride)
        xt = torch.from_numpy(x).cuda()
        big = torch.full((s.n_dm, s.n_out + 77), -7, dtype=plan.out_dtype, device="cuda")
        out = big[:, 5:5 + s.n_out]
        plan.forward(xt, out=out)
        torch.cuda.synchronize()
        b = big.cpu().numpy()
        assert (b[:, :5] == -7).all() and (b[:, 5 + s.n_out:] == -7).all()
        ref, scale = oracle_window(d, x, dtype, 0, s.n_dm, 0, s.n_out)
        assert_parity(b[:, 5:5 + s.n_out], ref, scale, dtype, where=f"strided {dtype}")


def test_unaligned_input_uses_plain_kernel(dd):
    s = synth.Setup("unaligned", 40, 1420.0, 2.0, 50e-6, 0.0, 0.25, 16, 999)
    plan = dd.Plan.from_setup(s, "f32")
    d = oracle_table(s)
    x, _ = make_input(s, "f32", 6, plan.n_in + 1, plan.n_in + 1)
    xt = torch.from_numpy(x).cuda()
    view = xt[:, 1:]          # 4-byte offset: not 16-byte aligned
    out = plan.forward(view)
    torch.cuda.synchronize()
    ref, scale = oracle_window(d, np.ascontiguousarray(x[:, 1:]), "f32", 0, s.n_dm, 0, s.n_out)
    assert_parity(out.cpu().numpy(), ref, scale, "f32", where="unaligned")


@pytest.mark.parametrize("n_out", [4000, 13000])
def test_forward_host_matches_device(dd, n_out):
    """The host-buffer entry point pipelines time chunks (copy in, kernel, copy
    out on separate streams); 13000 samples make chunks of 4096, 8192 and 712."""
    s = synth.Setup("host", 256, 1420.0, 1.171875, 50e-6, 0.0, 0.25, 64, n_out)
    for dtype in ("f32", "u8"):
        plan = dd.Plan.from_setup(s, dtype)
        d = oracle_table(s)
        x, _ = make_input(s, dtype, 7, plan.n_in)
        w = synth.weights(7, s.channels) if dtype == "f32" else None
        xh = torch.from_numpy(x).pin_memory()
        wh = torch.from_numpy(w) if w is not None else None
        got = plan.forward_host(xh, wh).numpy()
        dev = plan.forward(torch.from_numpy(np.ascontiguousarray(
            np.pad(x, ((0, 0), (0, plan.padded_in_stride() - plan.n_in))))).cuda(),
            torch.from_numpy(w).cuda() if w is not None else None).cpu().numpy()
        assert (got == dev).all()
        ref, scale = oracle_window(d, x, dtype, 0, s.n_dm, 0, s.n_out, w)
        assert_parity(got, ref, scale, dtype, where=f"host {dtype} {n_out}")


def test_errors(dd):
    s = synth.TINY
    plan = dd.Plan.from_setup(s, "u8")
    x = plan.alloc_input()
    w = torch.ones(s.channels, device="cuda")
    with pytest.raises(dd.DDError) as e:
        plan.forward(x, w)
    assert e.value.name == "DD_ERR_UNSUPPORTED"
    short = torch.zeros((s.channels, plan.n_in - 1), dtype=torch.uint8, device="cuda")
    with pytest.raises(dd.DDError) as e:
        plan.forward(short)
    assert e.value.name == "DD_ERR_SHAPE"
    with pytest.raises(dd.DDError) as e:
        dd.Plan(0, 1400.0, 1.0, 1e-3, 0.0, 1.0, 4, 100)
    assert e.value.name == "DD_ERR_ARG"


SATURATED = [
    synth.Setup(f"sat-{c}", c, 1420.0, 300.0 / c, 50e-6, 0.0, 0.25, 12, 2100) for c in (255, 256, 257, 512, 513, 1024)
]


@pytest.mark.parametrize("setup", SATURATED, ids=lambda s: s.name)
def test_u8_saturated_sums_are_exact(dd, setup):
    """8-bit sums at their largest: every sample 255 gives exactly 255 * C at
    every output (a closed form, no oracle), and random 0/255 samples match the
    oracle bit for bit.  Channel counts straddle the 256-channel periods over
    which the packed kernels' 16-bit partial sums are exact."""
    c = setup.channels
    d = oracle_table(setup)
    for cfg in _all_configs(dd, setup, "u8"):
        plan = dd.Plan.from_setup(setup, "u8")
        plan.select(cfg)
        stride = plan.padded_in_stride()
        full = torch.full((c, stride), 255, dtype=torch.uint8, device="cuda")
        out = plan.forward(full).cpu().numpy()
        assert plan.device_status() == 0
        assert (out == 255 * c).all(), f"{setup.name} {cfg}: saturated sum {out.min()}..{out.max()} != {255 * c}"
        rng = np.random.default_rng(c)
        x = np.zeros((c, stride), dtype=np.uint8)
        x[:, :plan.n_in] = rng.choice(np.array([0, 255], dtype=np.uint8), size=(c, plan.n_in))
        got = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
        assert plan.device_status() == 0
        ref, _ = oracle_window(d, x, "u8", 0, setup.n_dm, 0, setup.n_out)
        assert_parity(got, ref, None, "u8", where=f"{setup.name} {cfg}")


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_dm_range_plans_tile_the_full_plan(dd, dtype):
    """One beam split by DM trials (dd_plan_dm_range): the plans of blocks
    [i0, i1) have the full plan's delay rows, and their outputs, stacked,
    equal the full plan's output bit for bit, for blocks that start on and
    off the kernels' trial tiles."""
    from paper_1601_01165_gb300.shard import split_dm_range
    s = synth.Setup("apertif-dm-split", 1024, 1420.0, 0.29296875, 50e-6, 0.0, 0.25, 100, 4500)
    full = dd.Plan.from_setup(s, dtype)
    d = full.delays()
    x, _ = make_input(s, dtype, 11, full.n_in, full.padded_in_stride())
    xt = torch.from_numpy(x).cuda()
    ref = full.forward(xt).cpu().numpy()
    for world, align in ((3, 6), (4, 1), (2, 64)):
        parts = split_dm_range(s.n_dm, world, align)
        rows = []
        for i0, i1 in parts:
            if i1 == i0:
                continue
            sub = dd.Plan.dm_range(s, i0, i1, dtype)
            assert (sub.delays() == d[i0:i1]).all()
            assert sub.n_in <= full.n_in
            rows.append(sub.forward(xt).cpu().numpy())   # the whole input, as every rank holds it
            assert sub.device_status() == 0
        got = np.concatenate(rows)
        assert got.shape == ref.shape
        assert np.array_equal(got, ref), f"world {world} align {align}"
