"""GPU parity of the Tensor-Memory window kernel (TMW6) at its edges: channel
counts that leave partial 3-channel steps, trial counts that leave partial
6-trial groups, time tails of one sample, the largest in-group offset the
windows hold (31 samples) and the layouts that send it to the shared-memory
fallback."""
import pytest

from paper_1601_01165_gb300 import synth
from helpers import assert_parity, make_input, oracle_table, oracle_window

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TMW6 = "tmw6_f32_d6_t4096"


@pytest.fixture(scope="module")
def dd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_01165_gb300 import binding
    binding.load()
    return binding


def _group_max_offset(s):
    d = oracle_table(s)
    worst = 0
    for g0 in range(0, s.n_dm, 6):
        g1 = min(g0 + 6, s.n_dm)
        worst = max(worst, int((d[g1 - 1] - d[g0]).max()))
    return worst


def _check(dd, s, seed, weighted, stride_pad=0, out_pad=0):
    plan = dd.Plan.from_setup(s, "f32")
    assert TMW6 in plan.configs(), s
    plan.select(TMW6)
    d = oracle_table(s)
    stride = plan.padded_in_stride() + stride_pad
    x, _ = make_input(s, "f32", seed, plan.n_in, stride)
    w = synth.weights(seed, s.channels) if weighted else None
    wt = torch.from_numpy(w).cuda() if w is not None else None
    big = torch.full((s.n_dm, s.n_out + out_pad), -7.0, device="cuda")
    out = big[:, :s.n_out]
    plan.forward(torch.from_numpy(x).cuda(), wt, out=out)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    b = big.cpu().numpy()
    if out_pad:
        assert (b[:, s.n_out:] == -7.0).all()
    ref, scale = oracle_window(d, x, "f32", 0, s.n_dm, 0, s.n_out, w)
    assert_parity(b[:, :s.n_out], ref, scale, "f32", where=f"{s.name} w={weighted} pad={stride_pad},{out_pad}")
    return b[:, :s.n_out]


def test_menu_gating(dd):
    assert TMW6 in dd.Plan.from_setup(synth.APERTIF, "f32").configs()
    assert dd.Plan.from_setup(synth.APERTIF, "f32").selected == TMW6
    assert TMW6 not in dd.Plan.from_setup(synth.LOFAR, "f32").configs()     # group offsets up to 180
    assert TMW6 not in dd.Plan.from_setup(synth.APERTIF, "u8").configs()


@pytest.mark.parametrize("C", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("n_dm,n_out", [(1, 1), (6, 4095), (7, 4097), (13, 8200)])
def test_partial_steps_and_groups(dd, C, n_dm, n_out):
    s = synth.Setup(f"edge-c{C}-d{n_dm}-t{n_out}", C, 1420.0, 300.0 / max(C, 2), 50e-6, 1.0, 0.25, n_dm, n_out)
    _check(dd, s, seed=C * 7 + n_dm, weighted=(C % 2 == 1))


def _setup_with_offset(target):
    """A small setup whose largest 6-trial in-group offset is exactly `target` samples."""
    for k in range(2000):
        step = 0.5 + 0.01 * k
        s = synth.Setup(f"offset{target}", 16, 400.0, 4.0, 1e-3, 0.0, step, 12, 5000)
        if _group_max_offset(s) == target:
            return s
    raise AssertionError(f"no dm_step gives an in-group offset of {target}")


def test_largest_window_offset(dd):
    s = _setup_with_offset(31)
    _check(dd, s, seed=3, weighted=True)
    _check(dd, s, seed=4, weighted=False, out_pad=3)
    too_far = _setup_with_offset(32)
    assert TMW6 not in dd.Plan.from_setup(too_far, "f32").configs()


def test_fallback_layouts_give_the_same_sums(dd):
    """Rows that are not a multiple of 128 bytes go to the staged fallback; the
    sums run in the same channel order, so the outputs are bit-identical."""
    s = synth.Setup("fallback", 64, 1420.0, 4.6875, 50e-6, 0.0, 0.25, 20, 5000)
    a = _check(dd, s, seed=9, weighted=True)
    b = _check(dd, s, seed=9, weighted=True, stride_pad=4, out_pad=1)   # odd output pitch too
    assert (a == b).all()


def test_full_apertif_equals_staged(dd):
    """On the full Apertif beam TMW6 and the staged kernel add every channel in
    the same order: their outputs are bit-identical."""
    s = synth.APERTIF
    plan = dd.Plan.from_setup(s, "f32")
    x = plan.alloc_input()
    x.normal_(generator=torch.Generator(device="cuda").manual_seed(5))
    plan.select(TMW6)
    a = plan.forward(x)
    plan.select("staged_d32_t512_c4_s3")
    b = plan.forward(x)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    assert torch.equal(a, b)
