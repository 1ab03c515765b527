"""GPU parity of the Tensor-Memory window kernels (TMW6: 6 trials per window,
TMW9: 9 trials per window, 4-float copies through eight tensor-map views) at
their edges: channel counts that leave partial 3-channel steps, trial counts
that leave partial groups, time tails of one sample, the largest in-group
offset the windows hold (31 samples), every start residue of a window, and
the layouts that send a launch to another kernel."""
import numpy as np
import pytest

from paper_1601_01165_gb300 import synth
from helpers import assert_parity, make_input, oracle_table, oracle_window

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TMW6 = "tmw6_f32_d6_t4096"
TMW9 = "tmw9_f32_d9_t4096"
KERNELS = [(TMW6, 6), (TMW9, 9)]
IDS = ["tmw6", "tmw9"]
MAX_OFFSET = {TMW6: 31, TMW9: 31}


@pytest.fixture(scope="module")
def dd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_01165_gb300 import binding
    binding.load()
    return binding


def _group_max_offset(s, group):
    d = oracle_table(s)
    worst = 0
    for g0 in range(0, s.n_dm, group):
        g1 = min(g0 + group, s.n_dm)
        worst = max(worst, int((d[g1 - 1] - d[g0]).max()))
    return worst


def _check(dd, s, kernel, seed, weighted, stride_pad=0, out_pad=0, stride=None):
    plan = dd.Plan.from_setup(s, "f32")
    assert kernel in plan.configs(), s
    plan.select(kernel)
    d = oracle_table(s)
    stride = (plan.padded_in_stride() if stride is None else stride) + stride_pad
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
    assert_parity(b[:, :s.n_out], ref, scale, "f32",
                  where=f"{s.name} {kernel} w={weighted} pad={stride_pad},{out_pad}")
    return b[:, :s.n_out]


def test_menu_gating(dd):
    ap = dd.Plan.from_setup(synth.APERTIF, "f32")
    assert all(k in ap.configs() for k, _ in KERNELS)
    assert ap.selected == TMW9
    lofar = dd.Plan.from_setup(synth.LOFAR, "f32").configs()     # group offsets up to 180 and more
    assert not any(k in lofar for k, _ in KERNELS)
    u8 = dd.Plan.from_setup(synth.APERTIF, "u8").configs()
    assert not any(k in u8 for k, _ in KERNELS)
    assert ap.padded_in_stride() % 32 == 0 and ap.padded_in_stride() >= ap.n_in + 28


@pytest.mark.parametrize("kernel,group", KERNELS, ids=IDS)
@pytest.mark.parametrize("C", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("n_dm,n_out", [(1, 1), (9, 4095), (13, 2049), (25, 8200)])
def test_partial_steps_and_groups(dd, kernel, group, C, n_dm, n_out):
    s = synth.Setup(f"edge-c{C}-d{n_dm}-t{n_out}", C, 1420.0, 300.0 / max(C, 2), 50e-6, 1.0, 0.25, n_dm, n_out)
    _check(dd, s, kernel, seed=C * 7 + n_dm, weighted=(C % 2 == 1))


def _setup_with_offset(target, group):
    """A small setup whose largest in-group offset (groups of `group` trials) is exactly `target` samples."""
    for k in range(4000):
        step = 0.3 + 0.005 * k
        s = synth.Setup(f"offset{target}-g{group}", 16, 400.0, 4.0, 1e-3, 0.0, step, 2 * group, 5000)
        if _group_max_offset(s, group) == target:
            return s
    raise AssertionError(f"no dm_step gives an in-group offset of {target}")


@pytest.mark.parametrize("kernel,group", KERNELS, ids=IDS)
def test_largest_window_offset(dd, kernel, group):
    most = MAX_OFFSET[kernel]
    s = _setup_with_offset(most, group)
    _check(dd, s, kernel, seed=3, weighted=True)
    _check(dd, s, kernel, seed=4, weighted=False, out_pad=3)
    too_far = _setup_with_offset(most + 1, group)
    assert kernel not in dd.Plan.from_setup(too_far, "f32").configs()


def test_every_window_residue(dd):
    """Windows whose first sample falls on each residue mod 32 (so each of
    TMW9's eight tensor-map views, and each of the four sub-chunk shifts),
    checked against the oracle: 64 channels spread the base delays."""
    s = synth.Setup("residues", 64, 1420.0, 4.6875, 50e-6, 7.0, 0.25, 27, 4500)
    d = oracle_table(s)
    res = {int(v) % 32 for v in d[::9].ravel()}
    assert res == set(range(32)), sorted(res)
    a = _check(dd, s, TMW9, seed=12, weighted=True)
    b = _check(dd, s, TMW6, seed=12, weighted=True)
    assert (a == b).all()


@pytest.mark.parametrize("kernel,group", KERNELS, ids=IDS)
def test_fallback_layouts_give_the_same_sums(dd, kernel, group):
    """Rows the kernel cannot take go to another kernel (TMW9 without 28 spare
    floats per row: TMW6; rows that are not a multiple of 128 bytes: the
    staged kernel); the sums run in the same channel order, so the outputs
    are bit-identical."""
    s = synth.Setup("fallback", 64, 1420.0, 4.6875, 50e-6, 0.0, 0.25, 20, 5000)
    a = _check(dd, s, kernel, seed=9, weighted=True)
    b = _check(dd, s, kernel, seed=9, weighted=True, stride_pad=4, out_pad=1)   # odd output pitch too
    assert (a == b).all()
    plan = dd.Plan.from_setup(s, "f32")
    tight = (plan.n_in + 31) // 32 * 32          # a 128-byte multiple with fewer than 28 spare floats
    if tight - plan.n_in < 28:
        c = _check(dd, s, kernel, seed=9, weighted=True, stride=tight)
        assert (a == c).all()


def test_full_apertif_equals_staged(dd):
    """On the full Apertif beam TMW9, TMW6 and the staged kernel add every
    channel in the same order: their outputs are bit-identical."""
    s = synth.APERTIF
    plan = dd.Plan.from_setup(s, "f32")
    x = plan.alloc_input()
    x.normal_(generator=torch.Generator(device="cuda").manual_seed(5))
    outs = []
    for cfg in (TMW9, TMW6, "staged_d32_t512_c4_s3"):
        plan.select(cfg)
        outs.append(plan.forward(x))
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    assert all(torch.equal(outs[0], o) for o in outs[1:])
