"""Failure detection on the GPU without a fault: a kernel's bounded wait is
made to expire (an mbarrier phase nothing completes, with a 1 ms limit); the
code must reach the plan's status word, be cleared by reading it, and leave
the context usable for the next forward launch."""
import pytest

from paper_1601_01165_gb300 import synth
from helpers import assert_parity, make_input, oracle_table, oracle_window

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_01165_gb300 import binding
    binding.load()
    return binding


def test_expired_wait_is_reported_and_the_context_survives(dd):
    s = synth.TINY
    plan = dd.Plan.from_setup(s, "f32")
    assert plan.device_status() == 0
    plan.check_wait_timeout(limit_cycles=2_000_000)      # about 1 ms at GB300 clocks
    assert plan.device_status() == 1                     # kDevWaitTimeout
    assert plan.device_status() == 0                     # reading clears the word
    d = oracle_table(s)
    x, _ = make_input(s, "f32", 11, plan.n_in, plan.padded_in_stride())
    out = plan.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    ref, scale = oracle_window(d, x, "f32", 0, s.n_dm, 0, s.n_out)
    assert_parity(out.cpu().numpy(), ref, scale, "f32", where="after an expired wait")


def test_wait_limit_out_of_range(dd):
    plan = dd.Plan.from_setup(synth.TINY, "f32")
    for bad in (0, -5, 3_000_000_000):
        with pytest.raises(dd.DDError) as e:
            plan.check_wait_timeout(limit_cycles=bad)
        assert e.value.name == "DD_ERR_ARG"
