"""Serving loop: admission denial on the host, and late chunks on the GPU
(a source slower than the beam's period makes chunks miss their deadline,
is reported as such, and still yields the same dedispersed output)."""
import time

import numpy as np
import pytest

from paper_1601_01165_gb300 import synth


def test_beam_larger_than_the_budget_is_refused():
    from paper_1601_01165_gb300.serve import AdmissionError, BeamSpec, Server, beam_bytes
    s = synth.Setup("big", 64, 1420.0, 300.0 / 64, 50e-6, 0.0, 0.25, 48, 0)
    spec = BeamSpec("big", s, "f32", chunk_len=2000, n_chunks=2, period_s=0.05)
    with pytest.raises(AdmissionError):
        Server(beam_bytes(spec) - 1).run([spec], lambda sp, k: None)


def test_beam_bytes_counts_tail_chunk_and_tables():
    """The admission size is the library's own footprint (host-only queries,
    no GPU): plan tables, the stream's plan and two tail buffers, chunks."""
    from paper_1601_01165_gb300 import binding
    from paper_1601_01165_gb300.serve import BeamSpec, beam_bytes
    s = synth.Setup("b", 32, 1420.0, 300.0 / 32, 50e-6, 0.0, 0.25, 16, 0)
    geo = (s.channels, s.f_low_mhz, s.chan_bw_mhz, s.t_samp_s, s.dm_first, s.dm_step, s.n_dm)
    max_d = int(binding.delay_table(*geo).max())
    for dtype, elem in (("u8", 1), ("f32", 4)):
        spec = BeamSpec("a", s, dtype, chunk_len=1000, n_chunks=1, period_s=1.0)
        plan = binding.plan_footprint(*geo, dtype=dtype)
        stream = binding.stream_footprint(*geo, 1000, dtype=dtype)
        # tables: the delay table and its transposed copy at least; the stream
        # holds its own plan's tables and two buffers of max_delay + chunk samples
        assert plan >= 2 * 4 * s.channels * s.n_dm
        assert stream >= plan + 2 * s.channels * (max_d + 1000) * elem
        assert beam_bytes(spec) == plan + stream + s.channels * 1000 * elem + 4 * s.n_dm * 1000
    # float plans also hold the Tensor-Memory window descriptors
    assert binding.plan_footprint(*geo, dtype="f32") > binding.plan_footprint(*geo, dtype="u8")
    with pytest.raises(binding.DDError):
        binding.plan_footprint(0, *geo[1:], dtype="f32")


@pytest.mark.gpu
def test_late_chunks_are_reported_and_still_correct():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_01165_gb300 import binding as dd
    from paper_1601_01165_gb300.serve import BeamSpec, Server
    s = synth.Setup("late", 64, 1420.0, 300.0 / 64, 50e-6, 0.0, 0.25, 32, 0)
    spec = BeamSpec("late", s, "u8", chunk_len=2000, n_chunks=4, period_s=0.02, keep_output=True)

    def slow_source(sp, k):
        if k == 2:
            time.sleep(0.1)                   # five periods late
        return synth.noise_u8(50 + k, sp.setup.channels, sp.chunk_len)

    # the footprints the admission used are what the created objects hold
    from paper_1601_01165_gb300.serve import beam_bytes
    geo = (s.channels, s.f_low_mhz, s.chan_bw_mhz, s.t_samp_s, s.dm_first, s.dm_step, s.n_dm)
    p0 = dd.Plan(*geo, spec.chunk_len, "u8")
    st0 = dd.Stream(p0, spec.chunk_len)
    assert p0.device_bytes == dd.plan_footprint(*geo, dtype="u8")
    assert st0.device_bytes() == dd.stream_footprint(*geo, spec.chunk_len, dtype="u8")
    assert beam_bytes(spec) == p0.device_bytes + st0.device_bytes() + s.channels * 2000 + 4 * s.n_dm * 2000
    st0.close()
    p0.close()
    rep = Server(1 << 34).run([spec], slow_source)
    assert rep["chunks"] == 4
    assert rep["deadline_misses"] >= 1
    plan = dd.Plan(s.channels, s.f_low_mhz, s.chan_bw_mhz, s.t_samp_s, s.dm_first, s.dm_step, s.n_dm,
                   spec.chunk_len, "u8")
    alone = dd.Stream(plan, spec.chunk_len)
    for k in range(spec.n_chunks):
        out, t0 = alone.push(torch.from_numpy(synth.noise_u8(50 + k, s.channels, spec.chunk_len)).cuda())
        assert t0 == rep["outputs"]["late"][k][0]
        assert np.array_equal(out.cpu().numpy(), rep["outputs"]["late"][k][1].numpy())
