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
    from paper_1601_01165_gb300.serve import BeamSpec, beam_bytes
    s = synth.Setup("b", 32, 1420.0, 300.0 / 32, 50e-6, 0.0, 0.25, 16, 0)
    u8 = beam_bytes(BeamSpec("a", s, "u8", chunk_len=1000, n_chunks=1, period_s=1.0))
    f32 = beam_bytes(BeamSpec("a", s, "f32", chunk_len=1000, n_chunks=1, period_s=1.0))
    assert f32 > u8 > 16 * 1000 * 4          # output chunk (int32 / float32) at least


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
