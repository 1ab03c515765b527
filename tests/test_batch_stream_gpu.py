"""GPU tests of the batched launch, streaming state, auto-tuner and serving loop."""
import json

import numpy as np
import pytest

import oracle
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


def _small_batch(seed=0):
    """Uneven beams of both grids and both dtypes, small enough for quick checks."""
    rng = np.random.default_rng(seed)
    beams = []
    for b in range(7):
        C = int(rng.choice([32, 64, 256]))
        n_dm = int(rng.choice([16, 40, 96]))
        n_out = int(rng.integers(1500, 9000))
        if b % 2:
            s = synth.Setup(f"b{b}", C, 1420.0, 300.0 / C, 50e-6, 0.0, 0.25, n_dm, n_out)
        else:
            s = synth.Setup(f"b{b}", C, 138.0, 6.25 / C, 5e-6, 0.0, 0.01, n_dm, n_out)
        beams.append((s, "u8" if b % 3 == 0 else "f32"))
    return beams


def _inputs(dd, beams, seed):
    plans, xs, hosts = [], [], []
    for k, (s, dt) in enumerate(beams):
        p = dd.Plan.from_setup(s, dt)
        d = oracle_table(s)
        x, _ = make_input(s, dt, seed + k, p.n_in, p.padded_in_stride(), pulses=1, d=d)
        plans.append(p)
        hosts.append(x)
        xs.append(torch.from_numpy(x).cuda())
    return plans, xs, hosts


def test_batch_equals_solo_forward(dd):
    beams = _small_batch()
    plans, xs, hosts = _inputs(dd, beams, 10)
    batch = dd.Batch(plans)
    outs = [torch.full((p.n_dm, p.n_out), -1, dtype=p.out_dtype, device="cuda") for p in plans]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.run(xs, outs, stream=stream)       # capture + launch
        batch.run(xs, outs, stream=stream)       # graph replay
    stream.synchronize()
    assert plans[0].device_status() == 0
    for (s, dt), p, x, h, o in zip(beams, plans, xs, hosts, outs):
        solo = p.forward(x)
        assert torch.equal(o, solo), s.name
        ref, scale = oracle_window(oracle_table(s), h, dt, 0, s.n_dm, 0, s.n_out)
        assert_parity(o.cpu().numpy(), ref, scale, dt, where=f"batch {s.name}")
    # a new pointer set is picked up (re-capture)
    outs2 = [torch.zeros_like(o) for o in outs]
    with torch.cuda.stream(stream):
        batch.run(xs, outs2, stream=stream)
    stream.synchronize()
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o, o2)
    batch.close()


def test_batch_tune_once_per_setup(dd, tmp_path):
    """dd_batch_tune runs dd_tune once per distinct setup (here two beams
    share each of three setups); beams of one setup take one configuration,
    the tuned batch still equals solo launches and the oracle, and the
    database then holds one record per setup."""
    base = _small_batch(3)[:3]
    beams = base + base            # every setup twice
    plans, xs, hosts = _inputs(dd, beams, 20)
    batch = dd.Batch(plans)
    db = str(tmp_path / "batch.jsonl")
    assert batch.tune(budget_s=0.0, db_path=db) == 3
    for k in range(3):
        assert plans[k].selected == plans[k + 3].selected
    with open(db) as f:
        assert len([json.loads(line) for line in f]) == 3
    outs = [torch.empty((p.n_dm, p.n_out), dtype=p.out_dtype, device="cuda") for p in plans]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.run(xs, outs, stream=stream)
    stream.synchronize()
    for (s, dt), p, x, h, o in zip(beams, plans, xs, hosts, outs):
        assert p.device_status() == 0
        assert torch.equal(o, p.forward(x)), s.name
        ref, scale = oracle_window(oracle_table(s), h, dt, 0, s.n_dm, 0, s.n_out)
        assert_parity(o.cpu().numpy(), ref, scale, dt, where=f"tuned batch {s.name}")
    batch.close()


def test_persistent_groups_with_mixed_beams(dd):
    """Persistent launches: several beams share each configuration (staged
    float on LOFAR-grid beams of different trial spreads, so different staged
    pitches; packed uint8; the 9-trial Tensor-Memory kernel), so one launch
    runs the tiles of beams of different sizes back to back in the same
    blocks.  The batch equals solo launches bit for bit, equals the oracle,
    and equals the one-launch-per-beam batch; a second run replays the graph."""
    rng = np.random.default_rng(5)
    beams, force = [], []
    for b in range(5):                      # LOFAR grid, float, one staged shape
        C = int(rng.choice([32, 64]))
        s = synth.Setup(f"st{b}", C, 138.0, 6.25 / C, 5e-6, 0.0, 0.01 * (b + 1), int(rng.choice([24, 40, 64])),
                        int(rng.integers(2500, 7000)))
        beams.append((s, "f32"))
        force.append("staged_d8_t1024_c4_s3")
    for b in range(4):                      # Apertif grid, uint8, one packed shape
        C = int(rng.choice([64, 256]))
        s = synth.Setup(f"u{b}", C, 1420.0, 300.0 / C, 50e-6, 0.0, 0.25, int(rng.choice([16, 48])),
                        int(rng.integers(2000, 9000)))
        beams.append((s, "u8"))
        force.append("u8pk_w8x1_d2_c32_st3")
    for b in range(3):                      # Apertif grid, float, the Tensor-Memory kernel
        C = int(rng.choice([64, 256]))
        s = synth.Setup(f"t{b}", C, 1420.0, 300.0 / C, 50e-6, 0.0, 0.25, int(rng.choice([18, 45])),
                        int(rng.integers(3000, 9000)))
        beams.append((s, "f32"))
        force.append("tmw9_f32_d9_t4096")
    plans, xs, hosts = _inputs(dd, beams, 40)
    for p, name in zip(plans, force):
        assert name in p.configs(), (p, name)
        p.select(name)
    batch = dd.Batch(plans)
    batch.set_persistent(2)                      # every group persistent, whatever its kind
    outs = [torch.full((p.n_dm, p.n_out), -1, dtype=p.out_dtype, device="cuda") for p in plans]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.run(xs, outs, stream=stream)       # upload, capture, launch
        batch.run(xs, outs, stream=stream)       # replay
    stream.synchronize()
    for (s, dt), p, x, h, o in zip(beams, plans, xs, hosts, outs):
        assert p.device_status() == 0, s.name
        assert torch.equal(o, p.forward(x)), s.name
        ref, scale = oracle_window(oracle_table(s), h, dt, 0, s.n_dm, 0, s.n_out)
        assert_parity(o.cpu().numpy(), ref, scale, dt, where=f"persistent batch {s.name}")
    for mode in (0, 1):                          # one launch per beam; untuned automatic choice
        batch.set_persistent(mode)
        outs2 = [torch.full_like(o, -1) for o in outs]
        with torch.cuda.stream(stream):
            batch.run(xs, outs2, stream=stream)
        stream.synchronize()
        assert all(torch.equal(o, o2) for o, o2 in zip(outs, outs2)), mode
    # tuning times each persistent group against its beams' own launches and
    # keeps the faster form; results stay the same
    batch.tune(budget_s=0.0)
    outs3 = [torch.full_like(o, -1) for o in outs]
    with torch.cuda.stream(stream):
        batch.run(xs, outs3, stream=stream)
    stream.synchronize()
    for p, x, o in zip(plans, xs, outs3):
        assert torch.equal(o, p.forward(x))
    batch.close()


def test_batch_rejects_unaligned(dd):
    s = synth.Setup("una", 32, 1420.0, 2.0, 50e-6, 0.0, 0.25, 16, 1000)
    p = dd.Plan.from_setup(s, "f32")
    x = torch.zeros((s.channels, p.padded_in_stride() + 1), device="cuda")[:, 1:]
    o = torch.zeros((s.n_dm, s.n_out), device="cuda")
    with pytest.raises(dd.DDError) as e:
        dd.Batch([p]).run([x], [o])
    assert e.value.name == "DD_ERR_ALIGN"


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_stream_chunks_equal_one_forward(dd, dtype):
    """Concatenated streamed outputs (t >= 0) equal dd_forward on the whole input."""
    s = synth.Setup("stream", 128, 1420.0, 2.34375, 50e-6, 0.0, 0.25, 48, 5000)
    N, K = 1250, 6
    plan = dd.Plan(s.channels, s.f_low_mhz, s.chan_bw_mhz, s.t_samp_s, s.dm_first, s.dm_step, s.n_dm, N, dtype)
    md = plan.max_delay
    total = N * K
    x, _ = make_input(s, dtype, 3, total, total)
    st = dd.Stream(plan, N)
    got = []
    for k in range(K):
        out, t0 = st.push(torch.from_numpy(np.ascontiguousarray(x[:, k * N:(k + 1) * N])).cuda())
        assert t0 == k * N - md
        got.append((t0, out.cpu().numpy()))
        if k == 2:
            saved = st.save()
    whole = np.concatenate([o for _, o in got], axis=1)[:, md:]          # times 0 .. total - md
    n_valid = total - md
    big = dd.Plan(s.channels, s.f_low_mhz, s.chan_bw_mhz, s.t_samp_s, s.dm_first, s.dm_step, s.n_dm, n_valid, dtype)
    ref_dev = big.forward(torch.from_numpy(
        np.ascontiguousarray(np.pad(x, ((0, 0), (0, big.padded_in_stride() - total))))).cuda()).cpu().numpy()
    assert (whole[:, :n_valid] == ref_dev).all()
    d = oracle_table(s)
    ref, scale = oracle_window(d, x, dtype, 0, s.n_dm, 0, n_valid)
    assert_parity(whole[:, :n_valid], ref, scale, dtype, where="stream vs oracle")
    # restore the state saved after chunk 2 and replay chunks 3.. identically
    st.restore(saved)
    for k in range(3, K):
        out, t0 = st.push(torch.from_numpy(np.ascontiguousarray(x[:, k * N:(k + 1) * N])).cuda())
        assert t0 == got[k][0] and (out.cpu().numpy() == got[k][1]).all()
    st.reset()
    out, t0 = st.push(torch.from_numpy(np.ascontiguousarray(x[:, :N])).cuda())
    assert t0 == -md and (out.cpu().numpy() == got[0][1]).all()


def test_tune_selects_and_records(dd, tmp_path):
    s = synth.Setup("tune", 256, 1420.0, 1.171875, 50e-6, 0.0, 0.25, 128, 6000)
    plan = dd.Plan.from_setup(s, "f32")
    db = str(tmp_path / "tune.jsonl")
    name, ms = plan.tune(budget_s=30.0, db_path=db)
    assert name in plan.configs() and ms > 0
    with open(db) as f:
        rec = json.loads(f.readline())
    assert rec["config"] == name and len(rec["timings"]) >= 3
    plan2 = dd.Plan.from_setup(s, "f32")
    name2, ms2 = plan2.tune(db_path=db)       # database hit: no timing
    assert name2 == name and abs(ms2 - rec["ms"]) < 1e-6
    import os
    os.environ["DD_TUNE_DB"] = db                 # plans made now start with the recorded choice
    try:
        assert dd.Plan.from_setup(s, "f32").selected == name
    finally:
        del os.environ["DD_TUNE_DB"]
    x = plan.alloc_input()
    x.normal_()
    assert torch.equal(plan.forward(x), plan2.forward(x))


def test_serving_mix_equals_alone_and_respects_budget(dd):
    from paper_1601_01165_gb300.serve import BeamSpec, Server, beam_bytes
    specs = []
    for b in range(5):
        C = 128 if b % 2 else 64
        s = synth.Setup(f"s{b}", C, 1420.0, 300.0 / C, 50e-6, 0.0, 0.25, 48, 0)
        specs.append(BeamSpec(f"beam{b}", s, "u8" if b % 2 else "f32", chunk_len=2000, n_chunks=4,
                              period_s=0.03, phase_s=0.007 * b, keep_output=True))
    need = [beam_bytes(sp) for sp in specs]
    budget = sum(sorted(need)[-3:]) + 1      # room for three beams at a time

    def source(sp, k):
        seed = 1000 * int(sp.name[4:]) + k
        if sp.dtype == "u8":
            return synth.noise_u8(seed, sp.setup.channels, sp.chunk_len)
        return synth.noise_f32(seed, sp.setup.channels, sp.chunk_len)

    rep = Server(budget).run(specs, source)
    assert rep["chunks"] == 5 * 4
    assert rep["peak_bytes"] <= budget and rep["peak_beams"] <= 3
    assert max(rep["admitted_at"].values()) > min(rep["admitted_at"].values())   # someone waited
    assert rep["latency_p99_s"] is not None
    for sp in specs:
        s = sp.setup
        plan = dd.Plan(s.channels, s.f_low_mhz, s.chan_bw_mhz, s.t_samp_s, s.dm_first, s.dm_step, s.n_dm,
                       sp.chunk_len, sp.dtype)
        alone = dd.Stream(plan, sp.chunk_len)
        mix = rep["outputs"][sp.name]
        assert len(mix) == sp.n_chunks
        for k in range(sp.n_chunks):
            out, t0 = alone.push(torch.from_numpy(source(sp, k)).cuda())
            assert t0 == mix[k][0]
            assert (out.cpu().numpy() == mix[k][1].numpy()).all(), (sp.name, k)
