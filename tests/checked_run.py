"""Runs every forward configuration of a set of small and ragged setups through
the library named by DD_LIBRARY (the checked build, whose kernels record any
out-of-range index in the plan's status word instead of making the access) and
compares with the oracle.  Exits nonzero on the first problem.  Started by
tests/test_checked_gpu.py in a process of its own."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_1601_01165_gb300 import binding as dd, synth  # noqa: E402
from helpers import assert_parity, make_input, oracle_table, oracle_window  # noqa: E402

SETUPS = [
    synth.TINY,
    synth.Setup("ragged-a", 37, 1420.0, 0.29296875 * 1024 / 37, 50e-6, 0.0, 0.25, 3, 1001),
    synth.Setup("ragged-c", 130, 1420.0, 2.0, 50e-6, 0.0, 0.5, 45, 2999),
    synth.Setup("lofar-cut", 32, 138.0, 0.1953125, 5e-6, 0.0, 0.01, 70, 3001),
    synth.Setup("apertif-cut", 1024, 1420.0, 0.29296875, 50e-6, 3.0, 0.25, 41, 4500),
    synth.Setup("edge-c7", 7, 1420.0, 300.0 / 7, 50e-6, 1.0, 0.25, 13, 8200),
]


def main():
    lib = dd.load()
    assert "checked" in os.environ.get("DD_LIBRARY", ""), "run with DD_LIBRARY naming the checked build"
    runs = 0
    for s in SETUPS:
        d = oracle_table(s)
        for dtype, weighted in (("f32", False), ("f32", True), ("u8", False)):
            plan = dd.Plan.from_setup(s, dtype)
            x, _ = make_input(s, dtype, 3, plan.n_in, plan.padded_in_stride())
            xt = torch.from_numpy(x).cuda()
            w = synth.weights(3, s.channels) if weighted else None
            wt = torch.from_numpy(w).cuda() if w is not None else None
            ref, scale = oracle_window(d, x, dtype, 0, s.n_dm, 0, s.n_out, w)
            for cfg in plan.configs():
                plan.select(cfg)
                out = plan.forward(xt, wt)
                torch.cuda.synchronize()
                code = plan.device_status()
                if code != 0:
                    print(f"{s.name} {dtype} w={weighted} {cfg}: device status {code}")
                    return 1
                assert_parity(out.cpu().numpy(), ref, scale, dtype, where=f"checked {s.name} {dtype} {cfg}")
                runs += 1
    print(f"checked build: {runs} launches in range and equal to the oracle")
    return 0 if lib is not None else 1


if __name__ == "__main__":
    sys.exit(main())
