"""Host logic of bench.py's measurement helpers, driven by a stand-in context on the CPU."""
import numpy as np

import bench
from paper_2605_20918_gb300 import synth


class _OracleColouring:
    """Implements color_update through the oracle on host arrays (numpy in place of device
    tensors)."""

    def __init__(self, oracle):
        self.o = oracle
        self.calls = 0

    def color_update(self, xyz, box, r_col, seed, colour, n_colours, *, skin=0.0):
        self.calls += 1
        col, nc, re = self.o.color_update(xyz, box, r_col, seed, colour, n_colours, skin=skin)
        colour[:] = col
        return nc, re


def test_colour_reuse_counts_recolourings(oracle_lib):
    seq = list(synth.md_sequence(400, 5))
    ctx = _OracleColouring(oracle_lib)
    colour = np.zeros(400, np.int32)
    out = bench.colour_reuse(ctx, [g.pos for g in seq], seq[0].box, 8.0, colour, skins=(0.0, 0.3))
    assert ctx.calls == 10
    tight, loose = out["skin_0_A"], out["skin_0.3_A"]
    # without a skin every 0.02 A step breaks the colouring; 0.3 A outlasts the sequence
    assert tight["recoloured"] == 5 and tight["ms_keep"] is None and tight["ms_recolour"] is not None
    assert loose["recoloured"] == 1 and loose["ms_keep"] is not None and loose["ms_recolour"] is None
    assert loose["n_colours"] == oracle_lib.color(seq[0].pos, seq[0].box, 8.3, 1004)[1]
    assert tight["n_colours"] == oracle_lib.color(seq[-1].pos, seq[-1].box, 8.0, 1004)[1]
    assert np.array_equal(colour, oracle_lib.color(seq[0].pos, seq[0].box, 8.3, 1004)[0])


def _run_bench(args, env_extra=None, timeout=600):
    import json
    import os
    import subprocess
    import sys
    from pathlib import Path
    root = Path(__file__).resolve().parents[1]
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run([sys.executable, str(root / "bench.py"), *args], cwd=root, env=env, capture_output=True,
                       text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_prints_the_contract_line(oracle_lib):
    """The oracle arm (bench.py --impl reference) on a small case: one JSON line with the
    contract's keys, the same metric as the GPU arm and a CPU-baseline description."""
    (line,) = _run_bench(["--impl", "reference", "--n-mol", "300", "--m", "4", "--steps", "2", "--warmup", "1"])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["higher_is_better"] is False and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and abs(line["ms_per_step"] - 1e3 * line["value"]) < 1e-9 * line["ms_per_step"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["n_mol"] == 300 and "workload" in line["config"]


def test_reference_arm_other_ranks_exit_quietly():
    assert _run_bench(["--impl", "reference", "--n-mol", "300", "--m", "4", "--steps", "1", "--warmup", "0"],
                      env_extra={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
