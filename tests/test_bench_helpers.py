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
