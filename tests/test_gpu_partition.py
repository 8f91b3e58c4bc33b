"""Colour-partitioned build through the library on one GPU (paper: each colour's probe block is an
independent right-hand side, paragraph after Eq. 4).

The colours are dealt to two "ranks" with shard.colour_partition; the two disjoint subsets run
one after the other through css_density_colours, first with CSS_RITZ_ONLY (Ritz lists of the
owned colours), then, after css_solve_mu on the gathered lists, with that mu (each rank's
unsymmetrised columns).  The Ritz lists, mu and the sum of the two parts must equal one
css_density call over all colours bit for bit, in FP64 and in mixed precision.
"""
import numpy as np
import pytest

import oracle
from paper_2605_20918_gb300 import shard, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def css(torch):
    import paper_2605_20918_gb300 as m
    from paper_2605_20918_gb300 import build
    build.build()
    oracle.build()
    return m


@pytest.mark.parametrize("n,kind,r_col,m,prec", [(125, "dzp", 8.0, 10, "fp64"), (216, "minimal", 8.0, 12, "mixed"),
                                                 (125, "dzp", 8.0, 10, "mixed")])
def test_two_rank_colour_partition_equals_one_call(torch, css, n, kind, r_col, m, prec):
    g = synth.water_box(n)
    H = synth.hamiltonian(g, kind)
    col, nc = oracle.color(g.pos, g.box, r_col, 1004)
    sign = oracle.probes(col, H.b, 1005)
    ne = synth.n_electrons(n)
    p = css.CSS_FP64 if prec == "fp64" else css.CSS_MIXED_FP32
    dev = "cuda"
    Hd = css.DeviceBSR.from_host(H, dev)
    dc, ds = torch.as_tensor(col, device=dev), torch.as_tensor(sign, device=dev)
    with css.Context(0) as ctx:
        P1 = torch.zeros((H.nnzb, H.b, H.b), dtype=torch.float64, device=dev)
        r1 = ctx.density(Hd, dc, ds, nc, P1, kT=0.05, n_elec=ne, m=m, precision=p, flags=0)
        ritz1 = ctx.ritz()
        parts = shard.colour_partition(np.bincount(col, minlength=nc), 2)
        assert sorted(sum(parts, [])) == list(range(nc))
        # phase 1: Ritz lists of each rank's colours, put back in colour order
        lists = [None] * nc
        for owned in parts:
            mask = np.zeros(nc, np.uint8)
            mask[owned] = 1
            scratch = torch.zeros_like(P1)
            ctx.density_colours(Hd, dc, ds, nc, mask, scratch, mu=0.0, m=m, precision=p, flags=css.CSS_RITZ_ONLY)
            assert float(scratch.abs().max().item()) == 0.0  # nothing extracted in this phase
            for c, lw in zip(owned, ctx.ritz()):
                lists[c] = lw
        for c in range(nc):
            assert np.array_equal(lists[c][0], ritz1[c][0]) and np.array_equal(lists[c][1], ritz1[c][1]), c
        # the one exchange: mu from the gathered lists, by the library
        mu = ctx.solve_mu(lists, kT=0.05, n_elec=ne)
        assert mu == r1["mu"]
        # phase 2: each rank's columns at that mu; the parts are disjoint and add up to one call
        total = torch.zeros_like(P1)
        trp = trph = 0.0
        for owned in parts:
            mask = np.zeros(nc, np.uint8)
            mask[owned] = 1
            Pr = torch.full_like(P1, float("nan"))
            rr = ctx.density_colours(Hd, dc, ds, nc, mask, Pr, mu=mu, m=m, precision=p)
            own_blocks = torch.as_tensor(np.isin(col[H.col_idx], owned), device=dev)
            assert float(Pr[~own_blocks].abs().max().item()) == 0.0
            total += Pr
            trp += rr["trP"]
            trph += rr["trPH"]
        torch.cuda.synchronize()
        assert torch.equal(total, P1)
        assert abs(trp - r1["trP"]) <= 1e-12 * max(1.0, abs(r1["trP"]))
        assert abs(trph - r1["trPH"]) <= 1e-12 * max(1.0, abs(r1["trPH"]))


def test_partition_arguments_are_checked(torch, css):
    g = synth.water_box(27)
    H = synth.hamiltonian(g)
    col, nc = oracle.color(g.pos, g.box, 5.0, 1004)
    sign = oracle.probes(col, H.b, 1005)
    Hd = css.DeviceBSR.from_host(H)
    dc, ds = torch.as_tensor(col, device="cuda"), torch.as_tensor(sign, device="cuda")
    P = torch.zeros((H.nnzb, H.b, H.b), dtype=torch.float64, device="cuda")
    with css.Context(0) as ctx:
        with pytest.raises(css.CSSError):  # symmetrisation needs every colour
            ctx.density_colours(Hd, dc, ds, nc, np.ones(nc, np.uint8), P, mu=-4.0, m=4, flags=css.CSS_SYMMETRIZE)
        with pytest.raises(css.CSSError):  # nothing owned
            ctx.density_colours(Hd, dc, ds, nc, np.zeros(nc, np.uint8), P, mu=-4.0, m=4)
        with pytest.raises(ValueError):  # one flag per colour
            ctx.density_colours(Hd, dc, ds, nc, np.ones(nc + 1, np.uint8), P, mu=-4.0, m=4)
