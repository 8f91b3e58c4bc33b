"""GPU parity of the colouring check and of keeping a colouring across MD steps.

css_color_check counts the same-coloured molecule pairs closer than R_col on a geometry
(integer work: bit-exact against the oracle's brute force); css_color_update keeps a
colouring while that count is zero and otherwise recolours at R_col + skin, which must give
exactly the oracle's fresh colouring.
"""
import numpy as np
import pytest

import oracle
from paper_2605_20918_gb300 import synth

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


@pytest.fixture(scope="module")
def ctx(css):
    c = css.Context(0)
    yield c
    c.close()


def _dev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


# one cell (box < 3 R_col), several cells per edge, the 10,000-molecule workload
@pytest.mark.parametrize("n,r_col,sigma,seed", [(1, 8.0, 0.0, 0), (64, 8.0, 0.5, 3001), (216, 8.0, 0.3, 3002),
                                                (1000, 10.0, 0.3, 3003), (4096, 10.0, 0.1, 3004),
                                                (10000, 10.0, 0.05, 3005)])
def test_check_counts_bit_exact(torch, ctx, n, r_col, sigma, seed):
    g0 = synth.water_box(n)
    col, nc = oracle.color(g0.pos, g0.box, r_col, 1004)
    g = synth.perturb(g0, seed, sigma=sigma) if sigma else g0
    xyz = _dev(torch, g.pos, torch.float64)
    c = _dev(torch, col, torch.int32)
    got = ctx.color_check(xyz, g.box, r_col, c, nc)
    assert got == oracle.color_conflicts(g.pos, g.box, r_col, col)
    assert ctx.color_check(_dev(torch, g0.pos, torch.float64), g0.box, r_col, c, nc) == 0
    # one colour for all: every edge of the colour graph is a conflict
    ptr, _ = oracle.neighbours(g.pos, g.box, r_col)
    one = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert ctx.color_check(xyz, g.box, r_col, one, 1) == int(ptr[-1]) // 2
    # R_col = 0: no pair is closer than 0
    assert ctx.color_check(xyz, g.box, 0.0, one, 1) == 0


def test_check_along_the_md_sequence(torch, ctx):
    """The 10,000-molecule, 23-orbital workload's MD-like sequence (0.02 A steps): conflicts of
    the first geometry's colouring at R_col = 10 A on each later geometry."""
    seq = list(synth.md_sequence(10000, 8))
    col, nc = oracle.color(seq[0].pos, seq[0].box, 10.0, 1004)
    c = _dev(torch, col, torch.int32)
    got = [ctx.color_check(_dev(torch, g.pos, torch.float64), g.box, 10.0, c, nc) for g in seq]
    want = [oracle.color_conflicts(g.pos, g.box, 10.0, col) for g in seq]
    assert got == want and got[0] == 0


@pytest.mark.parametrize("skin", [0.0, 0.3])
def test_update_keeps_or_recolours_like_the_oracle(torch, ctx, skin):
    seq = list(synth.md_sequence(1000, 6))
    r_col = 8.0
    col = torch.zeros(1000, dtype=torch.int32, device="cuda")
    ref, nref = np.zeros(1000, np.int32), 0
    nc = 0
    decisions = []
    for g in seq:
        xyz = _dev(torch, g.pos, torch.float64)
        nc, re = ctx.color_update(xyz, g.box, r_col, 1004, col, nc, skin=skin)
        ref, nref, re_ref = oracle.color_update(g.pos, g.box, r_col, 1004, ref, nref, skin=skin)
        assert re == re_ref and nc == nref
        assert np.array_equal(col.cpu().numpy(), ref)
        decisions.append(re)
    assert decisions[0]  # the first step has no colouring to keep
    if skin > 0:
        assert not any(decisions[1:])  # 0.3 A of room outlasts five 0.02 A steps here


def test_update_recolours_out_of_range_colours(torch, ctx):
    g = synth.water_box(216)
    xyz = _dev(torch, g.pos, torch.float64)
    fresh, nf = oracle.color(g.pos, g.box, 8.0, 1004)
    bad = _dev(torch, fresh - 1, torch.int32)  # -1 is out of range
    nc, re = ctx.color_update(xyz, g.box, 8.0, 1004, bad, nf)
    assert re and nc == nf and np.array_equal(bad.cpu().numpy(), fresh)


def test_check_rejects_bad_arguments(torch, css, ctx):
    g = synth.water_box(64)
    xyz = _dev(torch, g.pos, torch.float64)
    col = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(css.CSSError) as e:
        ctx.color_check(xyz, g.box, 8.0, col, 0)
    assert e.value.status == css.CSS_ERR_INVALID_ARG
    col[5] = 3
    with pytest.raises(css.CSSError) as e:
        ctx.color_check(xyz, g.box, 8.0, col, 2)  # colour 3 outside [0, 2)
    assert e.value.status == css.CSS_ERR_INVALID_ARG
    with pytest.raises(css.CSSError):
        ctx.color_update(xyz, g.box, 8.0, 1004, col, 4, skin=-1.0)
    # the context stays usable after the errors
    assert ctx.color_check(xyz, g.box, 8.0, torch.arange(64, dtype=torch.int32, device="cuda"), 64) == 0
