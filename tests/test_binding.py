"""Argument checks of the Python binding, on the CPU: a buffer of the wrong size is refused
before any pointer reaches the library (the C-ABI takes raw pointers and cannot check
lengths), and correctly sized host tensors are still refused as not being CUDA tensors."""
import numpy as np
import pytest

import paper_2605_20918_gb300 as css
from paper_2605_20918_gb300 import synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sys64():
    g = synth.water_box(64)
    H = synth.hamiltonian(g, "minimal")
    return g, H, css.DeviceBSR.from_host(H, device="cpu")


def _i32(n):
    return torch.zeros(n, dtype=torch.int32)


def test_from_host_checks_the_pattern(sys64):
    _, H, _ = sys64
    bad_ptr = synth.BSR(H.n_brow, H.b, H.row_ptr.copy(), H.col_idx, H.val)
    bad_ptr.row_ptr[5], bad_ptr.row_ptr[6] = bad_ptr.row_ptr[6], bad_ptr.row_ptr[5] - 1
    with pytest.raises(ValueError, match="row_ptr"):
        css.DeviceBSR.from_host(bad_ptr, device="cpu")
    short = synth.BSR(H.n_brow, H.b, H.row_ptr, H.col_idx[:-1], H.val[:-1])
    with pytest.raises(ValueError, match="row_ptr"):
        css.DeviceBSR.from_host(short, device="cpu")
    col = H.col_idx.copy()
    col[3] = H.n_brow
    with pytest.raises(ValueError, match="col_idx"):
        css.DeviceBSR.from_host(synth.BSR(H.n_brow, H.b, H.row_ptr, col, H.val), device="cpu")
    with pytest.raises(ValueError, match="val"):
        css.DeviceBSR.from_host(synth.BSR(H.n_brow, H.b, H.row_ptr, H.col_idx, H.val[:, :, :-1]), device="cpu")


def test_density_refuses_wrong_sizes(sys64):
    _, H, Hd = sys64
    n, b = H.n_brow, H.b
    col, sign = _i32(n), torch.ones(n * b, dtype=torch.int8)
    P = torch.zeros((H.nnzb, b, b), dtype=torch.float64)
    with pytest.raises(ValueError, match="P has"):
        css.css_density(None, Hd, col, sign, 4, P[:-1])
    with pytest.raises(ValueError, match="colour has"):
        css.css_density(None, Hd, _i32(n - 1), sign, 4, P)
    with pytest.raises(ValueError, match="sign has"):
        css.css_density(None, Hd, col, sign[:-1], 4, P)
    with pytest.raises(TypeError, match="CUDA tensor"):
        css.css_density(None, Hd, col, sign, 4, P)
    with pytest.raises(ValueError, match="P has"):
        css.css_density_batch(None, [Hd], [col], [sign], [4], [P[:-1]], [{}])
    with pytest.raises(ValueError, match="one colour"):
        css.css_density_batch(None, [Hd, Hd], [col], [sign], [4], [P], [{}])


def test_colouring_and_probes_refuse_wrong_sizes(sys64):
    g, H, _ = sys64
    xyz = torch.as_tensor(g.pos)
    with pytest.raises(ValueError, match="colour has"):
        css.css_color(None, xyz, g.box, 8.0, 1004, _i32(63))
    with pytest.raises(ValueError, match="xyz has"):
        css.css_color(None, xyz.reshape(-1)[:-3].reshape(-1, 3)[:, :2].contiguous(), g.box, 8.0, 1004, _i32(63))
    with pytest.raises(ValueError, match="colour has"):
        css.css_color_check(None, xyz, g.box, 8.0, _i32(65), 3)
    with pytest.raises(ValueError, match="colour has"):
        css.css_color_update(None, xyz, g.box, 8.0, 1004, _i32(65), 3)
    with pytest.raises(ValueError, match="sign has"):
        css.css_probes(None, _i32(64), H.b, 1005, torch.ones(64 * H.b + 1, dtype=torch.int8))
    with pytest.raises(ValueError, match="colour has"):
        css.css_color_graph(None, _i32(65), _i32(0), 1004, _i32(63))
    with pytest.raises(TypeError, match="CUDA tensor"):
        css.css_color(None, xyz, g.box, 8.0, 1004, _i32(64))


def test_hprime_pbuild_eigen_refuse_wrong_sizes(sys64):
    g, H, Hd = sys64
    n, b = H.n_brow, H.b
    col, sign = _i32(n), torch.ones(n * b, dtype=torch.int8)
    P = torch.zeros((H.nnzb, b, b), dtype=torch.float64)
    with pytest.raises(ValueError, match="Hp has"):
        css.css_hprime(None, Hd, Hd, col, sign, 4, P, P[:-1])
    with pytest.raises(ValueError, match="P has"):
        css.css_pbuild(None, g.pos, g.box, H, np.zeros(5), r_col=8.0, flags=css.CSS_HOST_IO)
    with pytest.raises(TypeError, match="C-contiguous"):
        css.css_pbuild(None, g.pos, g.box, H, np.zeros((b, b, H.nnzb)).transpose(2, 0, 1), r_col=8.0,
                       flags=css.CSS_HOST_IO)
    with pytest.raises(ValueError, match="colour_out has"):
        css.css_pbuild(None, g.pos, g.box, H, np.zeros((H.nnzb, b, b)), r_col=8.0, flags=css.CSS_HOST_IO,
                       colour_out=np.zeros(3, np.int32))
    A = torch.zeros((3, 4, b, b), dtype=torch.float64)
    with pytest.raises(ValueError, match="nblk has"):
        css.css_eigen_blocks(None, A, A, _i32(2), _i32(3))


def test_density_nonorth_refuses_wrong_sizes(sys64):
    _, H, Hd = sys64
    n, b = H.n_brow, H.b
    col, sign = _i32(n), torch.ones(n * b, dtype=torch.int8)
    P = torch.zeros((H.nnzb, b, b), dtype=torch.float64)
    with pytest.raises(ValueError, match="Sinv has"):
        css.css_density_nonorth(None, Hd, P[:-1], Hd, P, col, sign, 4, P)
    with pytest.raises(ValueError, match="H_val has"):
        css.css_density_nonorth(None, Hd, P, Hd, P[:-1], col, sign, 4, P)
    with pytest.raises(ValueError, match="P has"):
        css.css_density_nonorth(None, Hd, P, Hd, P, col, sign, 4, P[:-1])
    with pytest.raises(TypeError, match="CUDA tensor"):
        css.css_density_nonorth(None, Hd, P, Hd, P, col, sign, 4, P)
