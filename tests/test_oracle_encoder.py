"""Pins of the encoder oracle: torch's float64 CPU convolution (an independent library
routine) for the forward, central finite differences for the backward, and the anchor
geometry of the decode (decoding zeros puts every Gaussian at its slot centre)."""
import numpy as np
import pytest

from oracle import encoder_ref as er


@pytest.mark.parametrize("stride", [1, 2])
def test_conv_forward_matches_torch(stride):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(stride)
    x = rng.standard_normal((2, 3, 9, 11))
    w = rng.standard_normal((5, 3, 3, 3))
    b = rng.standard_normal(5)
    for relu in (False, True):
        y = er.conv3x3_fwd(x, w, b, stride, relu)
        t = torch.nn.functional.conv2d(torch.tensor(x), torch.tensor(w), torch.tensor(b),
                                       stride=stride, padding=1)
        if relu:
            t = torch.relu(t)
        assert np.abs(y - t.numpy()).max() < 1e-12


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((2, 3, 7, 8))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    dy = rng.standard_normal((2, 4, 4, 4))

    def loss(x_, w_, b_):
        return float(np.sum(dy * er.conv3x3_fwd(x_, w_, b_, 2, True)))

    y = er.conv3x3_fwd(x, w, b, 2, True)
    dx, dw, db = er.conv3x3_bwd(x, w, y, dy, 2, True)
    h = 1e-6
    for arr, grad, which in ((x, dx, 0), (w, dw, 1), (b, db, 2)):
        for flat in range(0, arr.size, max(1, arr.size // 9)):
            idx = np.unravel_index(flat, arr.shape)
            args = [x.copy(), w.copy(), b.copy()]
            args[which][idx] += h
            lp = loss(*args)
            args[which][idx] -= 2 * h
            lm = loss(*args)
            assert abs((lp - lm) / (2 * h) - grad[idx]) < 1e-6 * max(1.0, abs(grad[idx]))


def test_decode_zero_output_is_the_anchor_grid():
    S, C, H, W = 16, 3, 64, 96
    out = np.zeros((1, S * (6 + 2 * C), 4, 6))
    p = er.decode(out, S, C, H, W)[0]
    x = (np.tanh(p["xy_raw"][:, 0]) + 1) / 2 * W
    y = (np.tanh(p["xy_raw"][:, 1]) + 1) / 2 * H
    # 4 x 6 cells of 16 x 16 pixels, 4 x 4 slots each: slot centres at 2, 6, 10, 14 px
    assert np.allclose(np.sort(np.unique(np.round(x % 16, 6))), [2, 6, 10, 14], atol=1e-4)
    assert np.allclose(np.sort(np.unique(np.round(y % 16, 6))), [2, 6, 10, 14], atol=1e-4)
    assert len(x) == 4 * 6 * 16
    assert np.allclose(np.exp(p["s_raw"]) + 0.1, 1.6)
    assert np.all(p["phase"] == 0) and np.allclose(p["amp"], 0.5) and np.allclose(p["alpha_raw"], -0.5)


def test_decode_bwd_is_the_adjoint():
    """<decode(out + e) - decode(out), g> = <e, decode_bwd(g)> for random out, e, g: the decode
    is affine, so the identity is exact up to rounding for any step e."""
    S, C, H, W, CY, CX = 9, 2, 40, 48, 2, 3
    rng = np.random.default_rng(11)
    out = rng.standard_normal((2, S * (6 + 2 * C), CY, CX))
    e = rng.standard_normal(out.shape)
    p0, p1 = er.decode(out, S, C, H, W), er.decode(out + e, S, C, H, W)
    g = [{k: rng.standard_normal(np.shape(v)) for k, v in d.items()} for d in p0]
    lhs = sum(float(np.sum((p1[b][k] - p0[b][k]) * g[b][k])) for b in range(2) for k in g[b])
    rhs = float(np.sum(e * er.decode_bwd(g, S, C, CY, CX)))
    assert abs(lhs - rhs) < 1e-9 * max(1.0, abs(lhs))
