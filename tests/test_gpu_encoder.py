"""GPU parity of the learned initialiser's kernels against the FP64 encoder oracle.

Inputs and weights are rounded to BF16 on the host first (the kernels' storage precision),
so the oracle sees the very values the kernels read.  What is left is the FP32
accumulation (rel. L2 1e-5 for FP32 outputs and gradients) and, for BF16 outputs, one
round-to-nearest-even of the result (at most 2^-8 relative per element).  The chain test
feeds the oracle's own activations, rounded to BF16 like the kernels store them, through
the oracle's step and convolution backward and compares every layer's weight gradient
within the hologram gradient tolerance (1e-3).
"""
import numpy as np
import pytest

import oracle
from oracle import encoder_ref as er
from paper_2511_15022_gb300 import inputs
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def bf16_round(a: np.ndarray) -> np.ndarray:
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def to_bf16(a: np.ndarray, dev):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(dev)


CONV_CASES = [  # B, CI, H, W, CO, stride
    (2, 5, 37, 29, 11, 1),
    (2, 5, 37, 29, 11, 2),
    (1, 3, 130, 66, 32, 2),     # first layer, ragged tail of the 128-pixel CTAs
    (2, 128, 32, 32, 192, 2),   # last layer of the 512 x 512 encoder at 32 x 32 input
    (1, 1, 1, 1, 1, 2),         # one pixel
    (1, 24, 20, 22, 72, 2),     # partial last channel chunk (24 = 16 + 8), partial 64-channel block
    (2, 16, 18, 34, 64, 1),     # stride 1, exactly one chunk and one block
]


@pytest.mark.parametrize("case", CONV_CASES)
@pytest.mark.parametrize("relu", [False, True])
def test_conv_fwd(case, relu, dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    B, CI, H, W, CO, s = case
    rng = np.random.default_rng(hash(case) % 1000)
    x = bf16_round(rng.standard_normal((B, CI, H, W)))
    w = bf16_round(rng.standard_normal((CO, CI, 3, 3)) / np.sqrt(9 * CI))
    b = rng.standard_normal(CO).astype(np.float32)
    ref = er.conv3x3_fwd(x, w, b.astype(np.float64), s, relu)
    xd, wd, bd = to_bf16(x, dev), to_bf16(w, dev), torch.from_numpy(b).to(dev)
    y32 = cgh.conv3x3_fwd(xd, wd, bd, s, relu, out_f32=True).cpu().numpy()
    assert rel_l2(y32, ref) < F32_TOL
    y16 = cgh.conv3x3_fwd(xd, wd, bd, s, relu, out_f32=False).float().cpu().numpy()
    scale = np.abs(ref).max() + 1e-30
    assert np.all(np.abs(y16 - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6 * scale)


@pytest.mark.parametrize("case", CONV_CASES)
@pytest.mark.parametrize("relu", [False, True])
@pytest.mark.parametrize("y_bf16", [False, True])
def test_conv_bwd(case, relu, y_bf16, dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    B, CI, H, W, CO, s = case
    rng = np.random.default_rng(hash(case) % 1000 + 1)
    x = bf16_round(rng.standard_normal((B, CI, H, W)))
    w = bf16_round(rng.standard_normal((CO, CI, 3, 3)) / np.sqrt(9 * CI))
    b = rng.standard_normal(CO)
    y = er.conv3x3_fwd(x, w, b, s, relu)
    # the mask source: the oracle's forward output, stored like the kernel stores it
    y_in = bf16_round(y) if y_bf16 else y.astype(np.float32).astype(np.float64)
    dy = rng.standard_normal(y.shape)
    dx_ref, dw_ref, db_ref = er.conv3x3_bwd(x, w, y_in, dy, s, relu)
    yd = to_bf16(y_in, dev) if y_bf16 else torch.from_numpy(y_in.astype(np.float32)).to(dev)
    dx, dw, db = cgh.conv3x3_bwd(to_bf16(x, dev), to_bf16(w, dev), yd,
                                 torch.from_numpy(dy.astype(np.float32)).to(dev), s, relu)
    assert rel_l2(dx.cpu().numpy(), dx_ref) < F32_TOL
    assert rel_l2(dw.cpu().numpy(), dw_ref) < F32_TOL
    assert rel_l2(db.cpu().numpy(), db_ref) < F32_TOL


def test_conv_bwd_skip_dx(dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    rng = np.random.default_rng(5)
    x = bf16_round(rng.standard_normal((2, 3, 20, 24)))
    w = bf16_round(rng.standard_normal((8, 3, 3, 3)))
    y = er.conv3x3_fwd(x, w, np.zeros(8), 2, False)
    dy = rng.standard_normal(y.shape)
    _, dw_ref, db_ref = er.conv3x3_bwd(x, w, y, dy, 2, False)
    dx, dw, db = cgh.conv3x3_bwd(to_bf16(x, dev), to_bf16(w, dev), None,
                                 torch.from_numpy(dy.astype(np.float32)).to(dev), 2, False,
                                 want_dx=False)
    assert dx is None
    assert rel_l2(dw.cpu().numpy(), dw_ref) < F32_TOL and rel_l2(db.cpu().numpy(), db_ref) < F32_TOL


def test_cast_bf16_round_to_nearest_even(dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.standard_normal(10007) * 10.0 ** rng.integers(-30, 30, 10007),
                        [0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 3.0e38]])
    a = a.astype(np.float32)
    got = cgh.cast_bf16(torch.from_numpy(a).to(dev)).float().cpu().numpy()
    # round-to-nearest-even on the raw bits (no NaNs in the input)
    bits = a.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    want = (((bits + 0x7FFF + lsb) >> 16) << 16).astype(np.uint32).view(np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("S,C,H,W,CY,CX", [(16, 3, 64, 80, 4, 5), (9, 1, 30, 45, 2, 3),
                                            (1, 2, 16, 16, 1, 1)])
def test_decode_and_adjoint(S, C, H, W, CY, CX, dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    rng = np.random.default_rng(S * 100 + C)
    B = 2
    out = rng.standard_normal((B, S * (6 + 2 * C), CY, CX)).astype(np.float32)
    p = cgh.encoder_decode(torch.from_numpy(out).to(dev), S, C, H, W)
    ref = er.decode(out.astype(np.float64), S, C, H, W)
    N = CY * CX * S
    for k in cgh.PARAM_KEYS:
        got = p[k].cpu().numpy().reshape((B, N) + ref[0][k].shape[1:])
        for b in range(B):
            assert np.abs(got[b] - ref[b][k]).max() < 2e-5 * (1 + np.abs(ref[b][k]).max()), k
    g = [{k: rng.standard_normal(np.shape(v)) for k, v in d.items()} for d in ref]
    gd = {k: torch.from_numpy(np.concatenate([gb[k] for gb in g]).astype(np.float32)).to(dev)
          for k in cgh.PARAM_KEYS}
    dout = cgh.encoder_decode_bwd(gd, B, CY, CX, S, C, H, W).cpu().numpy()
    assert rel_l2(dout, er.decode_bwd(g, S, C, CY, CX)) < 1e-6


def test_mse_grad(dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    rng = np.random.default_rng(8)
    pred, tgt, g0 = (rng.standard_normal(70001) for _ in range(3))
    P, T = (torch.from_numpy(a.astype(np.float32)).to(dev) for a in (pred, tgt))
    G = torch.from_numpy(g0.astype(np.float32)).to(dev)
    acc = torch.zeros(1, device=dev)
    cgh.mse_grad(P, T, 0.25, G, accumulate=True, loss_accum=acc)
    p32, t32 = pred.astype(np.float32).astype(np.float64), tgt.astype(np.float32).astype(np.float64)
    assert rel_l2(G.cpu().numpy(), g0.astype(np.float32) + 0.5 * (p32 - t32)) < 1e-6
    assert abs(float(acc) - 0.25 * np.sum((p32 - t32) ** 2)) < 1e-5 * 0.25 * np.sum((p32 - t32) ** 2)
    cgh.mse_grad(P, T, 0.25, G, accumulate=False)
    assert rel_l2(G.cpu().numpy(), 0.5 * (p32 - t32)) < 1e-6


def test_encoder_training_gradient_chain(dev):
    """Every layer's weight and bias gradient of the intensity loss of the decoded prediction
    (target -> 4 convolutions -> decode -> raster -> BLASM -> loss, and back) against the
    oracle's step, decode adjoint and convolution backward."""
    import torch
    from paper_2511_15022_gb300 import cgh
    from paper_2511_15022_gb300.encoder import STRIDE, Encoder
    H = W = 64
    wl, pitch, z = (638e-9, 520e-9, 450e-9), 8e-6, (5e-3,)
    C, S, B = 3, 16, 2
    enc = Encoder(C, S, device=dev, seed=3)
    # a last layer with weights of the same order as the hidden ones, so that the decoded
    # Gaussians move away from their anchors and every parameter kind carries gradient
    enc.w[-1].normal_(0.0, 0.05, generator=torch.Generator(device=dev).manual_seed(4))
    enc.sync_bf16()
    tgt = inputs.blob_targets(B, C, H, W, seed=17).astype(np.float32)
    tgt_d = torch.from_numpy(tgt).to(dev)
    cy, cx = enc.cells(H, W)
    N = cy * cx * S
    plan = cgh.Plan(H, W, wl, pitch, z, max_gaussians=N, device=dev)
    out, acts = enc.forward(tgt_d)
    prm = cgh.encoder_decode(out, S, C, H, W)
    grads = cgh.param_dict(B * N, C, dev)
    for b in range(B):
        sl = {k: v[b * N:(b + 1) * N] for k, v in prm.items()}
        gs = {k: v[b * N:(b + 1) * N] for k, v in grads.items()}
        plan.step(sl, tgt_d[b:b + 1].contiguous(), grads=gs)
    dout = cgh.encoder_decode_bwd(grads, B, cy, cx, S, C, H, W)
    enc.backward(acts, dout)

    # oracle: BF16-rounded weights and input, activations rounded to BF16 between layers
    ws = [bf16_round(w.cpu().numpy()) for w in enc.w]
    bs = [b.cpu().numpy().astype(np.float64) for b in enc.b]
    a = [bf16_round(tgt)]
    for i in range(4):
        y = er.conv3x3_fwd(a[-1], ws[i], bs[i], STRIDE, i < 3)
        a.append(bf16_round(y) if i < 3 else y)
    dec = er.decode(a[-1], S, C, H, W)
    g_ref = [oracle.step(dec[b], tgt[b][None].astype(np.float64), H, W, wl, pitch, z)["grads"]
             for b in range(B)]
    dy = er.decode_bwd(g_ref, S, C, cy, cx)
    for i in reversed(range(4)):
        dx, dw, db = er.conv3x3_bwd(a[i], ws[i], a[i + 1], dy, STRIDE, i < 3)
        assert rel_l2(enc.dw[i].cpu().numpy(), dw) < GRAD_TOL, f"layer {i} weights"
        assert rel_l2(enc.db[i].cpu().numpy(), db) < GRAD_TOL, f"layer {i} bias"
        dy = dx
