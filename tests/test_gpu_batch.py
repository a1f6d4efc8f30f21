"""Batched holograms in one CUDA graph, the block-shape autotuner and the table Adam:
every hologram of a batch against the FP64 oracle's step directly, and the batch against the
single-hologram entry points."""
import numpy as np
import pytest

import oracle
from paper_2511_15022_gb300 import inputs
from tests.gpu_util import rel_l2, to64, to_dev

LOSS_TOL = 1e-4
GRAD_TOL = 1e-3

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def _plan(w, dev):
    from paper_2511_15022_gb300 import cgh
    return cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, cutoff=w.cutoff,
                    max_gaussians=w.N, device=dev)


def test_batch_graph_and_sequential_match_single_steps(dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    ws = [inputs.custom(64, 96, 400, wavelengths_m=(638e-9, 520e-9, 450e-9), z_m=(0.0, 5e-3), seed=81),
          inputs.custom(256, 256, 2048, seed=82),
          inputs.custom(100, 120, 900, wavelengths_m=(520e-9,), z_m=(3e-3, 6e-3, 9e-3), seed=83)]
    plans = [_plan(w, dev) for w in ws]
    batch = cgh.Batch(plans)
    data = []
    for i, (w, plan) in enumerate(zip(ws, plans)):
        p = to_dev(inputs.params_for(w), dev)
        t = torch.from_numpy(inputs.blob_targets(w.L, w.C, w.H, w.W, seed=90 + i)).to(dev)
        g = plan.empty_grads(w.N)
        loss = torch.empty(1, device=dev)
        batch.bind(i, p, t, g, loss)
        ref_loss, ref_g = plan.step(p, t)
        data.append((loss, g, ref_loss.clone(), {k: v.clone() for k, v in ref_g.items()}))
    for use_graph in (True, True, False):  # capture + replay, replay again, sequential
        for loss, g, _, _ in data:
            loss.fill_(-1.0)
            for v in g.values():
                v.fill_(float("nan"))
        batch.step(use_graph=use_graph)
        torch.cuda.synchronize()
        for loss, g, ref_loss, ref_g in data:
            assert abs(loss.item() - ref_loss.item()) <= 1e-5 * abs(ref_loss.item())
            for k in g:
                assert rel_l2(g[k].cpu().numpy(), ref_g[k].cpu().numpy()) < 1e-4, k
    assert batch.kernels_per_step > 3 * 10


def test_batch_matches_oracle_per_hologram(dev):
    """Each hologram of a mixed batch (sizes, channel and plane counts differ; one plane at
    z = 0) after a graph replay, against the oracle's forward + backward of that hologram."""
    import torch
    from paper_2511_15022_gb300 import cgh
    ws = [inputs.custom(64, 96, 400, wavelengths_m=(638e-9, 520e-9, 450e-9), z_m=(0.0, 5e-3), seed=84),
          inputs.custom(128, 128, 1500, seed=85),
          inputs.custom(100, 120, 900, wavelengths_m=(520e-9,), z_m=(3e-3, 6e-3, 9e-3), seed=86),
          inputs.custom(96, 160, 1200, wavelengths_m=(638e-9, 450e-9), z_m=(0.0, 4e-3, 8e-3), seed=87)]
    plans = [_plan(w, dev) for w in ws]
    batch = cgh.Batch(plans)
    data = []
    for i, (w, plan) in enumerate(zip(ws, plans)):
        p_np = inputs.params_for(w)
        t_np = inputs.blob_targets(w.L, w.C, w.H, w.W, seed=95 + i)
        g = plan.empty_grads(w.N)
        loss = torch.empty(1, device=dev)
        batch.bind(i, to_dev(p_np, dev), torch.from_numpy(t_np).to(dev), g, loss)
        data.append((w, p_np, t_np, loss, g))
    batch.step(use_graph=True)
    batch.step(use_graph=True)  # a replay of the captured graph
    torch.cuda.synchronize()
    for w, p_np, t_np, loss, g in data:
        ref = oracle.step(to64(p_np), t_np.astype(np.float64), w.H, w.W, w.wavelengths_m,
                          w.pitch_m, w.z_m, cutoff=w.cutoff)
        assert abs(loss.item() - ref["loss"]) <= LOSS_TOL * abs(ref["loss"]), w.name
        for k in g:
            assert rel_l2(g[k].double().cpu().numpy(), ref["grads"][k]) < GRAD_TOL, (w.name, k)


def test_autotune_keeps_a_valid_fastest_shape(dev):
    import torch
    w = inputs.custom(100, 120, 1500, wavelengths_m=(638e-9, 520e-9, 450e-9),
                      z_m=(0.0, 5e-3, 10e-3), seed=12)
    plan = _plan(w, dev)
    p = to_dev(inputs.params_for(w), dev)
    t = torch.from_numpy(inputs.blob_targets(w.L, w.C, w.H, w.W)).to(dev)
    ref_loss, ref_g = plan.step(p, t)
    ref_g = {k: v.clone() for k, v in ref_g.items()}
    best = plan.autotune(p, t, iters=2)
    assert best == plan.get_tuning()
    loss, g = plan.step(p, t)
    assert abs(loss.item() - ref_loss.item()) < 1e-5 * ref_loss.item()
    for k in g:
        assert rel_l2(g[k].cpu().numpy(), ref_g[k].cpu().numpy()) < 1e-4


def test_adam_table_matches_per_group_adam(dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    gen = torch.Generator().manual_seed(3)
    sizes = [5, 1000, 37, 4096, 1]
    a = [torch.randn(n, generator=gen).to(dev) for n in sizes]
    b = [x.clone() for x in a]
    ma = [torch.zeros_like(x) for x in a]; va = [torch.zeros_like(x) for x in a]
    mb = [torch.zeros_like(x) for x in a]; vb = [torch.zeros_like(x) for x in a]
    grads = [torch.randn(n, generator=gen).to(dev) for n in sizes]
    lrs = [1e-2, 5e-3, 1e-3, 2.5e-2, 0.1]
    table = cgh.AdamTable([(a[i], ma[i], va[i], grads[i], lrs[i]) for i in range(len(sizes))])
    for step in range(1, 4):
        table.step()
        cgh.adam_step([(b[i], grads[i], mb[i], vb[i], lrs[i]) for i in range(len(sizes))], step)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.allclose(x, y, rtol=1e-6, atol=1e-7)
