"""The batched step as one persistent kernel (cgh_batch_step_persistent): every hologram of a
mixed batch against the FP64 oracle's step and against the graph-captured batch, two steps in
a row, and the bounded grid barrier: with the test hook making CTA 0 skip one arrival, the
launch ends with CGH_ERR_TIMEOUT reported instead of hanging, and the next step is correct."""
import numpy as np
import pytest

import oracle
from paper_2511_15022_gb300 import inputs
from tests.gpu_util import rel_l2, to64, to_dev

pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-4
GRAD_TOL = 1e-3
RGB = (638e-9, 520e-9, 450e-9)


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def _batch(ws, dev, seed0):
    import torch
    from paper_2511_15022_gb300 import cgh
    plans = [cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, cutoff=w.cutoff,
                      max_gaussians=w.N, device=dev) for w in ws]
    batch = cgh.Batch(plans)
    data = []
    for i, (w, plan) in enumerate(zip(ws, plans)):
        p_np = inputs.params_for(w)
        t_np = inputs.blob_targets(w.L, w.C, w.H, w.W, seed=seed0 + i)
        g = plan.empty_grads(w.N)
        loss = torch.empty(1, device=dev)
        batch.bind(i, to_dev(p_np, dev), torch.from_numpy(t_np).to(dev), g, loss)
        data.append((w, p_np, t_np, loss, g))
    return plans, batch, data


WS = [inputs.custom(64, 96, 400, wavelengths_m=RGB, z_m=(0.0, 5e-3), seed=91),
      inputs.custom(128, 128, 1500, seed=92),
      inputs.custom(100, 120, 900, wavelengths_m=(520e-9,), z_m=(3e-3, 6e-3, 9e-3), seed=93),
      inputs.custom(96, 160, 1200, wavelengths_m=(638e-9, 450e-9), z_m=(0.0,), seed=94),
      inputs.custom(80, 80, 0, seed=95)]  # a hologram without Gaussians


def test_persistent_step_matches_oracle_and_graph(dev):
    import torch
    plans, batch, data = _batch(WS, dev, 100)
    for _ in range(2):  # the second launch starts from the first one's workspace contents
        for _, _, _, loss, g in data:
            loss.fill_(-1.0)
            for v in g.values():
                v.fill_(float("nan"))
        batch.step_persistent()
        assert not batch.persistent_status()
        torch.cuda.synchronize()
        for w, p_np, t_np, loss, g in data:
            ref = oracle.step(to64(p_np), t_np.astype(np.float64), w.H, w.W, w.wavelengths_m,
                              w.pitch_m, w.z_m, cutoff=w.cutoff)
            assert abs(loss.item() - ref["loss"]) <= LOSS_TOL * abs(ref["loss"]), w.name
            for k in g:
                if w.N:
                    assert rel_l2(g[k].double().cpu().numpy(), ref["grads"][k]) < GRAD_TOL, (w.name, k)
    assert batch.persistent_grid > 0
    persistent = [(loss.item(), {k: v.clone() for k, v in g.items()}) for _, _, _, loss, g in data]
    batch.step(use_graph=True)
    torch.cuda.synchronize()
    for (l0, g0), (w, _, _, loss, g) in zip(persistent, data):
        assert abs(l0 - loss.item()) <= 1e-5 * abs(loss.item()), w.name
        for k in g:
            if w.N:
                assert rel_l2(g0[k].double().cpu().numpy(), g[k].double().cpu().numpy()) < 1e-4, (w.name, k)


def test_persistent_barrier_timeout_is_reported_not_hung(dev):
    """CTA 0 does not arrive at grid barrier 3: no wait can complete, every wait runs out
    after 50 ms of clock, the kernel returns and the host reads the timeout; with the hook
    off, the next step is correct again."""
    import torch
    plans, batch, data = _batch(WS[:3], dev, 110)
    batch.persistent_test(skip_barrier=3, timeout_s=0.05)
    batch.step_persistent()
    assert batch.persistent_status() is True
    batch.persistent_test(skip_barrier=-1, timeout_s=0.0)
    batch.step_persistent()
    assert batch.persistent_status() is False
    torch.cuda.synchronize()
    w, p_np, t_np, loss, g = data[1]
    ref = oracle.step(to64(p_np), t_np.astype(np.float64), w.H, w.W, w.wavelengths_m, w.pitch_m,
                      w.z_m, cutoff=w.cutoff)
    assert abs(loss.item() - ref["loss"]) <= LOSS_TOL * abs(ref["loss"])
