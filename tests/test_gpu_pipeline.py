"""The double-buffered input pipeline hands every step exactly the input put for it, also
when steps queue faster than the copies finish."""
import pytest

pytestmark = pytest.mark.gpu


def test_pipeline_order_and_reuse():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15022_gb300.pipeline import InputPipeline
    dev = torch.device("cuda", 0)
    n = 1 << 20
    hosts = [torch.full((n,), float(k)).pin_memory() for k in range(7)]
    pipe = InputPipeline((n,), torch.float32, dev)
    acc = torch.zeros(7, device=dev)
    pipe.put(hosts[0])
    for k in range(7):
        x = pipe.get()
        if k + 1 < 7:
            pipe.put(hosts[k + 1])
        # a slow reader: the next put into this buffer must wait for it
        acc[k] = (x * 1.0).sum() / n + 0 * torch.cumsum(x, 0)[-1]
        pipe.release()
    torch.cuda.synchronize()
    assert acc.cpu().tolist() == [float(k) for k in range(7)]
