"""The FP64 throughput kernel behind the bench's FP64 roof: it runs, its
operation count is the documented one, and the rate it gives lies within a
factor of two of GB300's FP64 figure (1.25 TFLOP/s dense)."""
import pytest
import torch

from paper_1705_02003_gb300 import ens

pytestmark = pytest.mark.gpu


def test_fp64_peak_kernel_rate(ens_lib):
    h = ens.Handle(0)
    blocks, iters = 152 * 8, 1024
    sink = torch.zeros(blocks, dtype=torch.float64, device="cuda")
    ens.ens_fp64_peak(h, blocks, iters, sink)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    flops = ens.ens_fp64_peak(h, blocks, iters, sink)
    e1.record()
    torch.cuda.synchronize()
    assert flops == 2 * 8 * iters * blocks * 256
    rate = flops / (e0.elapsed_time(e1) * 1e-3) / 1e12
    assert 0.6 < rate < 2.5, rate
    assert not sink.any()  # the sink is never written for these seeds
    with pytest.raises(ens.EnsError):
        ens.ens_fp64_peak(h, 0, iters, sink)
    h.close()
