"""The binary64 pipe probe (the peak of the worker kernel's roofline): it runs one CTA per SM with k warps
per sub-partition, reports the lane-operations it executes, and more warps per sub-partition never make
the pipe slower per operation by much (the pipe saturates, it does not thrash)."""
import pytest
import torch

pytestmark = pytest.mark.gpu

fhd = pytest.importorskip("paper_2505_07158_gb300")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_probe_counts_and_rates():
    dev = torch.device("cuda:0")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(sms, dtype=torch.float64, device=dev)
    rates = {}
    for k in (1, 2, 4):
        fhd.fhd_fp64_probe(k, 256, sink)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ops = fhd.fhd_fp64_probe(k, 4096, sink)
        b.record()
        b.synchronize()
        assert ops == sms * 128 * k * 4096 * 8
        rates[k] = ops / a.elapsed_time(b)
    assert rates[2] > 0.9 * rates[1] and rates[4] > 0.9 * rates[2]
    assert torch.count_nonzero(sink) == 0      # the guarded store never fires for these constants
