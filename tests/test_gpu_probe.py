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


def test_integer_binary64_equals_the_binary64_instructions():
    """The integer-pipe multiply and add (the integer worker mix) give the binary64 instructions' results
    bit for bit on 2^26 generated operand pairs of every class the generator has (any bit patterns, the
    chaotic range, near cancellation, the sum's alignment boundary, few significand bits for exact products
    and ties, zeros and subnormals), and their integer fast path takes most of them."""
    n = 1 << 26
    r = fhd.fhd_binary64_check(n, seed=20261204)
    assert r["bad_mul"] == 0 and r["bad_add"] == 0, r
    assert r["fast_mul"] > n // 2 and r["fast_add"] > n // 2, r
    r2 = fhd.fhd_binary64_check(1 << 20, seed=7)
    assert r2["bad_mul"] == 0 and r2["bad_add"] == 0, r2
