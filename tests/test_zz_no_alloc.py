"""fhd_frame_digest_noalloc -- the digest entry point for callers that cannot
allocate device memory (a real-time capture/encode loop, where an allocator
call can block or synchronise the device and stall work in flight, or a host
framework that reserves all device memory up front).  It must give exactly
the digests of the allocating entry point fhd_frame_digest and of the oracle,
call after call, although every call reuses the same fixed device array.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test; it passes on its own too."""
import ctypes

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

fhd = pytest.importorskip("paper_2505_07158_gb300")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_digest_equals_allocating_digest_two_calls_in_a_row():
    lib = fhd.load()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    g = np.random.Generator(np.random.PCG64(2024))
    # Two different calls in a row through the C ABI; the second uses fewer
    # sub-frame slots than the first, so stale contents of the shared array
    # would show if the entry point read anything it had not written.
    for nbytes, n, count in [(1920 * 1080 * 3, 32, 2), (12345, 12, 3)]:
        data = torch.from_numpy(g.integers(0, 256, size=nbytes * count, dtype=np.uint8)).to(dev)
        out = torch.full((count, 32), 0xAB, dtype=torch.uint8, device=dev)
        rc = lib.fhd_frame_digest_noalloc(_ptr(data), nbytes, n, count, _ptr(out), ctypes.c_void_p(stream.cuda_stream))
        assert rc == fhd.FHD_OK, lib.cipher_last_error(None)
        ref = fhd.fhd_frame_digest(data, n=n, count=count)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        host = data.cpu().numpy()
        for k in range(count):   # and the oracle's digest of each buffer (Sec. II-A)
            assert bytes(out[k].cpu().numpy()) == oracle.frame_digest(host[k * nbytes:(k + 1) * nbytes], n=n), k


def test_noalloc_rejects_requests_beyond_the_fixed_array():
    lib = fhd.load()
    dev = torch.device("cuda:0")
    data = torch.zeros(1024 * 65, dtype=torch.uint8, device=dev)
    out = torch.zeros((65, 32), dtype=torch.uint8, device=dev)
    rc = lib.fhd_frame_digest_noalloc(_ptr(data), 1024, 1024, 65, _ptr(out), None)   # 66560 > 65536 digests
    assert rc == fhd.FHD_ERR_TOO_LARGE
    assert b"FHD_NOALLOC_MAX_SUBFRAMES" in lib.cipher_last_error(None)
