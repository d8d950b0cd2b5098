"""The entry point's smoke() -- one small frame encrypted and decrypted on cuda:0 through the C ABI in both
worker layouts, checked against the oracle -- runs and returns."""
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_smoke_runs():
    import __graft_entry__ as g
    g.smoke()
