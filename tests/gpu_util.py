"""Helpers shared by the GPU tests (device transfer of oracle-shaped arrays)."""
import numpy as np
import torch


def dev():
    return torch.device("cuda:0")


def to_dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def d16(D: np.ndarray) -> torch.Tensor:
    """uint16 distances as an int16 CUDA tensor with the same bits."""
    return to_dev(np.ascontiguousarray(D, dtype=np.uint16).view(np.int16))


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()


def host_u16(t: torch.Tensor) -> np.ndarray:
    return host(t).view(np.uint16)
