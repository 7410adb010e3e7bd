"""Helpers shared by the GPU parity tests (CUDA path through the C ABI vs the FP64 oracle)."""
import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")


def lib():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2510_05975_gb300.cng as cng

    return cng


def tensor(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()
