"""Helpers shared by the GPU tests (device buffers through torch)."""
import numpy as np

import paper_2609_02394_b300 as P


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def dev(a, dtype=np.float64):
    torch = torch_cuda()
    return torch.tensor(np.ascontiguousarray(a, dtype=dtype), device="cuda")


def host(t):
    torch = torch_cuda()
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def overlap_singular_values(C_ref, C_gpu):
    """Singular values of C_ref^T C_gpu (columns are basis vectors): all 1 when
    the two retained subspaces coincide, whatever basis each side chose."""
    return np.linalg.svd(C_ref.T @ C_gpu, compute_uv=False)
