"""Helpers shared by the GPU tests (no method arithmetic here)."""
import numpy as np
import torch

from paper_1312_1869_gb300 import ckinv as ck


def col(a):
    """numpy (n, m) -> CUDA column-major float32 tensor."""
    a = np.asarray(a, dtype=np.float32)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    t = torch.from_numpy(np.ascontiguousarray(a.T)).cuda()
    return t.t()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def bits_to_signs(bits_t, n):
    b = bits_t.cpu().numpy().view(np.uint32)
    k = np.arange(n)
    s = (b[k >> 5] >> (k & 31).astype(np.uint32)) & 1
    return np.where(s == 0, 1.0, -1.0)


def kernel(kind, ell, var, tau):
    return ck.Kernel(kind, ell, var, tau)
