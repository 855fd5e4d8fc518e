"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_gpu(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def to_np(t):
    return t.detach().double().cpu().numpy()
