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


def grad_tol(ref, ref_perturbed, floor: float = 1e-2) -> float:
    """Tolerance of a gradient of the BF16 blocks against the FP64 reference: the
    1e-2 bar, widened to twice the reference's own change when its input is perturbed
    by 1e-6 relative (the FP32 rounding scale). BF16 roundings of activations make
    some gradients discontinuous at that scale, so no FP32 evaluation can be closer."""
    return max(floor, 2.0 * rel_l2(ref_perturbed, ref))
