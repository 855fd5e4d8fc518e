"""FP64 reference of the training step around the learned reconstruction (test
infrastructure only; plain NumPy, element by element where it matters).

  * masked_mse: the image loss over the full field of view. The paper (Sec. 2.6,
    image-loss equation) takes its loss over FullFoV, the voxels present in at
    least half of the projections, i.e. V >= 1/2 with V the field-of-view tensor;
    the reading used here is the mean squared error over {V >= thr}:
        count = #{i : V_i >= thr},  loss = sum_{V_i >= thr} (x_i - r_i)^2 / count,
        dloss/dx_i = 2 (x_i - r_i) / count on the mask, 0 off it (0 when count = 0).
  * adam: the optimiser the paper trains with (Sec. 2.6, Adam with learning rate
    1e-3), as defined by Kingma & Ba (2014, Algorithm 1), with the gradient first
    multiplied by grad_scale:
        g = grad_scale * grad
        m <- beta1 m + (1 - beta1) g,      v <- beta2 v + (1 - beta2) g^2
        m_hat = m / (1 - beta1^t),         v_hat = v / (1 - beta2^t)
        theta <- theta - lr m_hat / (sqrt(v_hat) + eps)
  * clip_grads: global gradient-norm clipping before the step,
        n = ||grad_scale g||,  g <- g min(1, max_norm / n)  (g <- 0 when n is not finite).
"""
from __future__ import annotations

import math

import numpy as np


def masked_mse(x: np.ndarray, ref: np.ndarray, V: np.ndarray | None = None, thr: float = 0.5):
    """(loss, grad) of the mean squared error over the voxels with V >= thr (all voxels
    when V is None)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    r = np.asarray(ref, dtype=np.float64).reshape(-1)
    mask = np.ones(x.shape, dtype=bool) if V is None else (np.asarray(V, dtype=np.float64).reshape(-1) >= thr)
    count = int(np.count_nonzero(mask))
    grad = np.zeros_like(x)
    if count == 0:
        return 0.0, grad
    d = x[mask] - r[mask]
    loss = math.fsum(d * d) / count
    grad[mask] = 2.0 * d / count
    return loss, grad


class Adam:
    """Adam state (first and second moments, step count) over a flat parameter vector."""

    def __init__(self, n: int):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0

    def step(self, theta: np.ndarray, grad: np.ndarray, lr: float, beta1: float = 0.9, beta2: float = 0.999,
             eps: float = 1e-8, grad_scale: float = 1.0) -> np.ndarray:
        """Returns the updated parameters (the input is not modified)."""
        self.t += 1
        g = grad_scale * np.asarray(grad, dtype=np.float64)
        self.m = beta1 * self.m + (1.0 - beta1) * g
        self.v = beta2 * self.v + (1.0 - beta2) * g * g
        m_hat = self.m / (1.0 - beta1 ** self.t)
        v_hat = self.v / (1.0 - beta2 ** self.t)
        return np.asarray(theta, dtype=np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps)


def clip_grads(grad: np.ndarray, max_norm: float, grad_scale: float = 1.0):
    """(norm of grad_scale * grad, clipped grad)."""
    g = np.asarray(grad, dtype=np.float64)
    n = math.sqrt(math.fsum((g * g).reshape(-1))) * abs(grad_scale)
    if not math.isfinite(n):
        return n, np.zeros_like(g)
    return n, g * (max_norm / n if n > max_norm else 1.0)
