"""FP64 reference of the learned surrogate -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
use this module; the CUDA library shares no code with it.

The surrogate (not in the paper; a learned stand-in for the tier-2 predictor of Sec. 2) maps
a standardized feature vector straight to the six per-optimization log speedups:

    h1 = gelu(W1 x + b1),  h2 = gelu(W2 h1 + b2),  out = W3 h2 + b3,
    gelu(u) = u (1 + tanh(c (u + a u^3))) / 2,  c = sqrt(2 / pi),  a = 0.044715
    (the tanh form of GELU, Hendrycks and Gimpel 2016, within 1e-3 of u * Phi(u)),

trained on the mean squared error  L = sum_{b, j} (out_bj - y_bj)^2 / (B * 6)  with AdamW
(bias-corrected first and second moments, decoupled weight decay).  Shapes: W1 [512, 256],
W2 [512, 512], W3 [6, 512] (rows = outputs), biases of the output width.  Plain numpy in
float64; matrix products are the only library primitive.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict

import numpy as np

DIMS = (256, 512, 512, 6)
NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def gelu(u: np.ndarray) -> np.ndarray:
    """The tanh form: u (1 + tanh(c (u + a u^3))) / 2."""
    u = np.asarray(u, dtype=np.float64)
    return 0.5 * u * (1.0 + np.tanh(GELU_C * (u + GELU_A * u ** 3)))


def gelu_grad(u: np.ndarray) -> np.ndarray:
    """d/du of the tanh form: (1 + t) / 2 + u (1 - t^2) c (1 + 3 a u^2) / 2,
    t = tanh(c (u + a u^3))."""
    u = np.asarray(u, dtype=np.float64)
    t = np.tanh(GELU_C * (u + GELU_A * u ** 3))
    return 0.5 * (1.0 + t) + 0.5 * u * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * u * u)


def init_params(seed: int = 0, dims=DIMS) -> Dict[str, np.ndarray]:
    """The seeded initial weights (drawn by the shared input generator, synth.init_mlp_params)."""
    from paper_1910_07776_gb300 import synth
    return synth.init_mlp_params(seed, dims)


def forward(p, x):
    """Returns (out, cache) for input rows x [B, 256]."""
    x = np.asarray(x, dtype=np.float64)
    u1 = x @ p["W1"].T + p["b1"]
    h1 = gelu(u1)
    u2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(u2)
    out = h2 @ p["W3"].T + p["b3"]
    return out, (x, u1, h1, u2, h2)


def loss_and_grads(p, x, y):
    """MSE over all outputs and its gradient with respect to every parameter."""
    out, (x, u1, h1, u2, h2) = forward(p, x)
    B = x.shape[0]
    r = out - np.asarray(y, dtype=np.float64)
    loss = float(np.sum(r * r) / (B * out.shape[1]))
    d_out = 2.0 * r / (B * out.shape[1])
    g = {}
    g["W3"] = d_out.T @ h2
    g["b3"] = d_out.sum(axis=0)
    d_h2 = d_out @ p["W3"]
    d_u2 = d_h2 * gelu_grad(u2)
    g["W2"] = d_u2.T @ h1
    g["b2"] = d_u2.sum(axis=0)
    d_h1 = d_u2 @ p["W2"]
    d_u1 = d_h1 * gelu_grad(u1)
    g["W1"] = d_u1.T @ x
    g["b1"] = d_u1.sum(axis=0)
    return loss, g


@dataclass
class AdamW:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    weight_decay: float = 0.0
    t: int = 0
    m: Dict[str, np.ndarray] = field(default_factory=dict)
    v: Dict[str, np.ndarray] = field(default_factory=dict)

    def step(self, p, g):
        """w <- w - lr * (mhat / (sqrt(vhat) + eps) + weight_decay * w)."""
        self.t += 1
        for k in NAMES:
            if k not in self.m:
                self.m[k] = np.zeros_like(p[k])
                self.v[k] = np.zeros_like(p[k])
            self.m[k] = self.beta1 * self.m[k] + (1 - self.beta1) * g[k]
            self.v[k] = self.beta2 * self.v[k] + (1 - self.beta2) * g[k] * g[k]
            mh = self.m[k] / (1 - self.beta1 ** self.t)
            vh = self.v[k] / (1 - self.beta2 ** self.t)
            p[k] = p[k] - self.lr * (mh / (np.sqrt(vh) + self.eps) + self.weight_decay * p[k])
        return p


def ood_score(x, mean, std):
    """Out-of-distribution score of each row: mean squared z of its features against the
    training set's per-feature mean and standard deviation."""
    z = (np.asarray(x, dtype=np.float64) - mean) / np.where(std > 0, std, 1.0)
    return np.mean(z * z, axis=1)
