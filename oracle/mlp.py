"""Oracle for the learned-entry MLP (test infrastructure only).

The paper has no learned component; this network is the project's own entry
predictor: a query goes through 256->512->512 ReLU layers (sizes are
parameters) to one logit per ghost node, and the top-P ghost nodes seed the
ghost stage of the search (Section 3.2.2 supplies the ghost set).

Everything is FP64 numpy, written as the definitions: affine maps, ReLU,
softmax cross-entropy averaged over the batch, its gradient by the chain
rule, and AdamW (decoupled weight decay). The GPU computes with BF16 GEMM
operands and FP32 accumulation; ``bf16=True`` rounds exactly the tensors the
GPU feeds to its GEMMs (queries, weights, hidden activations, the logit and
activation gradients) to BF16 before using them, and accumulates in FP64.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, Optional

import numpy as np

LAYERS = ("W1", "b1", "W2", "b2", "W3", "b3")


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32.
    BF16 keeps the top 16 bits of the FP32 pattern; the discarded low half
    decides the rounding. Inputs are finite."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(f.shape)


@dataclass
class MLP:
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray
    # per-dimension input standardisation x' = (x - mean) * inv_std, applied
    # in FP32 before the BF16 rounding of the queries (None = identity)
    mean: Optional[np.ndarray] = None
    inv_std: Optional[np.ndarray] = None

    def params(self) -> Dict[str, np.ndarray]:
        return {k: getattr(self, k) for k in LAYERS}

    def copy(self) -> "MLP":
        c = MLP(**{k: v.copy() for k, v in self.params().items()})
        if self.mean is not None:
            c.mean, c.inv_std = self.mean.copy(), self.inv_std.copy()
        return c


def _q(x, bf16):
    return bf16_round(x).astype(np.float64) if bf16 else np.asarray(x, dtype=np.float64)


def standardise(m: MLP, X: np.ndarray) -> np.ndarray:
    """(x - mean) * inv_std elementwise, each operation rounded to FP32."""
    X = np.asarray(X, dtype=np.float32)
    if m.mean is None:
        return X
    d = np.subtract(X, np.asarray(m.mean, dtype=np.float32), dtype=np.float32)
    return np.multiply(d, np.asarray(m.inv_std, dtype=np.float32), dtype=np.float32)


def forward(m: MLP, X: np.ndarray, bf16: bool = True) -> Dict[str, np.ndarray]:
    """x' = standardise(x); h1 = relu(x' W1^T + b1), h2 = relu(h1 W2^T + b2),
    z = h2 W3^T + b3."""
    Xq = _q(standardise(m, X), bf16)
    a1 = Xq @ _q(m.W1, bf16).T + m.b1.astype(np.float64)
    h1 = np.maximum(a1, 0.0)
    h1q = _q(h1.astype(np.float32), bf16) if bf16 else h1
    a2 = h1q @ _q(m.W2, bf16).T + m.b2.astype(np.float64)
    h2 = np.maximum(a2, 0.0)
    h2q = _q(h2.astype(np.float32), bf16) if bf16 else h2
    z = h2q @ _q(m.W3, bf16).T + m.b3.astype(np.float64)
    return {"Xq": Xq, "a1": a1, "h1q": h1q, "a2": a2, "h2q": h2q, "z": z}


def softmax(z: np.ndarray) -> np.ndarray:
    e = np.exp(z - z.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def loss(m: MLP, X: np.ndarray, y: np.ndarray, bf16: bool = True) -> float:
    """Mean softmax cross-entropy: mean_i (logsumexp(z_i) - z_i[y_i])."""
    z = forward(m, X, bf16)["z"]
    mx = z.max(axis=1)
    lse = mx + np.log(np.exp(z - mx[:, None]).sum(axis=1))
    return float(np.mean(lse - z[np.arange(len(y)), y]))


def gradients(m: MLP, X: np.ndarray, y: np.ndarray, bf16: bool = True) -> Dict[str, np.ndarray]:
    """Chain rule through the three layers. dz = (softmax(z) - onehot(y)) / B;
    a ReLU passes the gradient where its input was positive."""
    f = forward(m, X, bf16)
    B = X.shape[0]
    dz = softmax(f["z"])
    dz[np.arange(B), y] -= 1.0
    dz /= B
    dzq = _q(dz.astype(np.float32), bf16) if bf16 else dz
    g = {"W3": dzq.T @ f["h2q"], "b3": dz.sum(axis=0)}
    dh2 = dzq @ _q(m.W3, bf16)
    da2 = dh2 * (f["a2"] > 0)
    da2q = _q(da2.astype(np.float32), bf16) if bf16 else da2
    g["W2"] = da2q.T @ f["h1q"]
    g["b2"] = da2.sum(axis=0)
    dh1 = da2q @ _q(m.W2, bf16)
    da1 = dh1 * (f["a1"] > 0)
    da1q = _q(da1.astype(np.float32), bf16) if bf16 else da1
    g["W1"] = da1q.T @ f["Xq"]
    g["b1"] = da1.sum(axis=0)
    return g


@dataclass
class AdamW:
    """Adam with decoupled weight decay (Loshchilov & Hutter): per parameter
    m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
    w <- w - lr * (m / (1-b1^t) / (sqrt(v / (1-b2^t)) + eps) + wd * w)."""

    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    wd: float = 0.0
    t: int = 0
    m: Dict[str, np.ndarray] = field(default_factory=dict)
    v: Dict[str, np.ndarray] = field(default_factory=dict)

    def step(self, model: MLP, grads: Dict[str, np.ndarray]) -> None:
        self.t += 1
        c1 = 1.0 - self.beta1 ** self.t
        c2 = 1.0 - self.beta2 ** self.t
        for k in LAYERS:
            w = getattr(model, k).astype(np.float64)
            gk = grads[k].astype(np.float64)
            mk = self.m.get(k, np.zeros_like(w))
            vk = self.v.get(k, np.zeros_like(w))
            mk = self.beta1 * mk + (1 - self.beta1) * gk
            vk = self.beta2 * vk + (1 - self.beta2) * gk * gk
            self.m[k], self.v[k] = mk, vk
            w = w - self.lr * ((mk / c1) / (np.sqrt(vk / c2) + self.eps) + self.wd * w)
            setattr(model, k, w.astype(np.float32))


def top_p(z: np.ndarray, P: int):
    """The P largest logits per row (ties: smaller index first), their ids,
    and the largest softmax probability (used to decide the fallback)."""
    order = np.lexsort((np.broadcast_to(np.arange(z.shape[1]), z.shape), -z), axis=1)[:, :P]
    p_max = 1.0 / np.exp(z - z.max(axis=1, keepdims=True)).sum(axis=1)
    return order.astype(np.uint32), p_max


def input_norm_stats(X: np.ndarray):
    """Per-dimension standardisation of training queries, written out as its
    definition in FP64: mean_j = (1/n) sum_i x_ij; std_j = sqrt((1/n) sum_i
    (x_ij - mean_j)^2) (population standard deviation); a floor of 1e-6 times
    the largest std (at least 1e-30) keeps constant dimensions finite;
    inv_std_j = 1 / max(std_j, floor). Returns (mean, inv_std) rounded to
    FP32, the precision the network applies them in."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    mean = X.sum(axis=0) / n
    dev = X - mean[None, :]
    std = np.sqrt((dev * dev).sum(axis=0) / n)
    floor = 1e-6 * max(float(std.max()), 1e-30)
    inv_std = 1.0 / np.maximum(std, floor)
    return mean.astype(np.float32), inv_std.astype(np.float32)


def lower_quantile(values: np.ndarray, q: float) -> float:
    """The fallback threshold tau: the value at 0-based position
    floor(min(q, 1) * (n - 1)) of the values sorted ascending (the "lower"
    quantile: no interpolation, always one of the values); 0 when there are
    no values or q <= 0 (nothing falls back)."""
    v = np.asarray(values, dtype=np.float32).ravel()
    if v.size == 0 or q <= 0.0:
        return 0.0
    pos = int(np.floor(min(float(q), 1.0) * (v.size - 1)))
    return float(np.sort(v, kind="stable")[pos])

