"""Learned refinement flags: per-element features and a 3-layer MLP.

The paper remarks (Sec. 5) that a velocity-magnitude criterion only fires
once intensification has begun; the learned part predicts the paper's
refinement flags (Sec. 3.1, values -1 / 0 / +1) some steps ahead from the
current state so that adaptation can be scheduled less often.

Features of element e: the five state fields at the 27 points of the element
with reference coordinates in {-1, 0, 1}^3 (the element's polynomial
evaluated there; for even N these are nodes), each divided by a per-field
scale, plus the element's level: 5 * 27 + 1 = 136 values, ordered
feature[f * 27 + (a + 3 b + 9 c)] for the point (a, b, c), then the level.

Network: Linear(136, 128) - ReLU - Linear(128, 128) - ReLU - Linear(128, 3),
softmax over the classes (coarsen, keep, refine) = flags (-1, 0, +1).
Loss: class-weighted mean cross-entropy,
    L = sum_n w_{y_n} (-log p_{n, y_n}) / sum_n w_{y_n}.
Optimiser: Adam with bias correction.

Precision (`emulate=True`, the contract of the GPU kernels): inputs, weights
and the two hidden activations enter their products rounded to bfloat16
(round to nearest even); sums and everything else in float64 here.
Gradients are those of the loss as a function of the rounded values.

Test infrastructure only (see oracle/__init__.py).
"""
import numpy as np

from . import basis

SIZES = (136, 128, 128, 3)


def bf16(x):
    """Round float values to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def features(mesh, qG, scales):
    """(Ne, 136) features of every element from the global state qG (5, NG)."""
    qL = mesh.to_local(qG)                       # (5, Ne, P)
    n1 = mesh.N + 1
    H = basis.lagrange_eval(mesh.xi, np.array([-1.0, 0.0, 1.0]))   # (3, n1)
    T = np.einsum("ck,bj,ai->abcijk", H, H, H).reshape(27, n1 ** 3)
    # local index l = i + n1 (j + n1 k); reorder T's columns to that order
    idx = np.zeros(n1 ** 3, dtype=np.int64)
    for i in range(n1):
        for j in range(n1):
            for k in range(n1):
                idx[i + n1 * (j + n1 * k)] = (i * n1 + j) * n1 + k
    T = T[:, idx]
    # T rows are ordered (a, b, c) with a slowest; reorder to a + 3b + 9c
    order = np.array([a * 9 + b * 3 + c for c in range(3) for b in range(3) for a in range(3)])
    T = T[order]
    F = np.zeros((mesh.Ne, 136))
    for f in range(5):
        F[:, f * 27:(f + 1) * 27] = (qL[f] @ T.T) / scales[f]
    F[:, 135] = mesh.level
    return F


def init_params(seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    out = []
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        lim = 1.0 / np.sqrt(a)
        out += [rng.uniform(-lim, lim, size=(a, b)), np.zeros(b)]
    return out


def forward(params, X, emulate=True):
    W1, b1, W2, b2, W3, b3 = params
    r = bf16 if emulate else (lambda v: np.asarray(v, dtype=np.float64))
    Xr = r(X)
    Z1 = Xr @ r(W1) + b1
    H1 = np.maximum(Z1, 0.0)
    H1r = r(H1)
    Z2 = H1r @ r(W2) + b2
    H2 = np.maximum(Z2, 0.0)
    H2r = r(H2)
    Z3 = H2r @ r(W3) + b3
    Z = Z3 - Z3.max(axis=1, keepdims=True)
    P = np.exp(Z) / np.exp(Z).sum(axis=1, keepdims=True)
    return dict(Xr=Xr, Z1=Z1, H1r=H1r, Z2=Z2, H2r=H2r, Z3=Z3, P=P)


def loss(params, X, y, class_w, emulate=True):
    """y in {0, 1, 2} (= flag + 1)."""
    P = forward(params, X, emulate)["P"]
    w = np.asarray(class_w)[y]
    return float(np.sum(w * -np.log(P[np.arange(len(y)), y])) / np.sum(w))


def grads(params, X, y, class_w, emulate=True):
    W1, b1, W2, b2, W3, b3 = params
    r = bf16 if emulate else (lambda v: np.asarray(v, dtype=np.float64))
    c = forward(params, X, emulate)
    w = np.asarray(class_w)[y]
    dZ3 = c["P"].copy()
    dZ3[np.arange(len(y)), y] -= 1.0
    dZ3 *= (w / np.sum(w))[:, None]
    gW3 = c["H2r"].T @ dZ3
    gb3 = dZ3.sum(axis=0)
    dZ2 = (dZ3 @ r(W3).T) * (c["Z2"] > 0)
    gW2 = c["H1r"].T @ dZ2
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ r(W2).T) * (c["Z1"] > 0)
    gW1 = c["Xr"].T @ dZ1
    gb1 = dZ1.sum(axis=0)
    return [gW1, gb1, gW2, gb2, gW3, gb3]


def adam(params, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new params, m, v."""
    out_p, out_m, out_v = [], [], []
    for p, gi, mi, vi in zip(params, g, m, v):
        mi = beta1 * mi + (1 - beta1) * gi
        vi = beta2 * vi + (1 - beta2) * gi * gi
        mh = mi / (1 - beta1 ** t)
        vh = vi / (1 - beta2 ** t)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mi)
        out_v.append(vi)
    return out_p, out_m, out_v
