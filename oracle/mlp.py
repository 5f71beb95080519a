"""Float64 NumPy oracle of the per-level variant selector -- TEST INFRASTRUCTURE ONLY.

The paper chooses between two SpMSV algorithms (sparse accumulator or heap
merge) by concurrency (Sec. 4.2, "a polyalgorithm"); the library generalises
that choice to a per-level pick among four expansion variants made by a small
network.  The paper fixes none of its details, so this module states them:

  - network: 12 inputs -> 64 (ReLU) -> 64 (ReLU) -> 4 outputs, float parameters
    packed flat in the order W1[12][64], b1[64], W2[64][64], b2[64], W3[64][4],
    b3[4] (row-major, 5,252 values);
  - outputs: predicted log2 of each variant's level time in microseconds; the
    selector picks the argmin;
  - loss: mean squared error over the batch and the four outputs;
  - initialisation: He-uniform, W = (2u - 1) * sqrt(6 / fan_in) from uniforms
    u in [0, 1) supplied by the caller, biases zero;
  - optimiser: Adam (Kingma and Ba 2015) with bias correction.

It shares no code with the CUDA kernels; only tests and the benchmark import it.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 12, 64, 4
SHAPES = [("W1", (N_IN, N_H)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_H, N_OUT)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 5252


def unpack(flat: np.ndarray) -> dict:
    """Views of the six parameter blocks inside a flat vector."""
    out, off = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = flat[off:off + size].reshape(shape)
        off += size
    assert off == flat.shape[0] == N_PARAMS
    return out


def he_uniform_init(u: np.ndarray) -> np.ndarray:
    """Parameters from N_PARAMS uniforms in [0, 1): weights He-uniform, biases 0."""
    flat = np.zeros(N_PARAMS, dtype=np.float64)
    p = unpack(flat)
    uu = unpack(np.asarray(u, dtype=np.float64))
    for name, _ in SHAPES:
        if name.startswith("W"):
            fan_in = p[name].shape[0]
            p[name][...] = (2.0 * uu[name] - 1.0) * np.sqrt(6.0 / fan_in)
    return flat


def forward(flat: np.ndarray, X: np.ndarray):
    """Returns (Y [B,4], cache) of the network on inputs X [B,12]."""
    p = unpack(np.asarray(flat, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    Y = h2 @ p["W3"] + p["b3"]
    return Y, (X, z1, h1, z2, h2)


def mse_loss(Y: np.ndarray, T: np.ndarray) -> float:
    return float(np.mean((Y - np.asarray(T, dtype=np.float64)) ** 2))


def backward(flat: np.ndarray, cache, dY: np.ndarray) -> np.ndarray:
    """Gradient of sum(dY * Y) with respect to the flat parameters (chain rule)."""
    p = unpack(np.asarray(flat, dtype=np.float64))
    X, z1, h1, z2, h2 = cache
    g = np.zeros(N_PARAMS, dtype=np.float64)
    gp = unpack(g)
    gp["W3"][...] = h2.T @ dY
    gp["b3"][...] = dY.sum(axis=0)
    dh2 = dY @ p["W3"].T
    dz2 = dh2 * (z2 > 0.0)
    gp["W2"][...] = h1.T @ dz2
    gp["b2"][...] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"].T
    dz1 = dh1 * (z1 > 0.0)
    gp["W1"][...] = X.T @ dz1
    gp["b1"][...] = dz1.sum(axis=0)
    return g


def loss_and_grad(flat: np.ndarray, X: np.ndarray, T: np.ndarray):
    """MSE loss and its gradient: dL/dY = 2 (Y - T) / (B * 4)."""
    Y, cache = forward(flat, X)
    T = np.asarray(T, dtype=np.float64)
    dY = 2.0 * (Y - T) / Y.size
    return mse_loss(Y, T), backward(flat, cache, dY)


def grad_scale(flat: np.ndarray, X: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Magnitude scale of each gradient entry: the chain rule of `loss_and_grad`
    evaluated on absolute values (weights, biases, inputs, hidden activations and
    the output error |Y| + |T|) with the ReLU masks of the exact evaluation.

    Every gradient entry is a sum of products; the rounding error of evaluating
    such an expression in floating point is bounded by a small multiple of the
    unit roundoff times the same expression with every operand replaced by its
    absolute value (Higham, "Accuracy and Stability of Numerical Algorithms",
    Ch. 3-4: |fl(sum x_i) - sum x_i| <= gamma_n sum |x_i|).  Where the terms
    cancel, the plain relative error is unbounded, so float32 results are
    compared with the float64 gradient relative to this scale.  It is never
    below |gradient|, and equals it when no term has a negative sign.
    """
    p = unpack(np.asarray(flat, dtype=np.float64))
    a = {k: np.abs(v) for k, v in p.items()}
    X = np.asarray(X, dtype=np.float64)
    Y, (_, z1, _, z2, _) = forward(flat, X)
    m1, m2 = z1 > 0.0, z2 > 0.0
    Xa = np.abs(X)
    h1 = np.where(m1, Xa @ a["W1"] + a["b1"], 0.0)
    h2 = np.where(m2, h1 @ a["W2"] + a["b2"], 0.0)
    dY = 2.0 * (np.abs(Y) + np.abs(np.asarray(T, dtype=np.float64))) / Y.size
    g = np.zeros(N_PARAMS, dtype=np.float64)
    gp = unpack(g)
    gp["W3"][...] = h2.T @ dY
    gp["b3"][...] = dY.sum(axis=0)
    dz2 = (dY @ a["W3"].T) * m2
    gp["W2"][...] = h1.T @ dz2
    gp["b2"][...] = dz2.sum(axis=0)
    dz1 = (dz2 @ a["W2"].T) * m1
    gp["W1"][...] = Xa.T @ dz1
    gp["b1"][...] = dz1.sum(axis=0)
    return g


def adam_step(flat, grad, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1; returns new (flat, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return flat - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ---------------- per-level features ----------------

FEATURE_BIN_EDGES = (32, 1024)  # degree <= 32 / <= 1024 / larger


def features(n: int, nnz: int, k: int, f_count: int, f_edges: int, unvisited: int,
             unvisited_edges: int, bin_counts) -> np.ndarray:
    """The 12 selector inputs of level k, each scaled to roughly [0, 1].

    log2 n / 32, log2 nnz / 32, log2(1 + k) / 10, log2(1 + |f|) / 32,
    log2(1 + sum deg f) / 32, |f| / n, sum deg f / nnz, unvisited / n,
    unvisited edges / nnz, and the fraction of frontier vertices with degree
    <= 32, <= 1024 and larger.
    """
    nn = max(n, 1)
    ne = max(nnz, 1)
    fc = max(f_count, 1)
    return np.array([
        np.log2(nn) / 32.0, np.log2(ne) / 32.0, np.log2(1.0 + k) / 10.0,
        np.log2(1.0 + f_count) / 32.0, np.log2(1.0 + f_edges) / 32.0,
        f_count / nn, f_edges / ne, unvisited / nn, unvisited_edges / ne,
        bin_counts[0] / fc, bin_counts[1] / fc, bin_counts[2] / fc,
    ], dtype=np.float64)
