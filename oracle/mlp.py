"""FP64 reference of the scoring network of the guided search -- TEST INFRASTRUCTURE ONLY.

The network (no counterpart in the paper): x = hist / n with n = sum(hist) the
number of processes (x = 0 for an all-zero row), h1 = relu(W1 x + b1),
h2 = relu(W2 h1 + b2), y = w3 . h2 + b3, loss = mean (y - label)^2, with the
parameter vector laid out W1 (128 x 16) | b1 | W2 (128 x 128) | b2 | w3 | b3.
Two forms are given.

* ``forward_reference`` is the network as defined: its weights W1, W2, w3
  are stored as bfloat16 (the parameter vector rounded once, as every kernel
  reads it), and everything else -- the features x = hist / n, both hidden
  layers and every sum -- is exact float64.  This is the FP64 reference the
  tensor-core scores are held to (within 1e-2 of the output's scale,
  ``output_scale``).
* ``forward`` / ``loss_and_grad`` with bf16=True are the arithmetic model of
  the tensor-core kernels, a second and tighter check of where they round.
  There both factors of every weight product are bfloat16 (the upper 16 bits
  of the IEEE binary32 pattern, round to nearest, ties to even), as on the
  tensor cores: the weights W1, W2, w3 are rounded, and so are x (from the
  binary32 product hist * (1 / n), both steps rounded to nearest in binary32)
  and h1 (from its binary32 value) before they enter their layers.  Everything
  else is float64.

Gradients are taken with respect to the unrounded parameters through the
rounded weights and activations (each rounding passes gradients unchanged),
which is what an optimiser on FP32 master weights sees.
"""
import numpy as np

IN, H = 16, 128
NPARAM = H * IN + H + H * H + H + H + 1


def bf16_round(a) -> np.ndarray:
    """float32 values rounded to the nearest bfloat16 (ties to even), as float32."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)


def unpack(p):
    p = np.asarray(p, dtype=np.float32)
    o = 0
    W1 = p[o:o + H * IN].reshape(H, IN); o += H * IN
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def _weights(p, bf16):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    if bf16:
        W1, W2, w3 = bf16_round(W1), bf16_round(W2), bf16_round(w3)
    f = lambda a: np.asarray(a, dtype=np.float64)
    return f(W1), f(b1), f(W2), f(b2), f(w3), float(b3)


def _act(z, bf16):
    """Layer input as the next product sees it: bfloat16 of its binary32 value."""
    return bf16_round(np.asarray(z, dtype=np.float32)).astype(np.float64) if bf16 else z


def features(hist, bf16=True):
    """x = hist / n, n = number of processes (row sum); 0 for an all-zero row."""
    h = np.asarray(hist, dtype=np.float64)
    n = h.sum(axis=1, keepdims=True)
    if not bf16:
        return np.divide(h, n, out=np.zeros_like(h), where=n > 0)
    inv = np.zeros(n.shape, dtype=np.float32)
    np.divide(np.float32(1), n.astype(np.float32), out=inv, where=n > 0)
    return bf16_round(h.astype(np.float32) * inv).astype(np.float64)


def forward(p, hist, bf16=True):
    W1, b1, W2, b2, w3, b3 = _weights(p, bf16)
    x = features(hist, bf16)
    a1 = x @ W1.T + b1
    z1 = _act(np.maximum(a1, 0), bf16)
    a2 = z1 @ W2.T + b2
    z2 = np.maximum(a2, 0)
    return z2 @ w3 + b3


def loss_and_grad(p, hist, label, bf16=True):
    W1, b1, W2, b2, w3, b3 = _weights(p, bf16)
    x = features(hist, bf16)
    t = np.asarray(label, dtype=np.float64)
    n = len(t)
    a1 = x @ W1.T + b1
    z1 = _act(np.maximum(a1, 0), bf16)
    a2 = z1 @ W2.T + b2
    z2 = np.maximum(a2, 0)
    y = z2 @ w3 + b3
    loss = np.mean((y - t) ** 2)
    dy = 2.0 * (y - t) / n
    gw3 = z2.T @ dy
    gb3 = dy.sum()
    d2 = np.outer(dy, w3) * (a2 > 0)
    gW2 = d2.T @ z1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (a1 > 0)
    gW1 = d1.T @ x
    gb1 = d1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return loss, g


def forward_reference(p, hist):
    """The scoring network by its definition: BF16 weights, float64 for the
    features (x = hist / n exactly, 0 for an all-zero row), the activations and
    every sum.  Returns (y, h2) with h2 the second hidden layer."""
    W1, b1, W2, b2, w3, b3 = _weights(p, True)
    x = features(hist, bf16=False)
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3, h2


def output_scale(p, h2):
    """Magnitude of the terms that sum to each output, sum_j |w3_j| h2_j + |b3|:
    the denominator of the relative error of a dot product, which stays
    meaningful when the terms cancel and the output itself is near zero."""
    _, _, _, _, w3, b3 = _weights(p, True)
    return np.asarray(h2, dtype=np.float64) @ np.abs(w3) + abs(b3)
