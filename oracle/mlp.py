"""FP64 CPU reference of the surrogate MLP (forward, backward, Adam, ensemble).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg are the only callers; the CUDA library and
its binding never import this module.

The network (the surrogate the sweep's solver results are fitted with; the
paper has no learned part, so the definitions here are the library's own):

    xh = 2 (x - lo) / (hi - lo) - 1                (5 inputs, box-normalised)
    h1 = silu(W1 xh + b1),  h2 = silu(W2 h1 + b2),  h3 = silu(W3 h2 + b3)
    yh = W4 h3 + b4                                 (2 outputs, standardised)
    y  = yh * y_std + y_mean                        (absorption, v_dc)

    silu(z) = z / (1 + exp(-z))
    loss    = (1 / (2 B)) sum_b sum_o (yh_bo - th_bo)^2,   th = (t - y_mean) / y_std

Weights are packed per member in the order W1 [H][5], b1 [H], W2 [H][H],
b2 [H], W3 [H][H], b3 [H], W4 [2][H], b4 [2] (133,634 values for H = 256).
Adam (Kingma & Ba, 2015) with bias correction:
    m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2
    p = p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
The ensemble mean and standard deviation are over members with divisor M
(population form).

Every function is plain numpy in float64, written from these definitions and
the chain rule; no blocking, fusion or reordering.
"""
from __future__ import annotations

import numpy as np

N_IN, N_OUT = 5, 2


def sizes(H: int = 256):
    """(name, shape) of every parameter tensor in packing order."""
    return [("W1", (H, N_IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
            ("W3", (H, H)), ("b3", (H,)), ("W4", (N_OUT, H)), ("b4", (N_OUT,))]


def n_params(H: int = 256) -> int:
    return sum(int(np.prod(s)) for _, s in sizes(H))


def unpack(flat: np.ndarray, H: int = 256) -> dict:
    out, o = {}, 0
    for name, shp in sizes(H):
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    assert o == flat.size
    return out


def pack(p: dict, H: int = 256) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in sizes(H)])


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    """d silu / dz = s (1 + z (1 - s)) with s = 1 / (1 + exp(-z))."""
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def normalise_x(x, lo, hi):
    x = np.asarray(x, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return 2.0 * (x - lo) / (hi - lo) - 1.0


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64:
    the float32 value's top 16 bits after adding 0x7fff plus the lowest kept
    bit (finite inputs)."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _id(a):
    return a


def forward(p: dict, xh: np.ndarray, mixed: bool = False):
    """Standardised outputs yh [B, 2] and the pre-activations / activations
    the backward pass needs.  mixed = True rounds what the tensor-core
    layers and the output layer read to bfloat16: the hidden activations
    h1, h2, h3 and the weights W2, W3 (all other arithmetic stays float64)."""
    r = bf16 if mixed else _id
    z1 = xh @ p["W1"].T + p["b1"]
    h1 = r(silu(z1))
    z2 = h1 @ r(p["W2"]).T + p["b2"]
    h2 = r(silu(z2))
    z3 = h2 @ r(p["W3"]).T + p["b3"]
    h3 = r(silu(z3))
    yh = h3 @ p["W4"].T + p["b4"]
    return yh, dict(xh=xh, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3)


def loss(yh, th):
    B = yh.shape[0]
    return 0.5 * np.sum((yh - th) ** 2) / B


def backward(p: dict, cache: dict, dyh: np.ndarray, mixed: bool = False) -> dict:
    """Gradients of every parameter given dL/dyh [B, 2] (chain rule, layer
    by layer from the output).  mixed = True also rounds the back-propagated
    pre-activation gradients dz3, dz2, dz1 and the weights W2, W3 to
    bfloat16, as the tensor-core path stores and reads them."""
    r = bf16 if mixed else _id
    g = {}
    g["W4"] = dyh.T @ cache["h3"]
    g["b4"] = dyh.sum(axis=0)
    dz3 = r((dyh @ p["W4"]) * silu_grad(cache["z3"]))
    g["W3"] = dz3.T @ cache["h2"]
    g["b3"] = dz3.sum(axis=0)
    dz2 = r((dz3 @ r(p["W3"])) * silu_grad(cache["z2"]))
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = r((dz2 @ r(p["W2"])) * silu_grad(cache["z1"]))
    g["W1"] = dz1.T @ cache["xh"]
    g["b1"] = dz1.sum(axis=0)
    return g


def loss_and_grad(p: dict, xh: np.ndarray, th: np.ndarray, mixed: bool = False):
    yh, cache = forward(p, xh, mixed)
    B = xh.shape[0]
    return loss(yh, th), backward(p, cache, (yh - th) / B, mixed)


def adam(flat, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step at step count t >= 1; returns (flat, m, v) as new arrays."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def init_member(seed: int, H: int = 256) -> np.ndarray:
    """Seeded initial weights: W ~ U(-sqrt(3 / fan_in), sqrt(3 / fan_in))
    (unit-variance pre-activations for unit-variance inputs), biases 0."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in sizes(H):
        if name.startswith("W"):
            lim = np.sqrt(3.0 / shp[1])
            p[name] = rng.uniform(-lim, lim, size=shp)
        else:
            p[name] = np.zeros(shp)
    return pack(p, H)


def ensemble(flats, x, lo, hi, y_mean, y_std, H: int = 256, mixed: bool = False):
    """Mean and population standard deviation over members of the
    de-standardised outputs, [B, 2] each."""
    xh = normalise_x(x, lo, hi)
    ys = []
    for f in flats:
        yh, _ = forward(unpack(f, H), xh, mixed)
        ys.append(yh * np.asarray(y_std) + np.asarray(y_mean))
    ys = np.stack(ys)
    mean = ys.mean(axis=0)
    std = np.sqrt(((ys - mean) ** 2).mean(axis=0))
    return mean, std
