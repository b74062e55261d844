"""CPU reference of the ranking network (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline
use this module; the library never does.

The network scores a candidate's feature vector x (128 values):
    h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3),
    z = w4 . h3 + b4, p = sigmoid(z),
trained on the mean binary cross-entropy  L = mean(log(1 + e^z) - y z),
whose gradient with respect to z is (p - y) / n.  Backpropagation gives
    dz3 = (dL/dz) w4 * [h3 > 0],  dz_{l-1} = (W_l^T dz_l) * [h_{l-1} > 0],
    dW_l = dz_l h_{l-1}^T,  db_l = sum over rows of dz_l,
    dw4 = sum_r (dL/dz_r) h3_r,  db4 = sum_r dL/dz_r.

``adam_step`` is the optimiser's update in float64.

``bf16=True`` rounds to bfloat16 (round to nearest even) exactly where the
GPU kernels store BF16: the features, the weight copies W1..W3 and w4, each
h_l, and each dz_l.  Biases, sums and the loss stay in the working precision
(``dtype``).  ``bf16=False, dtype=float64`` is the plain mathematics above,
which the finite-difference tests pin.

Parameter layout (flat, as the library's): W1[256][128] b1[256] W2[256][256]
b2[256] W3[256][256] b3[256] w4[256] b4.
"""
from __future__ import annotations

import numpy as np

IN, HID = 128, 256
SIZES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
         ("W3", (HID, HID)), ("b3", (HID,)), ("w4", (HID,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def offsets() -> dict:
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = (o, o + n, shape)
        o += n
    return out


def unpack(p) -> dict:
    p = np.asarray(p)
    return {k: p[a:b].reshape(s) for k, (a, b, s) in offsets().items()}


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[k], dtype=np.float64).ravel() for k, _ in SIZES])


def bf16(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float32: keep the top 16 bits after adding half an ulp of bf16."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(a.shape)


def forward(p, X, bf16_points: bool = True, dtype=np.float32):
    """Scores and the cached activations of the rows of X."""
    P = unpack(p)
    rnd = (lambda v: bf16(v).astype(dtype)) if bf16_points else (lambda v: np.asarray(v, dtype=dtype))
    x = rnd(X)
    W = [rnd(P["W1"]), rnd(P["W2"]), rnd(P["W3"])]
    b = [np.asarray(P[k], dtype=dtype) for k in ("b1", "b2", "b3")]
    hs = [x]
    for l in range(3):
        z = hs[-1] @ W[l].T.astype(dtype) + b[l]
        hs.append(rnd(np.maximum(z, 0)))
    w4 = rnd(P["w4"])
    z = hs[3] @ w4 + np.asarray(P["b4"], dtype=dtype)[0]
    prob = 1.0 / (1.0 + np.exp(-z))
    return prob, dict(h=hs, W=W, w4=w4, z=z)


def loss_and_grad(p, X, y, bf16_points: bool = True, dtype=np.float32):
    """Mean binary cross-entropy of the rows of X with labels y and its
    gradient with respect to the flat parameter vector."""
    y = np.asarray(y, dtype=dtype)
    n = X.shape[0]
    prob, c = forward(p, X, bf16_points, dtype)
    z = c["z"]
    loss = np.mean(np.maximum(z, 0) + np.log1p(np.exp(-np.abs(z))) - y * z)
    rnd = (lambda v: bf16(v).astype(dtype)) if bf16_points else (lambda v: np.asarray(v, dtype=dtype))
    dl = (prob - y) / n                                  # dL/dz per row
    g = {"w4": dl @ c["h"][3], "b4": np.array([dl.sum()])}
    dz = rnd(np.outer(dl, c["w4"]) * (c["h"][3] > 0))  # dz3
    for l in (2, 1, 0):                                  # layers 3, 2, 1
        g[f"W{l + 1}"] = dz.T @ c["h"][l]
        g[f"b{l + 1}"] = dz.sum(axis=0)
        if l > 0:
            dz = rnd((dz @ c["W"][l]) * (c["h"][l] > 0))
    return float(loss), pack(g)


def adam_step(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba, "Adam: A Method for Stochastic
    Optimization", Algorithm 1), in float64: the moments decay by b1 and b2
    and take in g and g^2; each is divided by its bias correction 1 - b^t
    (t = 1 for the first update); the parameters move by lr times the
    corrected first moment over (square root of the corrected second moment
    + eps).  Returns the new (p, m, v)."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    m_hat = m / (1.0 - b1 ** t)
    v_hat = v / (1.0 - b2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def shuffle(n: int, seed: int) -> np.ndarray:
    """The training loop's row order for one epoch: a Fisher-Yates shuffle of
    0..n-1 (from the last position down, position i swapped with the one at
    splitmix64() mod (i + 1)), splitmix64 being Steele, Lea and Flood's
    generator (state advanced by 0x9E3779B97F4A7C15, then three xor-shift /
    multiply mixing rounds).  Returns the permutation and nothing of the
    network's arithmetic; a test uses it to feed the reference the rows in
    the order the library trains on them."""
    mask = (1 << 64) - 1
    state = seed & mask
    perm = list(range(n))
    for i in range(n - 1, 0, -1):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z ^= z >> 31
        j = z % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return np.asarray(perm, dtype=np.int64), state


def init_params(seed: int) -> np.ndarray:
    """Random parameters for tests (not the library's initialiser)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SIZES:
        fan = shape[-1] if len(shape) == 2 else HID
        d[name] = rng.uniform(-1, 1, size=shape) * (np.sqrt(6.0 / fan) if name[0] == "W" else 0.1)
    d["w4"] = rng.uniform(-1, 1, size=(HID,)) * np.sqrt(3.0 / HID)
    return pack(d)
