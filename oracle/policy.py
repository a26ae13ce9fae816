"""Plain numpy oracle of the actor-critic network that consumes the
observation stack (§4.1, "Network architecture").

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``'s CPU
legs, never by the product package; it shares no code with the CUDA path.

The network, as §4.1 states it:
- input: the stack of 4 frames in the paper's (4, 64, 32) orientation
  (frame, x, y), pixel values 0/1;
- conv1: 32 filters, kernel (8, 4), stride (4, 2)  -> 32 x 15 x 15;
- conv2: 64 filters, kernel 4, stride 2           -> 64 x 6 x 6;
- conv3: 64 filters, kernel 3, stride 1           -> 64 x 4 x 4;
- ReLU after every convolution; the features are flattened;
- actor head: one hidden layer of 256 units with ReLU, then the logits;
- critic head: one hidden layer of 256 units with ReLU, then the value.

Readings where §4.1 is silent (each also listed in the design notes):
- padding is VALID (no padding): the kernel/stride pairs then map 64 x 32
  to the square 15 x 15 grid;
- every layer has a bias; the flatten order is (channel, x, y);
- the actor has n_actions + 1 logits (the game's keys and the no-op, the
  environment's action indices 0..n_actions);
- actions are sampled from softmax(logits) by inverse CDF with one uniform
  number per instance and step.

``forward`` computes in float64. With ``storage="bf16"`` the weights of
the three convolutions and of the two hidden layers, and every stored
activation (the convolution outputs, which include the flattened
features), are rounded to bfloat16 (round to nearest even) first: the
storage precision of the tensor-core kernels. The output layers (wa2, wc2)
and all biases stay float32 values, as the kernels keep them; dot products
stay float64. Parameter names: w1 [32,4,8,4] (out, frame, kx, ky), b1 [32];
w2 [64,32,4,4], b2; w3 [64,64,3,3], b3; wa1 [256,1024], ba1; wa2 [L,256],
ba2 [L]; wc1 [256,1024], bc1; wc2 [256], bc2 (scalar).
"""
from __future__ import annotations

import numpy as np

CONV_SPECS = (  # (in channels, out channels, kernel (kx, ky), stride (sx, sy)), §4.1
    (4, 32, (8, 4), (4, 2)),
    (32, 64, (4, 4), (2, 2)),
    (64, 64, (3, 3), (1, 1)),
)
HIDDEN = 256
BF16_WEIGHTS = ("w1", "w2", "w3", "wa1", "wc1")   # stored in bfloat16 by the tensor-core kernels


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned
    as float64. Done on the float32 bit pattern: keep the top 16 bits after
    adding half of the dropped range (plus the kept lsb for ties)."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv_out(size: int, k: int, s: int) -> int:
    """Output length of a VALID convolution."""
    return (size - k) // s + 1


def conv2d_valid(x: np.ndarray, w: np.ndarray, b: np.ndarray, stride: tuple) -> np.ndarray:
    """x [n, C, X, Y], w [O, C, kx, ky], b [O] -> [n, O, X', Y'] with
    out[n, o, i, j] = b[o] + sum_{c, u, v} w[o, c, u, v] x[n, c, s_x i + u, s_y j + v]."""
    n, C, X, Y = x.shape
    O, C2, kx, ky = w.shape
    assert C == C2
    sx, sy = stride
    OX, OY = conv_out(X, kx, sx), conv_out(Y, ky, sy)
    out = np.empty((n, O, OX, OY), dtype=np.float64)
    wf = w.reshape(O, -1)
    for i in range(OX):
        for j in range(OY):
            patch = x[:, :, sx * i:sx * i + kx, sy * j:sy * j + ky].reshape(n, -1)
            out[:, :, i, j] = patch @ wf.T + b
    return out


def relu(a: np.ndarray) -> np.ndarray:
    return np.maximum(a, 0.0)


def to_paper_orientation(obs: np.ndarray) -> np.ndarray:
    """uint8 frames [n, 4, 32 (y), 64 (x)] -> float64 [n, 4, 64 (x), 32 (y)]."""
    return np.ascontiguousarray(np.transpose(obs, (0, 1, 3, 2))).astype(np.float64)


def forward(params: dict, obs: np.ndarray, storage: str = "f64", features: bool = False):
    """Logits [n, L] and value [n] of the network for observation stacks
    obs uint8 [n, 4, 32, 64] (values 0/1)."""
    q = bf16_round if storage == "bf16" else (lambda a: np.asarray(a, dtype=np.float64))
    p = {k: q(v) if k in BF16_WEIGHTS else np.asarray(v, dtype=np.float64) for k, v in params.items()}
    h = to_paper_orientation(obs)
    acts = []
    for li, (_, _, _, stride) in enumerate(CONV_SPECS, start=1):
        h = q(relu(conv2d_valid(h, p[f"w{li}"], p[f"b{li}"], stride)))
        acts.append(h)
    flat = h.reshape(h.shape[0], -1)                    # (channel, x, y) order
    ha = relu(flat @ p["wa1"].T + p["ba1"])
    hc = relu(flat @ p["wc1"].T + p["bc1"])
    logits = ha @ p["wa2"].T + p["ba2"]
    value = hc @ p["wc2"] + p["bc2"]
    if features:
        return logits, value, acts
    return logits, value


def sample(logits: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Inverse-CDF categorical draw: the smallest a with u < sum_{j<=a} p_j,
    p = softmax(logits) (float64); u in [0, 1) per row."""
    z = logits - logits.max(axis=1, keepdims=True)
    e = np.exp(z)
    cdf = np.cumsum(e / e.sum(axis=1, keepdims=True), axis=1)
    a = (u[:, None] >= cdf).sum(axis=1)
    return np.minimum(a, logits.shape[1] - 1).astype(np.uint8)


def cdf_margin(logits: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Distance of u from the nearest CDF boundary (where a draw could flip
    under a rounding difference of the logits)."""
    z = logits - logits.max(axis=1, keepdims=True)
    e = np.exp(z)
    cdf = np.cumsum(e / e.sum(axis=1, keepdims=True), axis=1)
    return np.abs(cdf - u[:, None]).min(axis=1)


def uniform_from_word(w: np.ndarray) -> np.ndarray:
    """u = (w >> 8) * 2^-24 for 32-bit words: 24 random bits, exact in float32."""
    return (np.asarray(w, dtype=np.uint64) >> 8).astype(np.float64) * 2.0 ** -24
