"""Oracle of the learned chunk-mode selector -- TEST INFRASTRUCTURE ONLY.

The network is not from the paper: it predicts, for each chunk a gate re-encodes,
whether the Solution D order (SPLIT, Section 4.2) is worth a trial encode, so the
exhaustive trial of Solution C and D can be replaced by one trial most of the time.
The codec itself enforces the error bound; the network only picks among lossless
re-orderings of the same truncated values.

Architecture: 16 inputs -> 32 (ReLU) -> 32 (ReLU) -> 8 outputs.  Outputs 0..5 are
logits over the chunk modes ZERO, CONST, PERIOD, STREAM, RAW, SPLIT; outputs 6 and 7
predict the STREAM and SPLIT image sizes as fractions of the RAW size.  Weights are
bfloat16 values.

Inference (what the simulator's decision depends on) is defined in float32 with a
fixed order: every unit sums its products over the inputs in index order, each
product and each sum rounded to float32 (no fused multiply-add), then adds its bias.
`forward32` implements exactly that.  Training uses float64 (`loss_and_grads`).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT, N_MODES = 16, 32, 8, 6
SHAPES = {"W1": (N_H, N_IN), "b1": (N_H,), "W2": (N_H, N_H), "b2": (N_H,), "W3": (N_OUT, N_H), "b3": (N_OUT,)}
ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).reshape(a.shape)


def init_params(seed: int) -> dict:
    """He-style random initialisation, rounded to bfloat16."""
    rng = np.random.default_rng(seed)
    p = {}
    for k in ORDER:
        shp = SHAPES[k]
        if k.startswith("W"):
            p[k] = bf16_round(rng.standard_normal(shp) * np.sqrt(2.0 / shp[1]))
        else:
            p[k] = np.zeros(shp, dtype=np.float32)
    return p


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float32).ravel() for k in ORDER])


def unflatten(v: np.ndarray) -> dict:
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = np.asarray(v[o:o + n], dtype=np.float32).reshape(SHAPES[k])
        o += n
    return out


N_PARAMS = sum(int(np.prod(s)) for s in SHAPES.values())


def _layer32(W, b, x):
    """float32, in input order, no fused multiply-add: acc = acc + W[:, i] * x[:, i]."""
    W = np.asarray(W, dtype=np.float32)
    acc = np.zeros((x.shape[0], W.shape[0]), dtype=np.float32)
    for i in range(W.shape[1]):
        acc = (acc + (x[:, i:i + 1] * W[None, :, i]).astype(np.float32)).astype(np.float32)
    return (acc + np.asarray(b, dtype=np.float32)[None, :]).astype(np.float32)


def forward32(p: dict, x) -> np.ndarray:
    """Outputs (float32) for feature rows x (float32), in the order that fixes decisions."""
    x = np.asarray(x, dtype=np.float32)
    z1 = _layer32(p["W1"], p["b1"], x)
    h1 = np.where(z1 > 0, z1, np.float32(0)).astype(np.float32)  # ReLU giving +0
    z2 = _layer32(p["W2"], p["b2"], h1)
    h2 = np.where(z2 > 0, z2, np.float32(0)).astype(np.float32)
    return _layer32(p["W3"], p["b3"], h2)


SPLIT_MARGIN = np.float32(2.0)


def wants_split(p: dict, x) -> np.ndarray:
    """The selector's decision: run the Solution D trial iff the SPLIT logit plus a
    margin of 2 reaches the largest mode logit (float32 sum and comparison).  The
    margin leans towards a trial: a missed SPLIT costs memory, a needless trial only
    time."""
    out = forward32(p, x)
    lifted = (out[:, 5] + SPLIT_MARGIN).astype(np.float32)
    return lifted >= out[:, :N_MODES].max(axis=1)


def loss_and_grads(p: dict, x, mode, sizes, w_size: float = 1.0):
    """Mean over the rows of: softmax cross-entropy of the mode logits against the best
    mode, plus w_size * squared error of outputs 6, 7 against the two size fractions.
    float64 throughout; returns (loss, grads dict)."""
    x = np.asarray(x, dtype=np.float64)
    B = x.shape[0]
    W1, b1 = p["W1"].astype(np.float64), p["b1"].astype(np.float64)
    W2, b2 = p["W2"].astype(np.float64), p["b2"].astype(np.float64)
    W3, b3 = p["W3"].astype(np.float64), p["b3"].astype(np.float64)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    o = h2 @ W3.T + b3
    lg = o[:, :N_MODES]
    m = lg.max(axis=1, keepdims=True)
    e = np.exp(lg - m)
    sm = e / e.sum(axis=1, keepdims=True)
    y = np.zeros_like(sm)
    y[np.arange(B), np.asarray(mode, dtype=np.int64)] = 1.0
    ce = -np.sum(y * np.log(sm + 1e-300)) / B
    diff = o[:, N_MODES:] - np.asarray(sizes, dtype=np.float64)
    mse = w_size * np.sum(diff * diff) / B
    do = np.zeros_like(o)
    do[:, :N_MODES] = (sm - y) / B
    do[:, N_MODES:] = 2.0 * w_size * diff / B
    gW3 = do.T @ h2
    gb3 = do.sum(axis=0)
    dh2 = do @ W3
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(axis=0)
    return ce + mse, {"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3}


def loss_only(p: dict, x, mode, sizes, w_size: float = 1.0) -> float:
    return loss_and_grads(p, x, mode, sizes, w_size)[0]


def zero_groups(values, kc: int) -> tuple[int, int, int]:
    """Splits the chunk's 2^kc amplitudes into G = min(2^kc, 256) equal groups and
    counts the groups whose real parts, and those whose imaginary parts, are all zero
    (+0 or -0).  Returns (real-zero groups, imaginary-zero groups, G)."""
    v = np.ascontiguousarray(values, dtype=np.complex128)
    A = 1 << kc
    G = min(A, 256)
    re = v.real.reshape(G, A // G)
    im = v.imag.reshape(G, A // G)
    return int(np.sum(np.all(re == 0, axis=1))), int(np.sum(np.all(im == 0, axis=1))), G


def features(prev_image: bytes, kc: int, u, target: int, S_gate: int, values) -> np.ndarray:
    """The selector's 16 inputs for one chunk about to be re-encoded (float32):
    one-hot of the previous image's mode (6), its size / RAW size, its S / 64, its
    residual bits / (64 N), whether the gate matrix is real, diagonal, a permutation,
    whether the target lies inside the chunk, the fraction of amplitude groups whose
    real parts are all zero, the gate's S / 64, and the fraction of groups whose
    imaginary parts are all zero.  `values` are the chunk's amplitudes after the gate."""
    f32 = np.float32
    mode, S = prev_image[0], prev_image[1]
    bits = int.from_bytes(prev_image[12:16], "little")
    zre, zim, G = zero_groups(values, kc)
    x = np.zeros(16, dtype=np.float32)
    x[mode] = 1
    x[6] = f32(len(prev_image)) / f32(16 + (16 << kc))
    x[7] = f32(S) / f32(64)
    x[8] = f32(bits) / f32(64 * (2 << kc))
    u = [float(v) for v in u]
    x[9] = float(u[1] == 0 and u[3] == 0 and u[5] == 0 and u[7] == 0)
    x[10] = float(u[2] == 0 and u[3] == 0 and u[4] == 0 and u[5] == 0)
    x[11] = float(u[0] == 0 and u[1] == 0 and u[6] == 0 and u[7] == 0)
    x[12] = float(target < kc)
    x[13] = f32(zre) / f32(G)
    x[14] = f32(S_gate) / f32(64)
    x[15] = f32(zim) / f32(G)
    return x
