"""Oracle of the learned chunk-mode selector -- TEST INFRASTRUCTURE ONLY.

The network is not from the paper: for each chunk a gate is about to rewrite it
predicts the best chunk mode and a bit budget (the best image's size as a fraction of
the RAW size), from the chunk's current image header and the gate alone, so that the
trial encodes of SPLIT (Solution D, Section 4.2) and PALETTE run only where they may
pay.  The exhaustive trial of every mode stays the fallback and the judge of the
network's choices; the codec itself enforces the error bound, the network only picks
among lossless codings of the same truncated values.

Architecture: 16 inputs -> 32 (ReLU) -> 32 (ReLU) -> 8 outputs.  Outputs 0..6 are
logits over the chunk modes ZERO, CONST, PERIOD, STREAM, RAW, SPLIT, PALETTE; output 7
is the bit budget.  Weights are bfloat16 values.

Inference (what the simulator's decision depends on) is defined in float32 with a
fixed order: every unit sums its products over the inputs in index order, each
product and each sum rounded to float32 (no fused multiply-add), then adds its bias.
`forward32` implements exactly that.  Training uses float64 (`loss_and_grads`).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT, N_MODES = 16, 32, 8, 7
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


TRIAL_MARGIN = np.float32(2.0)


def trials(p: dict, x) -> np.ndarray:
    """The selector's decision per row: bit 0 runs the SPLIT trial, bit 1 the PALETTE
    trial; each iff that mode's logit plus a margin of 2 reaches the largest of the
    seven logits, and both when the bit budget (output 7) is below half the chunk's
    current size fraction (input 7) -- float32 sums and comparisons.  Both rules lean
    towards a trial (a missed one costs memory, a needless one only time); the budget
    rule catches a predicted collapse of the image that the mode logits may miss."""
    x = np.asarray(x, dtype=np.float32)
    out = forward32(p, x)
    mx = out[:, :N_MODES].max(axis=1)
    shrink = out[:, 7] < (x[:, 7] * np.float32(0.5)).astype(np.float32)
    split = ((out[:, 5] + TRIAL_MARGIN).astype(np.float32) >= mx) | shrink
    pal = ((out[:, 6] + TRIAL_MARGIN).astype(np.float32) >= mx) | shrink
    return split.astype(np.int64) | (pal.astype(np.int64) << 1)


def loss_and_grads(p: dict, x, mode, sizes, w_size: float = 1.0):
    """Mean over the rows of: softmax cross-entropy of the seven mode logits against
    the best mode, plus w_size * squared error of the bit budget (output 7) against the
    best image's size fraction (`sizes`, one per row).  float64 throughout; returns
    (loss, grads dict)."""
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
    diff = o[:, N_MODES:] - np.asarray(sizes, dtype=np.float64).reshape(B, N_OUT - N_MODES)
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


def features(image: bytes, kc: int, u, target: int, S_gate: int) -> np.ndarray:
    """The selector's 16 inputs (float32) for a chunk whose current image is `image`,
    about to be rewritten by the gate (matrix u, target) at S_gate bits: one-hot of the
    image mode (7), its size / RAW size, its S / 64, header word 3 / (64 N) (residual
    bits; the palette size for PALETTE), header byte 2 / 16, whether the gate matrix is
    real, diagonal, anti-diagonal, whether the target lies inside the chunk, S_gate / 64."""
    f32 = np.float32
    mode, S, b2 = image[0], image[1], image[2]
    w3 = int.from_bytes(image[12:16], "little")
    x = np.zeros(16, dtype=np.float32)
    if mode < 7:
        x[mode] = 1
    x[7] = f32(len(image)) / f32(16 + (16 << kc))
    x[8] = f32(S) / f32(64)
    x[9] = f32(w3) / f32(64 * (2 << kc))
    x[10] = f32(b2) / f32(16)
    u = [float(v) for v in u]
    x[11] = float(u[1] == 0 and u[3] == 0 and u[5] == 0 and u[7] == 0)
    x[12] = float(u[2] == 0 and u[3] == 0 and u[4] == 0 and u[5] == 0)
    x[13] = float(u[0] == 0 and u[1] == 0 and u[6] == 0 and u[7] == 0)
    x[14] = float(target < kc)
    x[15] = f32(S_gate) / f32(64)
    return x
