"""Pins of the selector network's oracle (oracle/mlp.py): bfloat16 rounding against
torch's conversion, the float32 fixed-order forward against a float64 forward,
backward against central finite differences of the loss, and a hand-computed path."""
import numpy as np
import pytest

from oracle import mlp as M


def test_bf16_rounding_matches_torch_and_hand_values():
    torch = pytest.importorskip("torch")
    # hand values: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> even (1.0);
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6 -> even (1 + 2^-6)
    assert M.bf16_round(np.float32(1 + 2.0 ** -8)) == np.float32(1.0)
    assert M.bf16_round(np.float32(1 + 3 * 2.0 ** -8)) == np.float32(1 + 2.0 ** -6)
    x = np.random.default_rng(1).standard_normal(10000).astype(np.float32) * 7
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(M.bf16_round(x), want)


def test_forward32_close_to_float64_forward():
    p = M.init_params(3)
    x = np.random.default_rng(2).standard_normal((64, M.N_IN)).astype(np.float32)
    out32 = M.forward32(p, x)
    h1 = np.maximum(x.astype(np.float64) @ p["W1"].T.astype(np.float64) + p["b1"], 0)
    h2 = np.maximum(h1 @ p["W2"].T.astype(np.float64) + p["b2"], 0)
    out64 = h2 @ p["W3"].T.astype(np.float64) + p["b3"]
    assert np.max(np.abs(out32 - out64)) <= 1e-4 * max(1.0, np.max(np.abs(out64)))


def test_hand_computed_path():
    p = {k: np.zeros(M.SHAPES[k], dtype=np.float32) for k in M.ORDER}
    p["W1"][0, 3] = 2.0   # h1[0] = relu(2 x3 - 1)
    p["b1"][0] = -1.0
    p["W2"][5, 0] = 0.5   # h2[5] = relu(0.5 h1[0])
    p["W3"][7, 5] = -4.0  # out[7] = -4 h2[5] + 0.25
    p["b3"][7] = 0.25
    x = np.zeros((2, M.N_IN), dtype=np.float32)
    x[0, 3] = 3.0         # h1 = 5, h2 = 2.5, out7 = -9.75
    x[1, 3] = 0.25        # h1 = relu(-0.5) = 0 -> out7 = 0.25
    out = M.forward32(p, x)
    assert out[0, 7] == np.float32(-9.75) and out[1, 7] == np.float32(0.25)
    assert np.all(out[:, :7] == 0)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(4)
    p = {k: v.astype(np.float64) for k, v in M.init_params(5).items()}
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(M.SHAPES[k]) * 0.1
    x = rng.standard_normal((32, M.N_IN))
    mode = rng.integers(0, M.N_MODES, size=32)
    sizes = rng.random((32, 1))
    _, g = M.loss_and_grads(p, x, mode, sizes)
    h = 1e-6
    for k in M.ORDER:
        flat = p[k].ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = M.loss_only(p, x, mode, sizes)
            flat[idx] = old - h
            lm = M.loss_only(p, x, mode, sizes)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].ravel()[idx]) <= 1e-6 + 1e-5 * abs(fd), (k, idx)


def test_plain_gradient_descent_reduces_the_loss():
    rng = np.random.default_rng(6)
    p = {k: v.astype(np.float64) for k, v in M.init_params(7).items()}
    x = rng.standard_normal((256, M.N_IN))
    mode = np.where(x[:, 0] > 0, 6, 3)  # a separable rule
    sizes = (0.4 + 0.1 * np.tanh(x[:, 1]))[:, None]
    l0, _ = M.loss_and_grads(p, x, mode, sizes)
    for _ in range(300):
        _, g = M.loss_and_grads(p, x, mode, sizes)
        for k in M.ORDER:
            p[k] -= 0.05 * g[k]
    l1, _ = M.loss_and_grads(p, x, mode, sizes)
    assert l1 < 0.5 * l0


def test_c_inference_equals_numpy_definition_bit_for_bit():
    import oracle as O

    rng = np.random.default_rng(11)
    for seed in range(3):
        p = M.init_params(seed)
        for k in ("b1", "b2", "b3"):
            p[k] = M.bf16_round(rng.standard_normal(M.SHAPES[k]).astype(np.float32) * 0.3)
        flat = M.flatten(p)
        x = rng.standard_normal((200, M.N_IN)).astype(np.float32)
        want = M.forward32(p, x)
        got = np.stack([O.mlp_forward_c(flat, row) for row in x])
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_decision_rule_margin_and_budget_edges():
    """Output layer weights zero: the logits and the budget are the biases b3, so the
    rule can be checked at its edges.  A trial mode's logit exactly 2 below the top one
    is a trial, and so is one whose float32 sum with 2 rounds up to the top; one float32
    step of the sum below is not.  A budget below half the current size fraction (input
    7) runs both trials whatever the logits say: equal to the half is not below.  C and
    numpy agree."""
    import oracle as O

    below1 = np.nextafter(np.float32(1), np.float32(0))  # 1 - 2^-24: + 2 rounds back to 3 in float32
    cases = [  # logits ZERO..PALETTE, budget, input 7, expected bits (1 SPLIT, 2 PALETTE)
        ([0, 0, 0, 3.0, 0, 1.0, 0], 0.3, 0.5, 1), ([0, 0, 0, 3.0, 0, below1, 0], 0.3, 0.5, 1),
        ([0, 0, 0, 3.0, 0, np.float32(1 - 2.0 ** -22), 0], 0.3, 0.5, 0),
        ([0, 0, 0, 3.0, 0, 0, 1.0], 0.3, 0.5, 2), ([0, 0, 0, 0, 0, 3.0, 3.0], 0.3, 0.5, 3),
        ([5.0, 0, 0, 0, 0, 3.0, 2.0], 0.3, 0.5, 1), ([0, 0, 8.0, 0, 0, 5.0, 5.0], 0.3, 0.5, 0),
        ([0, 0, 8.0, 0, 0, 5.0, 5.0], 0.25, 0.5, 0),
        ([0, 0, 8.0, 0, 0, 5.0, 5.0], np.nextafter(np.float32(0.25), np.float32(0)), 0.5, 3),
        ([0, 0, 8.0, 0, 0, 5.0, 5.0], 0.1, 0.5, 3), ([0, 0, 8.0, 0, 0, 5.0, 5.0], 0.1, 0.2, 0),
        ([1.0] * 7, 0.9, 0.5, 3),
    ]
    for b, budget, x7, want in cases:
        p = M.init_params(0)
        p["W3"] = np.zeros_like(p["W3"])
        p["b3"] = np.array(list(b) + [budget], dtype=np.float32)
        x = np.zeros((1, M.N_IN), dtype=np.float32)
        x[0, 7] = x7
        assert M.trials(p, x)[0] == want, (b, budget)
        assert O.mlp_trials_c(M.flatten(p), x[0]) == want, (b, budget)


def test_features_c_equal_python_definition():
    import oracle as O
    from paper_1911_04034_gb300 import circuits as Cc

    rng = np.random.default_rng(12)
    for kc in (3, 6, 10):
        A = 1 << kc
        a = rng.standard_normal(A) + 1j * rng.standard_normal(A)
        few = np.resize(np.array([0.5, -0.5, 0.25]), A) + 0j
        imgs = [O.encode_chunk(a, kc, 26), O.encode_chunk(np.zeros(A, complex), kc, 64),
                O.encode_chunk(a, kc, 26, force_mode=5), O.encode_chunk(few, kc, 26, force_mode=6, modes=O.ALL_MODES)]
        if kc >= 2:
            imgs.append(O.encode_chunk(np.tile(a[:2], A // 2), kc, 26, force_mode=2))
        for img in imgs:
            for g in (Cc.gate(2, Cc.H), Cc.gate(9, Cc.T, {1: 1}), Cc.gate(2, Cc.X), Cc.gate(7, Cc.SX)):
                for S in (64, 26):
                    want = M.features(img, kc, g["u"], int(g["target"]), S)
                    got = O.mlp_features_c(img, kc, g, S)
                    assert np.array_equal(got, want)
    img = O.encode_chunk(few, 10, 26, force_mode=6, modes=O.ALL_MODES)
    x = M.features(img, 10, Cc.X.ravel().view(np.float64), 3, 26)
    # PALETTE one-hot, k = 2 -> 2 / 16, palette size 4 (0.5, -0.5, 0.25 and the zero imaginary parts)
    assert x[6] == 1.0 and x[10] == np.float32(2 / 16) and x[9] == np.float32(4 / (64 * 2048))
    assert x[11] == 1.0 and x[12] == 0.0 and x[13] == 1.0 and x[14] == 1.0 and x[15] == np.float32(26 / 64)
