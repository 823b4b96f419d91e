"""Pins for the MLP reference (oracle/mlp.py) against calculus and library routines."""
import numpy as np
import torch

from oracle import mlp
import synth


def test_bf16_rounding_matches_torch():
    x = np.concatenate([np.random.default_rng(0).standard_normal(5000) * 10.0,
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -0.0, 65504.0, 1e-30, 3.0e38]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0                 # tie goes to the even mantissa
    assert mlp.bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7


def test_features_layout():
    q = synth.packed(3, 77)
    X = mlp.features(q)
    assert X.shape == (3, 167)
    s = synth.packed_to_strings(q)
    for row, st in zip(X, s):
        assert row[:166].tolist() == [float(c) for c in st]
        assert row[166] == mlp.bf16(st.count("1") / 166.0)


def test_backward_matches_central_differences():
    # smooth loss (mean squared error) and no bf16 rounding: the gradient must match finite differences
    rng = np.random.default_rng(1)
    flat = mlp.init_params(3).astype(np.float64)
    packed = synth.packed(16, 78)
    t = rng.uniform(10, 30, 16)
    X = mlp.features(packed)

    def loss(f):
        y, _ = mlp.forward(mlp.unflatten(f), X, round_bf16=False)
        return float(np.mean((y - t) ** 2))

    y, cache = mlp.forward(mlp.unflatten(flat), X, round_bf16=False)
    g = mlp.flatten(mlp.backward(cache, 2.0 * (y - t) / len(t)))
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    for gi, (name, _) in enumerate(mlp.SHAPES):
        idx = rng.choice(np.arange(offs[gi], offs[gi + 1]), size=min(12, offs[gi + 1] - offs[gi]), replace=False)
        for i in idx:
            h = 1e-5 * max(1.0, abs(flat[i]))
            fp, fm = flat.copy(), flat.copy()
            fp[i] += h
            fm[i] -= h
            fd = (loss(fp) - loss(fm)) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (name, i, fd, g[i])


def test_pinball_gradient_and_value():
    y = np.array([1.0, 2.0, 3.0, 4.0])
    t = np.array([2.5, 1.0, 3.5, 0.0])
    q = 0.9
    # hand values: residuals 1.5, -1, 0.5, -4 -> 0.9*1.5, 0.1*1, 0.9*0.5, 0.1*4
    assert np.isclose(mlp.pinball(y, t, q), (1.35 + 0.1 + 0.45 + 0.4) / 4)
    g = mlp.pinball_grad(y, t, q)
    for i in range(4):
        e = np.zeros(4)
        e[i] = 1e-6
        fd = (mlp.pinball(y + e, t, q) - mlp.pinball(y - e, t, q)) / 2e-6
        assert np.isclose(fd, g[i], atol=1e-6)


def test_forward_tiny_network_by_hand():
    p = {n: np.zeros(s) for n, s in mlp.SHAPES}
    p["W1"][0, 166] = 2.0          # h1_0 = relu(2 * popc/166 + 1)
    p["b1"][0] = 1.0
    p["W1"][1, 5] = -3.0           # h1_1 = relu(-3 * bit5) = 0
    p["W2"][0, 0] = 0.5            # h2_0 = relu(0.5 * h1_0)
    p["w3"][0] = 4.0
    p["b3"][0] = -1.0
    q = np.zeros((1, 3), np.uint64)
    q[0, 0] = np.uint64(0b100000)  # key 5 set, popc = 1
    X = mlp.features(q)
    y, _ = mlp.forward(p, X, round_bf16=False)
    pc = mlp.bf16(1 / 166.0)
    assert np.isclose(y[0], 4.0 * 0.5 * (2.0 * pc + 1.0) - 1.0)


def test_adam_first_step_is_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3, 0.0], np.float32)
    p0 = np.ones(4, np.float32)
    p1, m, v = mlp.adam(p0, g, np.zeros(4), np.zeros(4), step=1, lr=0.01)
    want = p0 - 0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(p1, want, atol=1e-7)
