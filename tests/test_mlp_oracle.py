"""Pins of the FP64 surrogate-MLP reference: central finite differences of
the loss for every parameter tensor, the closed-form logit gradient
sigmoid(z) - y, an independent autograd implementation (torch, CPU, float64),
a hand-computed one-unit case, Adam's first step, and bfloat16 rounding."""
import numpy as np
import pytest

from oracle import mlp


def _small(seed=0, B=16, sizes=(5, 7, 6, 1)):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(rng, sizes)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    x = rng.standard_normal((B, sizes[0]))
    y = (rng.random(B) < 0.5).astype(float)
    return p, x, y


def test_gradients_match_finite_differences():
    p, x, y = _small()
    z, cache = mlp.forward(p, x)
    g = mlp.backward(p, cache, z, y)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[i]
            flat[i] = old + h
            lp = mlp.bce(mlp.forward(p, x)[0], y)
            flat[i] = old - h
            lm = mlp.bce(mlp.forward(p, x)[0], y)
            flat[i] = old
            assert abs((lp - lm) / (2 * h) - g[k].reshape(-1)[i]) < 1e-6, k


def test_logit_gradient_closed_form_and_one_unit_case():
    # one hidden unit per layer, hand-computed: x = 2, W1 = 0.5, W2 = 3, W3 = -1
    p = {"W1": np.array([[0.5]]), "b1": np.array([0.0]), "W2": np.array([[3.0]]), "b2": np.array([1.0]),
         "W3": np.array([[-1.0]]), "b3": np.array([0.25])}
    x = np.array([[2.0]])
    z, cache = mlp.forward(p, x)
    assert z[0] == pytest.approx(-(3.0 * 1.0 + 1.0) + 0.25)
    y = np.array([1.0])
    g = mlp.backward(p, cache, z, y)
    s = 1 / (1 + np.exp(-z[0]))
    assert g["b3"][0] == pytest.approx(s - 1.0)           # d/dz of BCE = sigmoid(z) - y
    assert g["W3"][0, 0] == pytest.approx((s - 1.0) * 4.0)  # h2 = 4
    assert g["W1"][0, 0] == pytest.approx((s - 1.0) * -1.0 * 3.0 * 2.0)


def test_gradients_match_independent_autograd():
    torch = pytest.importorskip("torch")
    p, x, y = _small(seed=3, B=32, sizes=(33, 16, 16, 1))
    z, cache = mlp.forward(p, x)
    g = mlp.backward(p, cache, z, y)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    tx = torch.tensor(x, dtype=torch.float64)
    ty = torch.tensor(y, dtype=torch.float64)
    h1 = torch.relu(tx @ tp["W1"] + tp["b1"])
    h2 = torch.relu(h1 @ tp["W2"] + tp["b2"])
    tz = (h2 @ tp["W3"] + tp["b3"])[:, 0]
    loss = torch.nn.functional.binary_cross_entropy_with_logits(tz, ty)
    loss.backward()
    assert abs(loss.item() - mlp.bce(z, y)) < 1e-12
    for k in p:
        assert np.max(np.abs(tp[k].grad.numpy() - g[k])) < 1e-12, k


def test_adam_first_step_moves_by_lr_times_sign():
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -0.1, 0.0])}
    mlp.adam(p, g, {}, lr=0.01)
    # first bias-corrected step is lr * g / (|g| + eps) = lr * sign(g)
    assert np.allclose(p["w"], [0.99, -1.99, 0.5], atol=1e-9)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 3.14159265, -1e-3, 0.0])
    r = mlp.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7  # tie to even, exact
    assert abs(r[3] - 3.140625) < 1e-12
    assert np.all(np.abs(r - v) <= np.abs(v) * 2 ** -8 + 1e-30)
