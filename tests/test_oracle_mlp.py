"""Pins of the triage-network oracle (oracle/mlp.py) against mathematics it
does not itself compute: central finite differences of the FP64 network,
the linear special case (all ReLUs active) collapsed to one affine map,
positive homogeneity, Adam's closed-form first steps, and the bfloat16
rounding rule against PyTorch's own conversion."""
import numpy as np
import pytest

from oracle import mlp as M

NIN = 6


def _random_net(rng, nin=NIN, scale=0.2):
    H = M.HIDDEN
    W1 = rng.normal(0, scale, (H, nin))
    b1 = rng.normal(0, 0.1, H)
    W2 = rng.normal(0, scale / 4, (H, H))
    b2 = rng.normal(0, 0.1, H)
    w3 = rng.normal(0, scale, H)
    return M.pack(W1, b1, W2, b2, w3, 0.3)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = _random_net(rng)
    x = rng.normal(0, 1, (5, NIN))
    t = rng.normal(-8, 2, 5)
    mu, sig = rng.normal(0, 0.1, NIN), rng.uniform(0.5, 2, NIN)
    my, sy = -7.0, 1.5
    loss, g = M.loss_and_grad(theta, x, t, NIN, mu, sig, my, sy, bf16_storage=False)
    # parameters sampled from every block: W1, b1, W2, b2, w3, b3
    n = M.nparams(NIN)
    H = M.HIDDEN
    starts = np.cumsum([0, H * NIN, H, H * H, H, H])
    idx = np.concatenate([rng.integers(s, e, 40) for s, e in zip(starts, list(starts[1:]) + [n])] + [[n - 1]])
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (M.loss_and_grad(tp, x, t, NIN, mu, sig, my, sy, False)[0] -
              M.loss_and_grad(tm, x, t, NIN, mu, sig, my, sy, False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_all_relus_active_is_one_affine_map():
    """Non-negative weights and inputs with positive biases keep every ReLU
    active, so the network collapses to y = (w3^T W2 W1) x + w3^T (W2 b1 + b2) + b3."""
    rng = np.random.default_rng(2)
    H = M.HIDDEN
    W1 = rng.uniform(0, 0.3, (H, NIN))
    b1 = rng.uniform(0.1, 0.2, H)
    W2 = rng.uniform(0, 0.05, (H, H))  # not symmetric
    b2 = rng.uniform(0.1, 0.2, H)
    w3 = rng.normal(0, 0.1, H)
    theta = M.pack(W1, b1, W2, b2, w3, -0.7)
    x = rng.uniform(0, 2, (7, NIN))
    y, _ = M.forward(theta, x, NIN, np.zeros(NIN), np.ones(NIN), bf16_storage=False)
    a = w3 @ W2 @ W1
    c = w3 @ (W2 @ b1 + b2) - 0.7
    assert np.allclose(y, x @ a + c, rtol=1e-12, atol=1e-12)


def test_positive_homogeneity_without_biases():
    rng = np.random.default_rng(3)
    H = M.HIDDEN
    theta = M.pack(rng.normal(0, 0.3, (H, NIN)), np.zeros(H), rng.normal(0, 0.1, (H, H)), np.zeros(H),
                   rng.normal(0, 0.3, H), 0.0)
    x = rng.normal(0, 1, (9, NIN))
    one = np.ones(NIN)
    y1, _ = M.forward(theta, x, NIN, 0 * one, one, False)
    y3, _ = M.forward(theta, 3.0 * x, NIN, 0 * one, one, False)
    assert np.allclose(y3, 3.0 * y1, rtol=1e-12, atol=1e-12)
    # and the input normalisation: x -> (x - mu) / sigma
    mu, sig = rng.normal(0, 1, NIN), rng.uniform(0.5, 2, NIN)
    yn, _ = M.forward(theta, x * sig + mu, NIN, mu, sig, False)
    assert np.allclose(yn, y1, rtol=1e-10, atol=1e-12)


def test_adam_closed_form_for_a_constant_gradient():
    """From m = v = 0 with a constant gradient g, every bias-corrected Adam
    step moves each parameter by lr * g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    theta = rng.normal(0, 1, 50)
    g = rng.normal(0, 1e-2, 50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr, eps = 1e-3, 1e-8
    th = theta.copy()
    for step in range(1, 6):
        th, m, v = M.adam(th, m, v, g, step, lr, eps=eps)
        assert np.allclose(th, theta - step * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-12)


def test_bf16_rounding_rule():
    one = 1.0
    assert M.bf16(one) == 1.0
    assert M.bf16(1 + 2.0 ** -7) == 1 + 2.0 ** -7          # representable
    assert M.bf16(1 + 2.0 ** -8) == 1.0                    # tie -> even
    assert M.bf16(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6      # tie -> even (upwards)
    assert M.bf16(1 + 2.0 ** -8 + 2.0 ** -20) == 1 + 2.0 ** -7
    assert M.bf16(-2.5) == -2.5 and M.bf16(0.0) == 0.0
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.normal(0, 10, 20000), rng.normal(0, 1e-3, 20000),
                        (rng.integers(-2 ** 15, 2 ** 15, 5000) * 2.0 ** -15 + 2.0 ** -24)])
    v32 = v.astype(np.float32)
    ref = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(M.bf16(v32), ref)


def test_bf16_storage_is_a_small_perturbation_of_the_fp64_network():
    rng = np.random.default_rng(6)
    theta = _random_net(rng)
    x = rng.normal(0, 1, (64, NIN))
    t = rng.normal(-8, 2, 64)
    one = np.ones(NIN)
    y0, _ = M.forward(theta, x, NIN, 0 * one, one, False)
    y1, _ = M.forward(theta, x, NIN, 0 * one, one, True)
    assert np.abs(y1 - y0).max() <= 2e-2 * np.abs(y0).max()
    l0, g0 = M.loss_and_grad(theta, x, t, NIN, 0 * one, one, -8.0, 2.0, False)
    l1, g1 = M.loss_and_grad(theta, x, t, NIN, 0 * one, one, -8.0, 2.0, True)
    assert abs(l1 - l0) <= 5e-2 * l0
    assert g0 @ g1 >= 0.99 * np.linalg.norm(g0) * np.linalg.norm(g1)
