"""Pins of the FP64 reference MLP (oracle/mlp.py) against things that do not
depend on its own code: central finite differences of the loss, closed forms
of special networks, the definition of Adam's first step, and the
population standard deviation."""
import numpy as np
import pytest

from oracle import mlp

H = 8  # small width: finite differences over every parameter stay cheap


def _net(seed, H=H, scale=1.0):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, mlp.n_params(H))


def _batch(seed, B=7):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, (B, 5)), rng.normal(0, 1, (B, 2))


def test_parameter_count_of_the_256_wide_network():
    assert mlp.n_params(256) == 133_634


def test_gradient_matches_central_differences():
    """Every gradient entry against (L(p + e) - L(p - e)) / 2e in FP64."""
    flat = _net(1, scale=0.7)
    xh, th = _batch(2)
    _, g = mlp.loss_and_grad(mlp.unpack(flat, H), xh, th)
    gflat = mlp.pack(g, H)
    eps = 1e-6
    fd = np.empty_like(flat)
    for i in range(flat.size):
        e = np.zeros_like(flat)
        e[i] = eps
        lp = mlp.loss(mlp.forward(mlp.unpack(flat + e, H), xh)[0], th)
        lm = mlp.loss(mlp.forward(mlp.unpack(flat - e, H), xh)[0], th)
        fd[i] = (lp - lm) / (2 * eps)
    err = np.abs(gflat - fd)
    assert np.max(err) <= 1e-6 * max(1.0, np.max(np.abs(fd)))
    assert np.linalg.norm(gflat - fd) <= 1e-7 * np.linalg.norm(fd)


def test_zero_hidden_weights_give_the_closed_form():
    """With W1 = W2 = W3 = 0 every sample sees h3 = silu(b3), so
    yh = W4 silu(b3) + b4 whatever the input."""
    rng = np.random.default_rng(3)
    p = mlp.unpack(_net(3), H)
    for k in ("W1", "W2", "W3"):
        p[k][:] = 0.0
    xh, _ = _batch(4)
    yh, _ = mlp.forward(p, xh)
    b3 = p["b3"]
    want = p["W4"] @ (b3 / (1 + np.exp(-b3))) + p["b4"]
    assert np.allclose(yh, want[None, :], rtol=0, atol=1e-14)


def test_silu_values_and_derivative():
    z = np.linspace(-30, 30, 601)
    assert mlp.silu(np.array(0.0)) == 0.0
    assert mlp.silu_grad(np.array(0.0)) == 0.5
    assert abs(mlp.silu(np.array(30.0)) - 30.0) < 1e-11
    assert abs(mlp.silu(np.array(-30.0))) < 1e-11
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.silu_grad(z))) < 1e-8


def test_perfect_fit_has_zero_loss_and_gradient():
    p = mlp.unpack(_net(5), H)
    xh, _ = _batch(6)
    yh, _ = mlp.forward(p, xh)
    L, g = mlp.loss_and_grad(p, xh, yh)
    assert L == 0.0
    assert all(np.all(v == 0.0) for v in g.values())


def test_output_bias_gradient_closed_form():
    """dL/db4 = (1/B) sum_b (yh_b - th_b)."""
    p = mlp.unpack(_net(7), H)
    xh, th = _batch(8, B=11)
    yh, _ = mlp.forward(p, xh)
    _, g = mlp.loss_and_grad(p, xh, th)
    assert np.allclose(g["b4"], (yh - th).mean(axis=0), rtol=0, atol=1e-15)


def test_adam_first_step_is_a_signed_lr_step():
    """From m = v = 0 the bias-corrected first step is lr g / (|g| + eps)."""
    rng = np.random.default_rng(9)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    g[3] = 0.0
    new, m, v = mlp.adam(p, g, np.zeros(50), np.zeros(50), t=1, lr=1e-3)
    want = p - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.allclose(new, want, rtol=0, atol=1e-15)
    assert new[3] == p[3]
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_moves_lr_per_step():
    """A constant gradient keeps m_hat = g and v_hat = g^2 at every step t."""
    p = np.array([1.0, -2.0])
    g = np.array([0.3, -4.0])
    m = v = np.zeros(2)
    for t in range(1, 6):
        p, m, v = mlp.adam(p, g, m, v, t, lr=0.01, eps=0.0)
    assert np.allclose(p, [1.0 - 0.05, -2.0 + 0.05], rtol=0, atol=1e-13)


def test_ensemble_statistics_by_brute_force():
    """Mean and population std of identical members: std 0; of two members
    differing only in b4: half the difference times y_std."""
    f = _net(10)
    lo, hi = np.zeros(5), np.full(5, 2.0)
    x = np.random.default_rng(11).uniform(0, 2, (4, 5))
    mean, std = mlp.ensemble([f, f, f], x, lo, hi, [0.5, -1.0], [2.0, 3.0], H)
    yh, _ = mlp.forward(mlp.unpack(f, H), mlp.normalise_x(x, lo, hi))
    assert np.allclose(mean, yh * [2.0, 3.0] + [0.5, -1.0], rtol=0, atol=1e-13)
    assert np.all(std == 0.0)
    f2 = f.copy()
    f2[-2:] += [0.4, -0.2]
    _, std2 = mlp.ensemble([f, f2], x, lo, hi, [0.0, 0.0], [2.0, 3.0], H)
    assert np.allclose(std2, [[0.4, 0.3]] * 4, rtol=0, atol=1e-13)


def test_input_normalisation_maps_the_box_to_minus_one_one():
    lo, hi = np.array([0, 0.01, 0.5, 0, 0.5]), np.array([6, 1, 6, 6, 10.0])
    assert np.allclose(mlp.normalise_x(lo, lo, hi), -1)
    assert np.allclose(mlp.normalise_x(hi, lo, hi), 1)
    assert np.allclose(mlp.normalise_x((lo + hi) / 2, lo, hi), 0)


def test_planted_mistake_is_caught_by_finite_differences(monkeypatch):
    """A dropped activation derivative in the backward pass (a plausible bug)
    fails the finite-difference comparison."""
    flat = _net(12, scale=0.7)
    xh, th = _batch(13)
    monkeypatch.setattr(mlp, "silu_grad", lambda z: np.ones_like(z))
    _, g = mlp.loss_and_grad(mlp.unpack(flat, H), xh, th)
    monkeypatch.undo()
    _, g_ok = mlp.loss_and_grad(mlp.unpack(flat, H), xh, th)
    assert np.linalg.norm(mlp.pack(g, H) - mlp.pack(g_ok, H)) > 1e-3 * np.linalg.norm(mlp.pack(g_ok, H))


def test_bf16_rounding_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(14)
    a = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 1000),
                        rng.uniform(-300, 300, 1000), [0.0, -0.0, 1.0, 2.0 ** -130]])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(a), ref)
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties go to the even 1.0;
    # 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6: even is 1 + 2^-6
    assert mlp.bf16(1 + 2.0 ** -8) == 1.0
    assert mlp.bf16(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6


def test_mixed_precision_network_stays_close_to_fp64():
    """The bfloat16-rounded network differs from the FP64 one by the
    bfloat16 unit roundoff (2^-9 relative) accumulated over three layers."""
    flat = _net(15, H=64, scale=0.2)
    xh, th = _batch(16, B=33)
    p = mlp.unpack(flat, 64)
    y64, _ = mlp.forward(p, xh)
    y16, _ = mlp.forward(p, xh, mixed=True)
    assert np.max(np.abs(y16 - y64)) <= 2e-2 * np.max(np.abs(y64))
    assert np.max(np.abs(y16 - y64)) > 0
    _, g64 = mlp.loss_and_grad(p, xh, th)
    _, g16 = mlp.loss_and_grad(p, xh, th, mixed=True)
    for k in g64:
        assert np.linalg.norm(g16[k] - g64[k]) <= 3e-2 * np.linalg.norm(g64[k]), k
