"""Pins of the FP64 MLP reference (oracle side) to central finite differences."""
import numpy as np

from oracle import mlp_ref


def test_gelu_grad_matches_fd():
    z = np.linspace(-6, 6, 97)
    d = 1e-6
    fd = (mlp_ref.gelu(z + d) - mlp_ref.gelu(z - d)) / (2 * d)
    np.testing.assert_allclose(mlp_ref.gelu_grad(z), fd, rtol=1e-7, atol=1e-8)
    # GELU(z) = z Phi(z): limits
    assert abs(mlp_ref.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    assert abs(mlp_ref.gelu(np.array([-10.0]))[0]) < 1e-12


def test_loss_gradient_matches_fd():
    rng = np.random.default_rng(3)
    D, B = 7, 11
    params = mlp_ref.init_params(D, H=128, seed=2)
    xs = rng.standard_normal((B, D))
    ts = rng.standard_normal((B, 2))
    L, g = mlp_ref.loss_and_grad(params, xs, ts)
    flat = mlp_ref.flatten(params)
    gflat = mlp_ref.flatten(g)
    idx = rng.choice(flat.size, 60, replace=False)
    for i in idx:
        e = 1e-5 * max(1.0, abs(flat[i]))
        fp, fm = flat.copy(), flat.copy()
        fp[i] += e
        fm[i] -= e
        Lp, _ = mlp_ref.loss_and_grad(mlp_ref.unflatten(fp, D), xs, ts)
        Lm, _ = mlp_ref.loss_and_grad(mlp_ref.unflatten(fm, D), xs, ts)
        fd = (Lp - Lm) / (2 * e)
        assert abs(fd - gflat[i]) <= 1e-6 * max(abs(fd), 1e-3), (i, fd, gflat[i])


def test_gelu_special_values():
    """GELU(z) = z Phi(z): Phi(1) and Phi(-1) of the standard normal (tabulated values)."""
    z = np.array([0.0, 1.0, -1.0, 2.0])
    want = np.array([0.0, 0.8413447460685429, -0.15865525393145707, 2.0 * 0.9772498680518208])
    np.testing.assert_allclose(mlp_ref.gelu(z), want, rtol=1e-15, atol=1e-16)


def test_forward_reduces_to_bias_path():
    """With W1 = W2 = 0 every row's output is W3 GELU(b2) + b3, whatever the input."""
    D = 5
    p = mlp_ref.init_params(D, H=128, seed=4)
    p["W1"][:] = 0.0
    p["W2"][:] = 0.0
    xs = np.random.default_rng(0).standard_normal((3, D))
    out, _ = mlp_ref.forward(p, xs)
    want = p["W3"] @ mlp_ref.gelu(p["b2"]) + p["b3"]
    np.testing.assert_allclose(out, np.tile(want, (3, 1)), rtol=1e-14)


def test_adam_first_step_by_hand():
    """t = 1: the bias-corrected moments are g and g^2, so each entry with |g| >> eps
    moves by lr against the sign of its gradient; a zero gradient moves nothing."""
    w = np.array([0.5, -0.25, 1.0, 3.0])
    g = np.array([2.0, -1e-3, 0.0, 40.0])
    w1, m1, v1, t1 = mlp_ref.adam_step(w, g, np.zeros(4), np.zeros(4), 0, lr=1e-2)
    assert t1 == 1
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)
    # lr g / (|g| + eps), by hand
    want = np.array([0.5 - 0.01 * 2.0 / (2.0 + 1e-8), -0.25 + 0.01 * 1e-3 / (1e-3 + 1e-8), 1.0,
                     3.0 - 0.01 * 40.0 / (40.0 + 1e-8)])
    np.testing.assert_allclose(w1, want, rtol=1e-15)


def test_adam_two_steps_by_hand():
    """g1 = 1, g2 = -1, lr 0.1, eps 0 (scalar, written out):
    step 1: m = 0.1, v = 0.001, m_hat = 1, v_hat = 1, w -= 0.1;
    step 2: m = 0.09 - 0.1 = -0.01, v = 0.000999 + 0.001 = 0.001999,
            m_hat = -0.01 / 0.19 = -1/19, v_hat = 0.001999 / 0.001999 = 1, w += 0.1 / 19."""
    w, m, v, t = np.array([2.0]), np.zeros(1), np.zeros(1), 0
    w, m, v, t = mlp_ref.adam_step(w, np.array([1.0]), m, v, t, lr=0.1, eps=0.0)
    np.testing.assert_allclose(w, [1.9], rtol=1e-15)
    w, m, v, t = mlp_ref.adam_step(w, np.array([-1.0]), m, v, t, lr=0.1, eps=0.0)
    np.testing.assert_allclose(m, [-0.01], rtol=1e-13)
    np.testing.assert_allclose(v, [0.001999], rtol=1e-13)
    np.testing.assert_allclose(w, [1.9 + 0.1 / 19.0], rtol=1e-14)
    assert t == 2
