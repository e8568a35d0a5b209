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
