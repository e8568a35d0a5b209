"""FP64 reference of the per-cell cost / initial-step network (oracle side).

TEST INFRASTRUCTURE ONLY: the GPU's BF16 forward and backward kernels are
checked against this module, and this module is checked against central finite
differences of its own loss.

Network (a part the paper does not have; it predicts, per cell, the cost the
integrator will spend and the first accepted step it will take, from the
method's own logs):
  features  x = [T/1000, ln p, ln(Y_k + 1e-20) for k = 1..K]      (K + 2)
  standardise  xs = (x - mu_x) / sd_x                              (training-set statistics)
  h1 = GELU(W1 xs + b1), h2 = GELU(W2 h1 + b2), out = W3 h2 + b3    (128, 128, 2)
  targets   t = [ln substeps, ln h_first], standardised ts = (t - mu_t) / sd_t
  loss      L = 1/(2B) sum_b sum_o (out_bo - ts_bo)^2
GELU(z) = z Phi(z) with the standard normal CDF Phi (the exact form).

Optimizer: Adam (D. P. Kingma and J. Ba, "Adam: a method for stochastic
optimization", ICLR 2015, Algorithm 1), one step per call of ``adam_step``.
"""
from __future__ import annotations

import math

import numpy as np

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def _erf(z):
    from scipy.special import erf

    return erf(z)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / SQRT2))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def features(T, p, Y):
    T = np.asarray(T, dtype=np.float64)
    return np.concatenate([(T / 1000.0)[:, None], np.log(np.asarray(p))[:, None],
                           np.log(np.asarray(Y) + 1e-20)], axis=1)


def targets(substeps, h_first):
    return np.stack([np.log(np.maximum(np.asarray(substeps, dtype=np.float64), 1.0)),
                     np.log(np.asarray(h_first, dtype=np.float64))], axis=1)


def init_params(D, H=128, seed=0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    rng = np.random.default_rng(seed)
    def u(shape, fan):
        return rng.uniform(-1.0, 1.0, size=shape) / math.sqrt(fan)
    return {"W1": u((H, D), D), "b1": u(H, D), "W2": u((H, H), H), "b2": u(H, H),
            "W3": u((2, H), H), "b3": u(2, H)}


def forward(params, xs):
    z1 = xs @ params["W1"].T + params["b1"]
    h1 = gelu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = gelu(z2)
    out = h2 @ params["W3"].T + params["b3"]
    return out, (xs, z1, h1, z2, h2)


def loss_and_grad(params, xs, ts):
    """L and dL/dparams by the chain rule written out layer by layer."""
    B = xs.shape[0]
    out, (x, z1, h1, z2, h2) = forward(params, xs)
    r = out - ts
    L = 0.5 * np.sum(r * r) / B
    dout = r / B
    g = {"W3": dout.T @ h2, "b3": dout.sum(axis=0)}
    dz2 = (dout @ params["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ params["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return L, g


ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def flatten(params):
    return np.concatenate([np.asarray(params[k], dtype=np.float64).ravel() for k in ORDER])


def unflatten(vec, D, H=128):
    shapes = {"W1": (H, D), "b1": (H,), "W2": (H, H), "b2": (H,), "W3": (2, H), "b3": (2,)}
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(shapes[k]))
        out[k] = np.asarray(vec[o:o + n], dtype=np.float64).reshape(shapes[k])
        o += n
    return out


def adam_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in FP64 (Kingma & Ba 2015, Algorithm 1).

    ``t`` is the number of updates taken before this one; the moments m, v start at
    zero. Biased first and second moment estimates, their bias corrections by
    1 - beta^t, and the parameter step lr * m_hat / (sqrt(v_hat) + eps).
    Returns (w_new, m_new, v_new, t + 1); the inputs are not modified."""
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    t1 = t + 1
    m1 = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v1 = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m1 / (1.0 - beta1 ** t1)
    v_hat = v1 / (1.0 - beta2 ** t1)
    return w - lr * m_hat / (np.sqrt(v_hat) + eps), m1, v1, t1
