"""FP64 reference of the learned Q' initial guess (test infrastructure).

The paper solves for Q' by Newton's method from the macroscopic state; the
learned guess is an addition of this project: a small network maps the
point's state to a correction Delta whose application gives the Newton
starting point.

Features x (9): rho, U_1..3, theta, the invariants of A = Pi/(rho theta)
  I1 = tr A, I2 = (tr(A)^2 - tr(A^2))/2, I3 = det A, and the local mean free
  path lambda = (mu/rho) sqrt(pi/(2 theta)) (the paper's definition).
Target Delta (5): rho'/rho - 1, (U' - U)/sqrt(theta), theta'/theta - 1.
Network: y = W3^T s(W2^T s(W1^T xn + b1) + b2) + b3 with s(z) = z sigmoid(z)
  (SiLU), widths 9 -> 64 -> 64 -> 5, xn = (x - x_mean)/x_std, and the output
  de-normalised as Delta = y * t_std + t_mean.
Loss: mean over the batch and the 5 outputs of (y - tn)^2, tn = (Delta - t_mean)/t_std.
"""
import numpy as np

from . import bgk

WIDTHS = (9, 64, 64, 5)


def features(m, gas):
    """x[P, 9] from raw moments m[P, 11] (slots as in oracle.bgk)."""
    rho, U, E, theta, pres, Pi = bgk.macroscopic(m, gas)
    A = Pi / (rho * theta)[:, None, None]
    tr = np.trace(A, axis1=1, axis2=2)
    tr2 = np.einsum("pij,pji->p", A, A)
    I2 = 0.5 * (tr * tr - tr2)
    I3 = np.linalg.det(A)
    mu = gas.viscosity(theta)
    lam = mu / rho * np.sqrt(np.pi / (2.0 * theta))
    return np.stack([rho, U[:, 0], U[:, 1], U[:, 2], theta, tr, I2, I3, lam], axis=1)


def target(m, qp, gas):
    """Delta[P, 5] from raw moments and the solved q' = (rho', U', theta')."""
    rho, U, E, theta, pres, Pi = bgk.macroscopic(m, gas)
    s = np.sqrt(theta)
    return np.stack([qp[:, 0] / rho - 1.0, (qp[:, 1] - U[:, 0]) / s, (qp[:, 2] - U[:, 1]) / s,
                     (qp[:, 3] - U[:, 2]) / s, qp[:, 4] / theta - 1.0], axis=1)


def guess(m, delta, gas):
    """q' guess from the state and a predicted Delta (inverse of target)."""
    rho, U, E, theta, pres, Pi = bgk.macroscopic(m, gas)
    s = np.sqrt(theta)
    return np.stack([rho * (1 + delta[:, 0]), U[:, 0] + s * delta[:, 1], U[:, 1] + s * delta[:, 2],
                     U[:, 2] + s * delta[:, 3], theta * (1 + delta[:, 4])], axis=1)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    sg = 1.0 / (1.0 + np.exp(-z))
    return sg * (1.0 + z * (1.0 - sg))


def init_params(seed, widths=WIDTHS):
    """He-style random weights (W[i] has shape [fan_in, fan_out]) and zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for a, b in zip(widths[:-1], widths[1:]):
        params.append(rng.standard_normal((a, b)) * np.sqrt(2.0 / a))
        params.append(np.zeros(b))
    return params


def forward(params, xn):
    """Returns (y, cache) for normalised inputs xn[B, 9]."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = xn @ W1 + b1
    h1 = silu(z1)
    z2 = h1 @ W2 + b2
    h2 = silu(z2)
    y = h2 @ W3 + b3
    return y, (xn, z1, h1, z2, h2)


def loss_and_grads(params, xn, tn):
    """MSE loss and its gradient w.r.t. every parameter (analytic backprop)."""
    W1, b1, W2, b2, W3, b3 = params
    y, (x, z1, h1, z2, h2) = forward(params, xn)
    n = y.size
    r = y - tn
    loss = float(np.sum(r * r) / n)
    dy = 2.0 * r / n
    gW3 = h2.T @ dy
    gb3 = dy.sum(axis=0)
    dh2 = dy @ W3.T
    dz2 = dh2 * silu_grad(z2)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2.T
    dz1 = dh1 * silu_grad(z1)
    gW1 = x.T @ dz1
    gb1 = dz1.sum(axis=0)
    return loss, [gW1, gb1, gW2, gb2, gW3, gb3]


def predict(params, norm, x):
    """Delta for raw features x: normalise, run the network, de-normalise."""
    x_mean, x_std, t_mean, t_std = norm
    y, _ = forward(params, (x - x_mean) / x_std)
    return y * t_std + t_mean


def bf16_round(x):
    """Nearest BF16 value (8 significant bits, ties to even) of each entry,
    taken from its FP32 rounding, as FP64.  The tensor cores and the BF16
    inference see layer inputs and weights in this format."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(params, xn, rnd=bf16_round):
    """The network with BF16 weights and layer inputs (normalised features and
    both hidden activations rounded with rnd), FP64 sums, exact biases:
    the arithmetic of the library's BF16 inference, with its FP32 sums
    replaced by exact ones."""
    W1, b1, W2, b2, W3, b3 = params
    h1 = rnd(silu(rnd(xn) @ rnd(W1) + b1))
    h2 = rnd(silu(h1 @ rnd(W2) + b2))
    return h2 @ rnd(W3) + b3
