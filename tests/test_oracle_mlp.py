"""Pins of the FP64 reference MLP: analytic backprop vs central differences,
SiLU closed forms, feature/target definitions against their special cases."""
import numpy as np
import pytest

from oracle import bgk, mlp
from oracle.velocity import VelocityGrid


def test_silu_closed_forms():
    z = np.array([-3.0, -0.5, 0.0, 0.7, 4.0])
    assert np.allclose(mlp.silu(z), z / (1 + np.exp(-z)), rtol=0, atol=0)
    assert mlp.silu(np.array([0.0]))[0] == 0.0
    assert mlp.silu_grad(np.array([0.0]))[0] == pytest.approx(0.5, abs=1e-16)
    h = 1e-6
    assert np.allclose(mlp.silu_grad(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), atol=1e-9)


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(0)
    params = mlp.init_params(3)
    xn = rng.standard_normal((7, 9))
    tn = rng.standard_normal((7, 5))
    loss, grads = mlp.loss_and_grads(params, xn, tn)
    for pi, (p, g) in enumerate(zip(params, grads)):
        flat = p.reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            h = 1e-6 * max(1.0, abs(old))
            flat[i] = old + h
            lp, _ = mlp.loss_and_grads(params, xn, tn)
            flat[i] = old - h
            lm, _ = mlp.loss_and_grads(params, xn, tn)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g.reshape(-1)[i]) <= 1e-7 * max(1.0, abs(fd)), (pi, i)


def test_linear_special_case():
    """With W1 = W2 = 0 the network is the constant b3 + silu(b2) W3."""
    params = mlp.init_params(1)
    params[0][:] = 0
    params[2][:] = 0
    params[3][:] = 0.3
    y, _ = mlp.forward(params, np.random.default_rng(2).standard_normal((4, 9)))
    expect = mlp.silu(np.full(64, 0.3)) @ params[4] + params[5]
    assert np.allclose(y, expect[None, :], atol=1e-14)


def test_features_and_target_special_cases():
    """Isotropic sampled Maxwellian: A = I (I1 = 3, I2 = 3, I3 = 1) on a fine grid,
    and the target of q' = q is zero; guess() inverts target()."""
    vg = VelocityGrid((26, 26, 26), (-8, -8, -8), (8, 8, 8))
    gas = bgk.Gas(delta=0.0, Pr=1.0, mu_ref=0.1, theta_ref=1.0, theta_S=0.5)
    rho = np.array([1.2, 0.8])
    U = np.array([[0.1, -0.2, 0.3], [0.0, 0.4, 0.0]])
    th = np.array([1.1, 0.9])
    m = bgk.raw_moments(bgk.maxwellian(vg, rho, U, th), None, vg)
    x = mlp.features(m, gas)
    assert np.allclose(x[:, 0], rho, rtol=1e-12) and np.allclose(x[:, 1:4], U, atol=1e-12)
    assert np.allclose(x[:, 4], th, rtol=1e-11)
    assert np.allclose(x[:, 5], 3.0, atol=1e-10) and np.allclose(x[:, 6], 3.0, atol=1e-10)
    assert np.allclose(x[:, 7], 1.0, atol=1e-10)
    lam = gas.viscosity(th) / rho * np.sqrt(np.pi / (2 * th))
    assert np.allclose(x[:, 8], lam, rtol=1e-11)
    r, Um, E, theta, P, Pi = bgk.macroscopic(m, gas)
    qp = np.concatenate([r[:, None], Um, theta[:, None]], axis=1)
    assert np.allclose(mlp.target(m, qp, gas), 0.0, atol=1e-15)
    d = np.random.default_rng(5).standard_normal((2, 5)) * 1e-3
    assert np.allclose(mlp.target(m, mlp.guess(m, d, gas), gas), d, atol=1e-14)


def test_invariants_of_a_rotated_anisotropic_state():
    """A sampled anisotropic Gaussian with covariance R diag(s) R^T (R a random
    rotation): A = Pi/(rho theta) has the eigenvalues s/theta, so I1, I2, I3 are
    the elementary symmetric functions of s/theta whatever R is."""
    vg = VelocityGrid((40, 40, 40), (-9, -9, -9), (9, 9, 9))
    gas = bgk.Gas(delta=0.0, Pr=2.0 / 3.0, mu_ref=0.05, theta_ref=1.0, theta_S=0.5)
    q, _ = np.linalg.qr(np.random.default_rng(7).standard_normal((3, 3)))
    s = np.array([0.7, 1.0, 1.45])
    T = q @ np.diag(s) @ q.T
    F = bgk.gaussian(vg.u, np.array([1.3]), np.array([[0.2, -0.1, 0.05]]), T[None])
    m = bgk.raw_moments(F, None, vg)
    x = mlp.features(m, gas)
    theta = s.mean()
    ev = s / theta
    assert np.isclose(x[0, 4], theta, rtol=1e-9)
    assert np.isclose(x[0, 5], ev.sum(), rtol=1e-9)
    assert np.isclose(x[0, 6], ev[0] * ev[1] + ev[0] * ev[2] + ev[1] * ev[2], rtol=1e-9)
    assert np.isclose(x[0, 7], ev.prod(), rtol=1e-9)


def test_bf16_rounding_closed_forms():
    """BF16 keeps 8 significant bits with ties to even: 1 + 2^-8 is a tie and
    rounds to 1, 1 + 3 2^-9 rounds up to 1 + 2^-7, -(1 + 3 2^-8) is a tie
    between 1 + 2^-7 (odd) and 1 + 2^-6 (even); BF16 values are fixed points;
    the relative error of any rounding is at most 2^-8."""
    r = mlp.bf16_round
    assert r(1 + 2.0 ** -8) == 1.0
    assert r(1 + 3 * 2.0 ** -9) == 1 + 2.0 ** -7
    assert r(-(1 + 3 * 2.0 ** -8)) == -(1 + 2.0 ** -6)
    assert r(0.0) == 0.0 and r(2.0 ** -100) == 2.0 ** -100
    rng = np.random.default_rng(4)
    v = rng.standard_normal(10000) * np.exp(rng.uniform(-20, 20, 10000))
    b = r(v)
    assert np.all(r(b) == b)
    assert np.max(np.abs(b - v) / np.abs(v)) <= 2.0 ** -8 * (1 + 1e-6)


def test_bf16_forward_structure():
    """With the identity for the rounding the BF16 forward pass is the FP64
    network; with BF16 rounding its outputs stay within the first-order bound
    of the roundings (2^-8 of the magnitudes that enter each layer)."""
    rng = np.random.default_rng(5)
    params = mlp.init_params(6)
    xn = rng.standard_normal((50, 9))
    y, _ = mlp.forward(params, xn)
    assert np.allclose(mlp.forward_bf16(params, xn, rnd=lambda a: a), y, rtol=0, atol=1e-14)
    yb = mlp.forward_bf16(params, xn)
    W1, b1, W2, b2, W3, b3 = params
    h1 = np.abs(mlp.silu(xn @ W1 + b1))
    bound = 8 * 2.0 ** -8 * (np.abs(mlp.silu(h1 @ W2 + b2)) @ np.abs(W3)
                             + (h1 @ np.abs(W2)) @ np.abs(W3) + ((np.abs(xn) @ np.abs(W1)) @ np.abs(W2)) @ np.abs(W3))
    assert np.all(np.abs(yb - y) <= bound)
