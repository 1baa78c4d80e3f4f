"""Pins of the oracle's 1-D FR operators against closed forms and textbook values."""
import os

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from oracle import fr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_gauss():
    rows = {}
    for line in open(os.path.join(GOLDEN, "gauss_legendre.txt")):
        if line.startswith("#") or not line.strip():
            continue
        n, x, w = line.split()
        rows.setdefault(int(n), []).append((float(x), float(w)))
    return rows


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_gauss_nodes_match_abramowitz_stegun(n):
    x, w = fr.gauss_legendre(n)
    ref = _golden_gauss()[n]
    xs = sorted({v for a, _ in ref for v in (a, -a)})
    ws = {abs(round(a, 12)): b for a, b in ref}
    assert np.allclose(x, xs, rtol=0, atol=1e-14)
    assert np.allclose(w, [ws[abs(round(v, 12))] for v in xs], rtol=0, atol=1e-14)


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_rule_matches_library_and_integrates_degree_2n_minus_1(n):
    x, w = fr.gauss_legendre(n)
    lx, lw = leggauss(n)
    assert np.allclose(x, lx, atol=1e-14) and np.allclose(w, lw, atol=1e-14)
    for deg in range(2 * n):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.sum(w * x ** deg) - exact) < 1e-14


def test_closed_form_nodes_p_le_3():
    r = 1 / np.sqrt(3)
    assert np.allclose(fr.gauss_legendre(2)[0], [-r, r], atol=1e-16)
    s = np.sqrt(3 / 5)
    assert np.allclose(fr.gauss_legendre(3)[0], [-s, 0, s], atol=1e-16)
    a = np.sqrt(3 / 7 - 2 / 7 * np.sqrt(6 / 5))
    b = np.sqrt(3 / 7 + 2 / 7 * np.sqrt(6 / 5))
    assert np.allclose(fr.gauss_legendre(4)[0], [-b, -a, a, b], atol=1e-15)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_derivative_and_traces_exact_on_degree_p(p):
    op = fr.FR1D(p)
    for m in range(p + 1):
        fx = op.xi ** m
        dfx = m * op.xi ** (m - 1) if m > 0 else np.zeros_like(op.xi)
        assert np.allclose(op.D @ fx, dfx, atol=1e-13)
        assert abs(op.l_minus @ fx - (-1.0) ** m) < 1e-13
        assert abs(op.l_plus @ fx - 1.0) < 1e-13


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_radau_correction_functions(p):
    """g_L(-1)=1, g_L(1)=0, g_R(-1)=0, g_R(1)=1, g_R(x) = g_L(-x); GL quadrature of
    g' (degree p) integrates it exactly: sum W g_R' = 1, sum W g_L' = -1."""
    x = np.array([-1.0, 1.0])
    gl = fr.correction_left(p, x)[0]
    gr = fr.correction_right(p, x)[0]
    assert np.allclose(gl, [1, 0], atol=1e-15) and np.allclose(gr, [0, 1], atol=1e-15)
    t = np.linspace(-1, 1, 11)
    assert np.allclose(fr.correction_right(p, t)[0], fr.correction_left(p, -t)[0], atol=1e-15)
    op = fr.FR1D(p)
    assert abs(op.wq @ op.dgR - 1.0) < 1e-14
    assert abs(op.wq @ op.dgL + 1.0) < 1e-14
    # g_L is the right Radau polynomial: it vanishes at the p+1 right-Radau points,
    # which include x = 1, and is orthogonal to degree p-1 polynomials.
    xq, wq = leggauss(p + 3)
    g = fr.correction_left(p, xq)[0]
    for m in range(p):
        assert abs(np.sum(wq * g * xq ** m)) < 1e-14


def test_legendre_values_against_library():
    from numpy.polynomial import legendre as L
    t = np.linspace(-1, 1, 17)
    for n in range(7):
        c = np.zeros(n + 1)
        c[n] = 1
        p, dp = fr.legendre(n, t)
        assert np.allclose(p, L.legval(t, c), atol=1e-14)
        assert np.allclose(dp, L.legval(t, L.legder(c)), atol=1e-12)
