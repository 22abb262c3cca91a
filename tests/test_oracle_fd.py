"""Pins for the oracle's finite differences (Sec. II.B): published weights, polynomial
exactness, the Fourier symbol of the periodic / Bloch-periodic stencil, Lap 1 = 0."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import hubbard as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fd12_weights.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows[parts[0]] = [float(Fraction(v)) for v in parts[1:]]
    return rows


def test_weights_match_published_table():
    g = _golden()
    c0, c = o.fd_laplacian_weights(6)
    np.testing.assert_allclose([c0, *c], g["second"], rtol=1e-14, atol=0)
    w = o.fd_gradient_weights(6, 1.0)
    np.testing.assert_allclose(w, g["first"][1:], rtol=1e-14, atol=0)


@pytest.mark.parametrize("n0", [1, 2, 3, 4, 6])
def test_second_derivative_exact_on_polynomials(n0):
    # exact for x^d, d <= 2 n0 + 1, at an arbitrary (non-node) centre
    c0, c = o.fd_laplacian_weights(n0)
    h, x0 = 0.37, 0.81
    for d in range(0, 2 * n0 + 2):
        f = lambda x: x ** d
        approx = c0 * f(x0) + sum(c[p - 1] * (f(x0 + p * h) + f(x0 - p * h)) for p in range(1, n0 + 1))
        approx /= h * h
        exact = d * (d - 1) * x0 ** (d - 2) if d >= 2 else 0.0
        assert abs(approx - exact) <= 1e-9 * max(1.0, abs(exact)) * 10 ** (d // 4), (n0, d)
    # and not exact at degree 2 n0 + 2 (the order is what it claims, no higher)
    d = 2 * n0 + 2
    approx = (c0 * x0 ** d + sum(c[p - 1] * ((x0 + p * h) ** d + (x0 - p * h) ** d)
                                 for p in range(1, n0 + 1))) / h ** 2
    assert abs(approx - d * (d - 1) * x0 ** (d - 2)) > 1e-8


@pytest.mark.parametrize("n0", [1, 2, 6])
def test_first_derivative_exact_on_polynomials(n0):
    w = o.fd_gradient_weights(n0, 0.29)
    x0 = -0.4
    for d in range(0, 2 * n0 + 1):
        approx = sum(w[p - 1] * ((x0 + p * 0.29) ** d - (x0 - p * 0.29) ** d) for p in range(1, n0 + 1))
        exact = d * x0 ** (d - 1) if d >= 1 else 0.0
        assert abs(approx - exact) < 1e-10 * 10 ** (d // 4), (n0, d)


def _symbol(q, h, n0):
    """Eigenvalue of the discrete Laplacian on exp(i q.x): sum_a h_a^-2 [c0 + 2 sum c_p cos(p q_a h_a)]."""
    c0, c = o.fd_laplacian_weights(n0)
    return sum((c0 + 2.0 * sum(c[p - 1] * np.cos(p * q[a] * h[a]) for p in range(1, n0 + 1))) / h[a] ** 2
               for a in range(3))


@pytest.mark.parametrize("kfrac", [(0.0, 0.0, 0.0), (0.13, -0.27, 0.41)])
def test_fourier_symbol_plane_and_bloch_waves(kfrac):
    n, L = (10, 12, 14), (3.1, 3.7, 4.3)
    Lv = np.asarray(L)
    k = 2 * np.pi * np.asarray(kfrac) / Lv
    g = o.Grid(n, L, k, 6)
    x = g.coords()
    for m in [(0, 0, 0), (1, 0, 0), (0, -2, 1), (3, 4, -5), (5, 6, 7)]:
        q = k + 2 * np.pi * np.asarray(m) / Lv         # Bloch wave with wavevector k + G
        psi = np.exp(1j * x @ q)
        if not g.is_complex:
            # real periodic case: cos(q.x) is an eigenfunction too
            f = np.cos(x @ q)[:, None]
            lap = o.laplacian(f, g)[:, 0]
            np.testing.assert_allclose(lap, _symbol(q, g.h, 6) * f[:, 0], atol=1e-10 * (1 + np.abs(_symbol(q, g.h, 6))))
        else:
            lap = o.laplacian(psi[:, None], g)[:, 0]
            sym = _symbol(q, g.h, 6)
            np.testing.assert_allclose(lap, sym * psi, atol=1e-10 * (1 + abs(sym)))
            # the symbol approaches -|q|^2 as h -> 0 (sanity: low mode)
    q_low = k + 2 * np.pi * np.array([1, 0, 0]) / Lv
    assert abs(_symbol(q_low, g.h, 6) + q_low @ q_low) < 1e-6 * (q_low @ q_low)


def test_laplacian_of_constant_is_zero_and_wraps_small_grids():
    # n < 2 n0 + 1: stencil points wrap onto each other several times
    g = o.Grid((5, 7, 4), (1.5, 2.1, 1.2))
    one = np.ones((g.Nd, 1))
    assert np.max(np.abs(o.laplacian(one, g))) < 1e-10
    x = g.coords()
    q = 2 * np.pi * np.array([1, 2, 1]) / g.L
    f = np.sin(x @ q)[:, None]
    np.testing.assert_allclose(o.laplacian(f, g)[:, 0], _symbol(q, g.h, 6) * f[:, 0], atol=1e-9)


def test_gradient_symbol():
    g = o.Grid((12, 10, 9), (3.0, 2.5, 2.7), (0.3, 0.0, -0.2))
    x = g.coords()
    q = g.kpt + 2 * np.pi * np.array([2, -1, 1]) / g.L
    psi = np.exp(1j * x @ q)[:, None]
    for a in range(3):
        w = o.fd_gradient_weights(6, g.h[a])
        sym = 2j * sum(w[p - 1] * np.sin(p * q[a] * g.h[a]) for p in range(1, 7))
        np.testing.assert_allclose(o.gradient(psi, g, a)[:, 0], sym * psi[:, 0], atol=1e-10)


def test_quadrature_integrates_periodic_functions():
    g = o.Grid((16, 18, 20), (4.0, 4.5, 5.0))
    x = g.coords()
    f = 1.0 + np.cos(2 * np.pi * x[:, 0] / 4.0) * np.sin(2 * np.pi * 2 * x[:, 2] / 5.0)
    assert abs(g.integrate(f) - 4.0 * 4.5 * 5.0) < 1e-10
