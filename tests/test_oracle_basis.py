"""Pins of oracle.basis against closed forms (Sec. 2.2.2)."""
import math

import numpy as np
import pytest

from oracle import basis


@pytest.mark.parametrize("n,expect", [
    (1, [0.0, 1.0]),
    (2, [0.0, 0.5, 1.0]),
    (3, [0.0, 0.5 - 0.5 / math.sqrt(5.0), 0.5 + 0.5 / math.sqrt(5.0), 1.0]),
    (4, [0.0, 0.5 - 0.5 * math.sqrt(3.0 / 7.0), 0.5, 0.5 + 0.5 * math.sqrt(3.0 / 7.0), 1.0]),
])
def test_gll_closed_forms(n, expect):
    assert np.allclose(basis.gll_nodes(n), expect, atol=1e-15, rtol=0)


@pytest.mark.parametrize("p", [2, 4, 6, 8])
def test_gll_quadrature_exactness(p):
    # the GLL rule with p+1 nodes is exact for degree 2p-1; weights from the Lagrange
    # basis integrals must reproduce int_0^1 x^k = 1/(k+1)
    x = basis.gll_nodes(p)
    g, w = basis.gauss_legendre(p + 1)
    v, _ = basis.lagrange(x, g)
    wl = w @ v
    for k in range(2 * p):
        assert abs(wl @ x ** k - 1.0 / (k + 1)) < 1e-14


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("p", [1, 3, 6, 8])
def test_partition_of_unity_and_derivative(kind, p):
    x = np.linspace(0, 1, 37)
    v, d = basis.basis_1d(kind, p, x)
    assert np.allclose(v.sum(1), 1.0, atol=1e-13)
    assert np.allclose(d.sum(1), 0.0, atol=1e-11)
    # derivative against a central difference
    h = 1e-6
    vp, _ = basis.basis_1d(kind, p, x + h)
    vm, _ = basis.basis_1d(kind, p, x - h)
    assert np.allclose((vp - vm) / (2 * h), d, atol=1e-6 * max(1, p ** 2))


@pytest.mark.parametrize("p", [2, 5, 6])
def test_lagrange_is_nodal(p):
    x = basis.gll_nodes(p)
    v, _ = basis.lagrange(x, x)
    assert np.allclose(v, np.eye(p + 1), atol=1e-13)


def test_bernstein_closed_form():
    x = np.array([0.3])
    v, d = basis.bernstein(3, x)
    assert np.allclose(v[0], [0.343, 0.441, 0.189, 0.027])
    assert np.allclose(d[0], [-3 * 0.49, 3 * (0.49 - 2 * 0.21), 3 * (2 * 0.21 - 0.09), 3 * 0.09])


def test_bernstein_and_gll_span_same_space():
    # a degree-p polynomial interpolated in both bases evaluates identically
    p = 5
    x = np.linspace(0, 1, 50)
    f = lambda t: 1 - 2 * t + 3 * t ** 4 - t ** 5
    nodes = basis.gll_nodes(p)
    vl, _ = basis.lagrange(nodes, x)
    vb_n, _ = basis.bernstein(p, nodes)
    coef_b = np.linalg.solve(vb_n, f(nodes))
    vb, _ = basis.bernstein(p, x)
    assert np.allclose(vl @ f(nodes), f(x), atol=1e-13)
    assert np.allclose(vb @ coef_b, f(x), atol=1e-12)


def test_tensor_ordering():
    # k = a + (p+1) b with a along xi1
    p = 2
    B, dB = basis.basis_2d(0, p, np.array([1.0]), np.array([0.0]))
    assert np.argmax(B[0]) == p            # (a=p, b=0)
    B, _ = basis.basis_2d(0, p, np.array([0.0]), np.array([1.0]))
    assert np.argmax(B[0]) == (p + 1) * p  # (a=0, b=p)
