"""Pins of the oracle's explicit Runge-Kutta map for a given tableau (stage s
uses only the slope of stage s-1: the family of the paper's RK4 and Euler
methods) and of its discrete adjoint, against closed forms and the methods'
textbook properties."""
import math

import numpy as np
import pytest
from scipy import linalg

import oracle
from paper_1906_03958_gb300 import netgen as ng

# (name, (a, b), order of accuracy)
TABLEAUS = [
    ("midpoint", ([0.5], [0.0, 1.0]), 2),
    ("heun2", ([1.0], [0.5, 0.5]), 2),
    ("ralston2", ([2.0 / 3.0], [0.25, 0.75]), 2),
    ("heun3", ([1.0 / 3.0, 2.0 / 3.0], [0.25, 0.0, 0.75]), 3),
    ("ralston3", ([0.5, 0.75], [2.0 / 9.0, 1.0 / 3.0, 4.0 / 9.0]), 3),
    ("rk4", ([0.5, 0.5, 1.0], [1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0]), 4),
]
RK4 = TABLEAUS[-1][1]
EULER = ([], [1.0])


def _A():
    return np.array([[-1.0, 4.0, 0.0], [0.0, -1.0, 4.0], [0.5, 0.0, -2.0]])


def _taylor(hA, p):
    P, term = np.eye(len(hA)), np.eye(len(hA))
    for k in range(1, p + 1):
        term = term @ hA / k
        P = P + term
    return P


@pytest.mark.parametrize("name,tab,p", TABLEAUS, ids=[t[0] for t in TABLEAUS])
def test_one_step_is_the_truncated_exponential(name, tab, p):
    # an explicit method with s = p stages and order p (p <= 4) maps y' = A y
    # by the degree-p Taylor polynomial of exp(hA), whatever its coefficients
    A, h = _A(), 0.1
    y0 = np.array([1.0, 2.0, -1.0])
    got = oracle.linear_integrate(A, y0, h, 1, tableau=tab)
    np.testing.assert_allclose(got, _taylor(h * A, p) @ y0, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("name,tab,p", TABLEAUS, ids=[t[0] for t in TABLEAUS])
def test_global_convergence_order(name, tab, p):
    A = np.array([[-0.5, 2.0], [-2.0, -0.5]])
    y0 = np.array([1.0, -0.5])
    T = 2.0
    exact = linalg.expm(A * T) @ y0
    h0 = {2: 0.02, 3: 0.05, 4: 0.1}[p]
    errs = []
    for h in (h0, h0 / 2, h0 / 4, h0 / 8):
        errs.append(np.max(np.abs(oracle.linear_integrate(A, y0, h, int(round(T / h)), tableau=tab) - exact)))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(s - p) < 0.1 for s in slopes), slopes


def test_rk4_and_euler_tableaus_are_the_named_methods():
    # the classic tableau gives the RK4 map up to rounding order, the
    # one-stage tableau b = (1) forward Euler, Eq. (euler), bit for bit
    spec = ng.antennal_lobe(seed=95, n_pn=12, n_ln=4)
    y0 = oracle.rest_state(spec)
    a, ra = oracle.integrate(spec, y0, 400, rec_stride=10)
    b, rb = oracle.integrate(spec, y0, 400, rec_stride=10, tableau=RK4)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))
    assert np.max(np.abs(ra - rb)) <= 1e-11
    c, _ = oracle.integrate(spec, y0, 400, order=1)
    d, _ = oracle.integrate(spec, y0, 400, tableau=EULER)
    np.testing.assert_array_equal(c, d)


@pytest.mark.parametrize("name,tab,p", TABLEAUS[:5], ids=[t[0] for t in TABLEAUS[:5]])
def test_linear_adjoint_closed_form(name, tab, p):
    # n steps of y -> R y with R the truncated exponential: the adjoint
    # carries lam back by (R^T)^n
    A, h, n = _A(), 0.05, 40
    y0 = np.array([1.0, 2.0, -1.0])
    lam_T = np.array([0.3, -1.2, 0.7])
    want = np.linalg.matrix_power(_taylor(h * A, p).T, n) @ lam_T
    np.testing.assert_allclose(oracle.linear_adjoint(A, y0, h, n, lam_T, tableau=tab), want, rtol=1e-13,
                               atol=1e-13)


def test_tableau_validation():
    with pytest.raises(ValueError):
        oracle.linear_integrate(_A(), np.ones(3), 0.1, 1, tableau=([0.5, 0.5], [0.5, 0.5]))
    with pytest.raises(ValueError):
        oracle.linear_integrate(_A(), np.ones(3), 0.1, 1, tableau=([0.5] * 4, [0.2] * 5))
    with pytest.raises(ValueError):
        oracle.linear_integrate(_A(), np.ones(3), 0.1, 1, order=2)
