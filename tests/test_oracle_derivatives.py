"""Pins of the oracle's compact finite differences (Sec. Governing equations,
the Lele 1992 schemes): closed-form modified wavenumbers, polynomial
exactness, exact zero on constants, the tridiagonal solvers against a dense
library solve, and the convergence order on a stretched grid; the reduced
operator's second-order explicit differences likewise."""
import math

import numpy as np
import pytest

import stab_inputs as si


def _kp1(kh):  # Lele's first-derivative modified wavenumber (times h)
    a, b, al = 14 / 9, 1 / 9, 1 / 3
    return (a * np.sin(kh) + (b / 2) * np.sin(2 * kh)) / (1 + 2 * al * np.cos(kh))


def _kp2(kh):  # second-derivative modified wavenumber squared (times h^2)
    a, b, al = 12 / 11, 3 / 11, 2 / 11
    return (2 * a * (1 - np.cos(kh)) + (b / 2) * (1 - np.cos(2 * kh))) / (1 + 2 * al * np.cos(kh))


@pytest.mark.parametrize("n", [16, 33, 64])
def test_periodic_modified_wavenumber(orc, n):
    h = 2 * np.pi / n
    x = np.arange(n) * h
    for k in range(0, n // 2):
        f = np.sin(k * x + 0.3)
        d1 = orc.core.deriv_line(f, h, 1, True)
        d2 = orc.core.deriv_line(f, h, 2, True)
        kh = k * h
        assert np.abs(d1 - _kp1(kh) / h * np.cos(k * x + 0.3)).max() < 1e-12 * (1 + k)
        assert np.abs(d2 + _kp2(kh) / h ** 2 * np.sin(k * x + 0.3)).max() < 1e-11 * (1 + k * k)


def test_periodic_sixth_order_convergence(orc):
    errs = []
    for n in (16, 32, 64):
        h = 2 * np.pi / n
        x = np.arange(n) * h
        f = np.exp(np.sin(x))
        errs.append(np.abs(orc.core.deriv_line(f, h, 1, True) - np.cos(x) * f).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 5.5


@pytest.mark.parametrize("n", [6, 9, 40])
def test_bounded_polynomial_exactness(orc, n):
    h = 0.37
    x = np.arange(n) * h - 1.1
    for deg in range(0, 4):  # first derivative: exact to degree 3 (boundary rows third order)
        d = orc.core.deriv_line(x ** deg, h, 1, False)
        ex = deg * x ** (deg - 1) if deg else 0 * x
        assert np.abs(d - ex).max() < 1e-12 * max(1, np.abs(ex).max())
    for deg in range(0, 5):  # second derivative: exact to degree 4
        d = orc.core.deriv_line(x ** deg, h, 2, False)
        ex = deg * (deg - 1) * x ** (deg - 2) if deg > 1 else 0 * x
        assert np.abs(d - ex).max() < 1e-11 * max(1, np.abs(ex).max())
    # degree 4 / 5 are NOT exact: the closures are third order
    assert np.abs(orc.core.deriv_line(x ** 4, h, 1, False) - 4 * x ** 3).max() > 1e-6


def test_constant_gives_zero(orc):
    """Exactly zero on periodic lines; rounding-level on bounded lines (the
    one-sided closure weights cancel only in exact arithmetic)."""
    for order in (1, 2):
        assert np.all(orc.core.deriv_line(np.full(24, 3.7), 0.1, order, True) == 0.0)
        d = orc.core.deriv_line(np.full(24, 3.7), 0.1, order, False)
        assert np.abs(d).max() < 1e-13 * 3.7 / 0.1 ** order


def _dense_scheme(n, h, order, periodic):
    """A and B of A f' = B f built from the scheme definitions, row by row."""
    A = np.eye(n)
    B = np.zeros((n, n))
    if order == 1:
        al, a, b = 1 / 3, 14 / 9, 1 / 9
        sten = {1: a / (2 * h), -1: -a / (2 * h), 2: b / (4 * h), -2: -b / (4 * h)}
    else:
        al, a, b = 2 / 11, 12 / 11, 3 / 11
        sten = {1: a / h ** 2, -1: a / h ** 2, 0: -2 * a / h ** 2 - 2 * b / (4 * h ** 2),
                2: b / (4 * h ** 2), -2: b / (4 * h ** 2)}
    for i in range(n):
        for off, c in ((-1, al), (1, al)):
            j = i + off
            if periodic or 0 <= j < n:
                A[i, j % n] = c
        for off, c in sten.items():
            j = i + off
            if periodic or 0 <= j < n:
                B[i, j % n] += c
    if not periodic:
        for i, sgn in ((0, 1), (n - 1, -1)):
            A[i, :] = 0
            B[i, :] = 0
            A[i, i] = 1
            nb = [i + sgn * k for k in range(4)]
            if order == 1:
                A[i, nb[1]] = 2
                for k, c in enumerate((-2.5, 2.0, 0.5)):
                    B[i, nb[k]] = sgn * c / h
            else:
                A[i, nb[1]] = 11
                for k, c in enumerate((13, -27, 15, -1)):
                    B[i, nb[k]] = c / h ** 2
        for i in (1, n - 2):
            A[i, :] = 0
            B[i, :] = 0
            A[i, i] = 1
            if order == 1:
                A[i, i - 1] = A[i, i + 1] = 0.25
                B[i, i + 1], B[i, i - 1] = 0.75 / h, -0.75 / h
            else:
                A[i, i - 1] = A[i, i + 1] = 0.1
                B[i, i + 1] = B[i, i - 1] = 1.2 / h ** 2
                B[i, i] = -2.4 / h ** 2
    return A, B


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("order", [1, 2])
def test_tridiagonal_solvers_match_dense_solve(orc, periodic, order):
    rng = np.random.default_rng(7)
    n, h = 29, 0.21
    A, B = _dense_scheme(n, h, order, periodic)
    f = rng.standard_normal(n)
    ref = np.linalg.solve(A, B @ f)
    got = orc.core.deriv_line(f, h, order, periodic)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_stretched_y_metric_convergence(orc):
    """d/dy and d2/dy2 on a sinh-stretched grid converge at (asymptotically) third order."""
    e1, e2 = [], []
    for ny in (96, 192, 384):
        g = si.Grid(2, 4, ny, 1, 1.0, -15.0, 15.0, 1.0, 2.5)
        P = orc.Problem.from_inputs(g, si.Flow(0.3, 1000.0))
        y = g.y()
        f = np.broadcast_to(np.sin(y / 3.0)[:, None], (ny, 4)).copy()
        d1 = orc.core.deriv_field(P, f, axis=1, order=1).reshape(ny, 4)[:, 0]
        d2 = orc.core.deriv_field(P, f, axis=1, order=2).reshape(ny, 4)[:, 0]
        e1.append(np.abs(d1 - np.cos(y / 3) / 3).max())
        e2.append(np.abs(d2 + np.sin(y / 3) / 9).max())
    assert np.log2(e1[0] / e1[1]) > 2.5 and np.log2(e1[1] / e1[2]) > 2.7
    assert np.log2(e2[0] / e2[1]) > 2.5 and np.log2(e2[1] / e2[2]) > 2.7


@pytest.mark.parametrize("n", [16, 33])
def test_reduced_operator_differences(orc, n):
    """The reduced operator's second-order explicit differences: periodic
    modified wavenumbers sin(kh)/h and 2 (1 - cos(kh))/h^2 on every Fourier
    mode; on a bounded line the first derivative exact for quadratics and the
    second for cubics, end rows included (second-order one-sided forms)."""
    h = 2 * math.pi / n
    x = np.arange(n) * h
    for k in range(1, n // 2):
        f = np.cos(k * x)
        d1 = orc.core.deriv_line(f, h, 1, True, low=True)
        d2 = orc.core.deriv_line(f, h, 2, True, low=True)
        assert np.abs(d1 + math.sin(k * h) / h * np.sin(k * x)).max() < 1e-12
        assert np.abs(d2 + 2 * (1 - math.cos(k * h)) / h ** 2 * f).max() < 1e-11
    hb = 0.37
    y = np.arange(n) * hb - 1.3
    f = 0.4 - 1.1 * y + 0.7 * y ** 2
    assert np.abs(orc.core.deriv_line(f, hb, 1, False, low=True) - (-1.1 + 1.4 * y)).max() < 1e-11
    f3 = f + 0.3 * y ** 3
    assert np.abs(orc.core.deriv_line(f3, hb, 2, False, low=True) - (1.4 + 1.8 * y)).max() < 1e-10
    assert np.abs(orc.core.deriv_line(np.full(n, 2.5), hb, 1, False, low=True)).max() < 1e-12
