"""Independent 1-D linear stability solver of the parallel tanh mixing layer
(test infrastructure: it pins the oracle; neither the oracle nor the library
uses it).

The compressible Navier-Stokes equations in primitive (p, u, v, s) form with
the closure of the Sec. "Governing equations" readings (ideal gas, entropy
s = c_v ln(p/p_ref) - c_p ln rho, Sutherland viscosity, lambda = mu c_p / Pr,
Stokes hypothesis plus an optional bulk viscosity) are written here a second
time, symbolically, and linearised by sympy about the frozen base state
q0 = (1/(gamma Ma^2), tanh y, 0, 0).  A perturbation q(y) exp(i k x + lambda t)
then obeys lambda q = L(k) q, with y discretised by Chebyshev collocation on a
sinh-mapped interval [-Y, Y] and q = 0 imposed at both ends (the modes of
interest have decayed there).

x derivatives enter through their symbols: d/dx -> i k1, d2/dx2 -> -k2^2.
With k1 = k2 = k this is the continuous problem; with the modified
wavenumbers of a compact scheme (``lele_k1``, ``lele_k2``, Lele 1992 Eqs.
2.1.7 / 2.2.7) it is the problem the 2-D discretisation solves for that
x-Fourier mode, up to the y discretisation.

Nothing here is shared with the oracle or the CUDA library: other variables
of differentiation (symbolic instead of hand-expanded), another y scheme
(Chebyshev instead of compact differences) and other boundary rows.
"""
from __future__ import annotations

import functools
import math

import numpy as np
import scipy.linalg as sla

GAMMA = 1.4
SUTHERLAND_S = 110.4 / 273.15


# ---------------------------------------------------------------------------
# Symbolic linearisation (cached per bulk-viscosity switch)
# ---------------------------------------------------------------------------
@functools.lru_cache(maxsize=None)
def _linear_terms(viscous: bool):
    """Coefficients of the linearised equations.

    Returns {(eq, var, ax, ay): f(y, Ma, Re, Pr, gamma, S, bulk)} where the
    term is f(y) * d^ax/dx^ax d^ay/dy^ay of perturbation variable var in
    equation eq (0 p, 1 u, 2 v, 3 s)."""
    import sympy as sp

    x, y, eps = sp.symbols("x y epsilon", real=True)
    Ma, Re, Pr, gam, S, bulk = sp.symbols("Ma Re Pr gamma S bulk", positive=True)
    Pp, Up, Vp, Sp_ = [sp.Function(n)(x, y) for n in ("Pp", "Up", "Vp", "Sp")]
    U0 = sp.Function("U0")(y)

    pref = 1 / (gam * Ma ** 2)
    R = pref
    cp = gam * R / (gam - 1)
    p = pref + eps * Pp
    u = U0 + eps * Up
    v = eps * Vp
    s = eps * Sp_
    rho = (p / pref) ** (1 / gam) * sp.exp(-s / cp)
    T = p / (rho * R)
    vel = [u, v]
    X = [x, y]
    div = sp.diff(u, x) + sp.diff(v, y)
    dpdt = -(u * sp.diff(p, x) + v * sp.diff(p, y)) - gam * p * div
    dudt = [-(u * sp.diff(vel[i], x) + v * sp.diff(vel[i], y)) - sp.diff(p, X[i]) / rho for i in range(2)]
    dsdt = -(u * sp.diff(s, x) + v * sp.diff(s, y))
    if viscous:
        mu = (1 / Re) * T ** sp.Rational(3, 2) * (1 + S) / (T + S)
        lam = mu * cp / Pr
        muv = bulk * mu
        sij = [[(sp.diff(vel[i], X[j]) + sp.diff(vel[j], X[i])) / 2 for j in range(2)] for i in range(2)]
        tau = [[2 * mu * (sij[i][j] - (div / 3 if i == j else 0)) + (muv * div if i == j else 0) for j in range(2)]
               for i in range(2)]
        Phi = sum(tau[i][j] * sij[i][j] for i in range(2) for j in range(2))
        heat = sum(sp.diff(lam * sp.diff(T, X[j]), X[j]) for j in range(2))
        dpdt += (gam - 1) * (heat + Phi)
        for i in range(2):
            dudt[i] += sum(sp.diff(tau[i][j], X[j]) for j in range(2)) / rho
        dsdt += (heat + Phi) / (rho * T)
    eqs = [dpdt, dudt[0], dudt[1], dsdt]
    pert = [Pp, Up, Vp, Sp_]
    out = {}
    params = (y, Ma, Re, Pr, gam, S, bulk)
    for e_i, expr in enumerate(eqs):
        lin = sp.diff(expr, eps).subs(eps, 0)
        lin = sp.expand(lin.doit())
        # replace every derivative of a perturbation by a plain symbol, then
        # read the coefficient of each symbol (the equation is linear in them)
        reps = {}
        for var_i, F in enumerate(pert):
            for ax in range(3):
                for ay in range(3):
                    if ax + ay > 2:
                        continue
                    if ax == 0 and ay == 0:
                        d = F
                    else:
                        args = []
                        if ax:
                            args.append((x, ax))
                        if ay:
                            args.append((y, ay))
                        d = sp.Derivative(F, *args)
                    reps[d] = sp.Symbol(f"w_{var_i}_{ax}_{ay}")
        # substitute the highest derivatives first so that sub-expressions stay intact
        keys = sorted(reps, key=lambda d: -sum(c for _, c in getattr(d, "variable_count", [])))
        lin_s = lin
        for d in keys:
            lin_s = lin_s.subs(d, reps[d])
        lin_s = sp.expand(lin_s)
        for d, w in reps.items():
            c = lin_s.coeff(w)
            if c == 0:
                continue
            var_i, ax, ay = (int(t) for t in w.name.split("_")[1:])
            c = sp.simplify(c)
            # base flow: U0 = tanh(y) and its derivatives
            c = c.subs({sp.Derivative(U0, (y, 2)): -2 * sp.tanh(y) * (1 - sp.tanh(y) ** 2)}) \
                 .subs({sp.Derivative(U0, y): 1 - sp.tanh(y) ** 2}).subs({U0: sp.tanh(y)})
            out[(e_i, var_i, ax, ay)] = sp.lambdify(params, c, "numpy")
        # nothing of the perturbation may be left over
        rest = lin_s.subs({w: 0 for w in reps.values()})
        assert sp.simplify(rest) == 0, f"equation {e_i}: non-linear or unmatched terms {rest}"
    return out


# ---------------------------------------------------------------------------
# Chebyshev collocation on a sinh-mapped interval
# ---------------------------------------------------------------------------
def cheb(N: int):
    """Chebyshev-Gauss-Lobatto points xi_j = cos(pi j / N) and the
    differentiation matrix (Trefethen, Spectral Methods in MATLAB, cheb.m)."""
    xi = np.cos(np.pi * np.arange(N + 1) / N)
    c = np.ones(N + 1)
    c[0] = c[-1] = 2.0
    c *= (-1.0) ** np.arange(N + 1)
    X = np.tile(xi, (N + 1, 1)).T
    dX = X - X.T
    D = np.outer(c, 1.0 / c) / (dX + np.eye(N + 1))
    D -= np.diag(D.sum(axis=1))
    return xi, D


def mapped_grid(N: int, Y: float, beta: float):
    """y = Y sinh(beta xi)/sinh(beta) with its first and second derivative matrices."""
    xi, Dxi = cheb(N)
    y = Y * np.sinh(beta * xi) / math.sinh(beta)
    yp = Y * beta * np.cosh(beta * xi) / math.sinh(beta)
    D1 = Dxi / yp[:, None]
    D2 = D1 @ D1
    return y, D1, D2


def lele_k1(k: float, h: float) -> float:
    """Modified wavenumber of the 6th-order compact first derivative
    (alpha = 1/3, a = 14/9, b = 1/9)."""
    w = k * h
    return (14.0 / 9.0 * math.sin(w) + (1.0 / 18.0) * math.sin(2 * w)) / (1.0 + 2.0 / 3.0 * math.cos(w)) / h


def lele_k2(k: float, h: float) -> float:
    """Modified wavenumber k2 (symbol -k2^2) of the 6th-order compact second
    derivative (alpha = 2/11, a = 12/11, b = 3/11)."""
    w = k * h
    num = 2 * (12.0 / 11.0) * (1 - math.cos(w)) + (3.0 / 11.0) / 2 * (1 - math.cos(2 * w))
    return math.sqrt(num / (1.0 + 4.0 / 11.0 * math.cos(w))) / h


def operator(k1: float, k2: float, Ma: float, Re: float | None, N: int = 160, Y: float = 60.0, beta: float = 4.0,
             Pr: float = 0.71, gamma: float = GAMMA, S: float = SUTHERLAND_S, bulk: float = 0.0):
    """Dense L(k) on the interior collocation points (q = 0 at y = +-Y), unknowns
    ordered [var][y]; returns (L, y_interior)."""
    viscous = bool(Re) and Re > 0
    terms = _linear_terms(viscous)
    y, D1, D2 = mapped_grid(N, Y, beta)
    I = np.eye(N + 1)
    Dy = [I, D1, D2]
    sym_x = [1.0, 1j * k1, -k2 * k2]
    Rev = Re if viscous else 1.0
    L = np.zeros((4 * (N + 1), 4 * (N + 1)), dtype=complex)
    for (e, var, ax, ay), f in terms.items():
        c = np.broadcast_to(np.asarray(f(y, Ma, Rev, Pr, gamma, S, bulk), dtype=float), y.shape)
        if ax == 1 and ay == 1:
            blk = sym_x[1] * Dy[1]
        else:
            blk = sym_x[ax] * Dy[ay]
        L[e * (N + 1):(e + 1) * (N + 1), var * (N + 1):(var + 1) * (N + 1)] += c[:, None] * blk
    keep = np.concatenate([v * (N + 1) + np.arange(1, N) for v in range(4)])
    return L[np.ix_(keep, keep)], y[1:N]


def kh_growth(k1: float, k2: float, Ma: float, Re: float | None, **kw) -> tuple[float, complex]:
    """Growth rate of the Kelvin-Helmholtz mode: the real part of the
    eigenvalue with the largest real part among the eigenvalues whose
    imaginary part is negligible (the tanh layer's unstable mode does not
    propagate); also returns that eigenvalue."""
    L, _ = operator(k1, k2, Ma, Re, **kw)
    lam = sla.eigvals(L)
    cand = lam[np.abs(lam.imag) < 1e-6 * max(1.0, np.abs(lam).max() * 1e-6) + 1e-7]
    if cand.size == 0:
        return float("nan"), complex("nan")
    lmax = cand[np.argmax(cand.real)]
    return float(lmax.real), complex(lmax)


def alpha_max(Ma: float, Re: float | None, lo: float = 0.1, hi: float = 0.7, xtol: float = 1e-4, **kw):
    """Wavenumber of the least stable mode and its growth rate (continuous in x)."""
    from scipy.optimize import minimize_scalar

    r = minimize_scalar(lambda a: -kh_growth(a, a, Ma, Re, **kw)[0], bounds=(lo, hi), method="bounded",
                        options={"xatol": xtol})
    return float(r.x), float(-r.fun)
