"""Pins of the oracle's right-hand side N(q) (Eq. navier_stokes with the
closure of Sec. Governing equations) and of its J(q0) v (Eq. frechet), each
against a closed form, an exact invariant or the mathematics of the
epsilon-quotient."""
import math

import numpy as np
import pytest

import stab_inputs as si

GAM = 1.4


def _problem(orc, nx=16, ny=24, Ma=0.3, Re=1000.0, stretch=0.0, dim=2, nz=1, bulk=0.0, low=0):
    g = si.Grid(dim, nx, ny, nz, 2 * math.pi / 0.4, -15.0, 15.0, 2 * math.pi / 0.4, stretch)
    f = si.Flow(Ma, Re)
    return g, f, orc.Problem.from_inputs(g, f, bulk, low)


def _uniform(g, f, U0=0.0, s0=0.0):
    q = np.zeros((g.nvars, g.nz, g.ny, g.nx))
    q[0] = 1.0 / (f.gamma * f.Ma ** 2)
    q[1] = U0
    q[-1] = s0
    return q


@pytest.mark.parametrize("Re", [1000.0, 0.0])
@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_state_at_rest_is_steady(orc, Re, dim):
    g, f, P = _problem(orc, Re=Re, dim=dim, nz=8 if dim == 3 else 1)
    r = orc.core.rhs(P, _uniform(g, f))
    assert np.abs(r).max() < 1e-11


def test_inviscid_tanh_layer_is_steady(orc):
    g, f, P = _problem(orc, Re=0.0)
    q0 = si.tanh_base_flow(g, f)
    assert np.all(orc.core.rhs(P, q0) == 0.0)


def test_galilean_shift_adds_convection(orc):
    """J at base + U0 e_x equals J at base minus U0 d/dx on every variable."""
    g, f, P = _problem(orc, nx=16, ny=20)
    q0 = si.tanh_base_flow(g, f)
    q1 = q0.copy()
    q1[1] += 0.7
    v = si.random_complex(11, g.n)
    j0 = orc.core.jv(P, q0, v)
    j1 = orc.core.jv(P, q1, v)
    dx = np.concatenate([orc.core.deriv_field(P, v.reshape(g.nvars, -1)[i].real, 0, 1)
                         + 1j * orc.core.deriv_field(P, v.reshape(g.nvars, -1)[i].imag, 0, 1)
                         for i in range(g.nvars)])
    assert np.linalg.norm(j1 - j0 + 0.7 * dx) < 1e-12 * np.linalg.norm(j0)


def _symbols(h, k, n, low=0):
    """Modified wavenumbers k' (first derivative) and k''^2 (second) of the
    compact schemes, or (low) of the reduced operator's second-order explicit
    differences: sin(kh)/h and 2 (1 - cos(kh))/h^2."""
    kh = 2 * math.pi * k / n
    if low:
        return math.sin(kh) / h, 2 * (1 - math.cos(kh)) / h ** 2
    k1 = (14 / 9 * math.sin(kh) + (1 / 18) * math.sin(2 * kh)) / (1 + 2 / 3 * math.cos(kh)) / h
    k2 = (24 / 11 * (1 - math.cos(kh)) + 3 / 22 * (1 - math.cos(2 * kh))) / (1 + 4 / 11 * math.cos(kh)) / h ** 2
    return k1, k2


@pytest.mark.parametrize("low", [0, 1])
@pytest.mark.parametrize("Re", [0.0, 200.0])
@pytest.mark.parametrize("k", [1, 3])
def test_x_fourier_modes_of_uniform_state(orc, Re, k, low):
    """On y-independent perturbations exp(i k x) of a uniform state at rest,
    J reduces to the linearised 1-D compressible Navier-Stokes symbol: a 3x3
    (p, u, s) block with the acoustic pair and conduction, and the shear mode
    lambda = -mu k''^2 / rho for v (derived by hand from the equations).  The
    reduced operator (low) has the same symbol with its own wavenumbers."""
    g, f, P = _problem(orc, nx=16, ny=12, Re=Re, Ma=0.4, low=low)
    q0 = _uniform(g, f)
    R = 1 / (GAM * f.Ma ** 2)
    p0 = R
    cp = GAM * R / (GAM - 1)
    mu0 = (1 / Re) if Re > 0 else 0.0
    lam0 = mu0 * cp / f.Pr
    Tp = (GAM - 1) / (GAM * p0)  # dT/dp at constant s, T0 = 1
    Ts = 1 / cp  # dT/ds at constant p
    k1, k2 = _symbols(g.lx / g.nx, k, g.nx, low)
    M = np.array([[-(GAM - 1) * lam0 * k2 * Tp, -1j * GAM * p0 * k1, -(GAM - 1) * lam0 * k2 * Ts],
                  [-1j * k1, -(4 / 3) * mu0 * k2, 0],
                  [-lam0 * k2 * Tp, 0, -lam0 * k2 * Ts]])
    lam, vec = np.linalg.eig(M)
    x = np.arange(g.nx) * g.lx / g.nx
    e = np.broadcast_to(np.exp(1j * k * 2 * math.pi / g.lx * x), (g.ny, g.nx)).reshape(-1)
    for i in range(3):
        v = np.zeros((4, g.ny * g.nx), dtype=complex)
        v[0], v[1], v[3] = vec[0, i] * e, vec[1, i] * e, vec[2, i] * e
        jv = orc.core.jv(P, q0, v.reshape(-1))
        assert np.linalg.norm(jv - lam[i] * v.reshape(-1)) < 1e-10 * np.linalg.norm(jv) + 1e-12
    if Re > 0:
        v = np.zeros((4, g.ny * g.nx), dtype=complex)
        v[2] = e
        jv = orc.core.jv(P, q0, v.reshape(-1))
        assert np.linalg.norm(jv + mu0 * k2 * v.reshape(-1)) < 1e-12 * np.linalg.norm(jv)
    if Re == 0:  # inviscid acoustic pair in closed form: +- i c0 k'
        c0 = math.sqrt(GAM * p0)
        assert np.allclose(sorted(lam.imag), sorted([-c0 * k1, 0.0, c0 * k1]), atol=1e-12)


@pytest.mark.parametrize("bulk", [0.0, 0.6])
def test_dissipation_of_uniform_strain(orc, bulk):
    """v0 = b y gives div u = b, s_yy = b and Phi = (4/3 + bulk) mu b^2;
    u0 = a y gives Phi = mu a^2.  Interior rows then satisfy
    p_t = -gamma p b + (gamma-1) Phi and s_t = Phi R/p (linear profiles are
    differentiated exactly), with mu from Sutherland's law at T = exp(s/c_p)."""
    g, f, P = _problem(orc, nx=8, ny=16, Re=50.0, bulk=bulk)
    R = 1 / (GAM * f.Ma ** 2)
    cp = GAM * R / (GAM - 1)
    s0 = 0.3 * cp  # T = exp(0.3)
    T = math.exp(0.3)
    mu = (1 / 50.0) * T ** 1.5 * (1 + f.S) / (T + f.S)
    y = g.y()
    a, b = 0.2, 0.05
    q = _uniform(g, f, s0=s0)
    q[1] = a * y[None, :, None]
    q[2] = b * y[None, :, None]
    r = orc.core.rhs(P, q).reshape(4, g.ny, g.nx)[:, 2:-2, :]
    p0 = R
    Phi = mu * a ** 2 + (4 / 3 + bulk) * mu * b ** 2
    assert np.allclose(r[0], -GAM * p0 * b + (GAM - 1) * Phi, rtol=1e-11, atol=1e-11)
    assert np.allclose(r[3], Phi * R / p0, rtol=1e-11, atol=1e-13)


def test_heat_flux_in_conservative_form(orc):
    """div(lambda grad T) in the expanded form lambda T'' + lambda'(T) T'^2
    matches the conservative form D(lambda(T) D T) up to discretisation error
    on a smooth temperature profile (pins lambda'(T) of Sutherland's law)."""
    g, f, P = _problem(orc, nx=4, ny=400, Re=10.0)
    R = 1 / (GAM * f.Ma ** 2)
    cp = GAM * R / (GAM - 1)
    y = g.y()
    q = _uniform(g, f)
    q[3] = (0.5 * np.tanh(y / 4))[None, :, None] * cp
    r = orc.core.rhs(P, q).reshape(4, g.ny, g.nx)
    T = np.exp(q[3, 0] / cp)  # uniform p: T = exp(s / c_p)
    mu = 0.1 * T ** 1.5 * (1 + f.S) / (T + f.S)
    lam = mu * cp / f.Pr
    dT = orc.core.deriv_field(P, T, 1, 1)
    heat = orc.core.deriv_field(P, lam.reshape(-1) * dT, 1, 1)
    sl = (slice(20, -20), 0)
    # s_t = (R/p) heat with p = R
    assert np.allclose(r[3][sl], heat.reshape(g.ny, g.nx)[sl], rtol=1e-6, atol=1e-8)


def test_nonreflective_boundaries_drop_incoming_waves(orc):
    """Linear-in-y perturbations carrying only X- (the wave running towards
    -y) leave the top row untouched and pass the bottom row unchanged; only X+
    the other way round (LODI-type reading, switch frozen on v0 = 0)."""
    g, f, P = _problem(orc, nx=8, ny=16, Re=0.0)
    q0 = _uniform(g, f)
    p0 = 1 / (GAM * f.Ma ** 2)
    c0 = math.sqrt(GAM * p0)
    y = np.broadcast_to(g.y()[:, None], (g.ny, g.nx))
    for sign in (+1, -1):  # sign -1: pure X- ; +1: pure X+
        v = np.zeros((4, g.ny, g.nx))
        v[0] = sign * c0 * y  # rho0 = 1
        v[2] = y
        jv = orc.core.jv(P, q0, v.reshape(-1).astype(complex)).real.reshape(4, g.ny, g.nx)
        interior_p = -GAM * p0  # -gamma p dv/dy
        interior_v = -sign * c0  # -(1/rho) dp/dy
        top, bot = jv[:, -1], jv[:, 0]
        assert np.allclose(jv[0, 1:-1], interior_p) and np.allclose(jv[2, 1:-1], interior_v)
        if sign < 0:  # X- incoming at the top: removed there, kept at the bottom
            assert np.allclose(top[0], 0.0, atol=1e-12) and np.allclose(top[2], 0.0, atol=1e-12)
            assert np.allclose(bot[0], interior_p) and np.allclose(bot[2], interior_v)
        else:
            assert np.allclose(bot[0], 0.0, atol=1e-12) and np.allclose(bot[2], 0.0, atol=1e-12)
            assert np.allclose(top[0], interior_p) and np.allclose(top[2], interior_v)


def test_tangent_is_linear(orc):
    g, f, P = _problem(orc, stretch=1.5)
    q0 = si.tanh_base_flow(g, f)
    a, b = si.random_complex(1, g.n), si.random_complex(2, g.n)
    lhs = orc.core.jv(P, q0, (0.3 - 2j) * a + 1.7 * b)
    rhs = (0.3 - 2j) * orc.core.jv(P, q0, a) + 1.7 * orc.core.jv(P, q0, b)
    assert np.linalg.norm(lhs - rhs) < 1e-14 * np.linalg.norm(lhs)


@pytest.mark.parametrize("dim", [2, 3])
def test_epsilon_quotient_taylor(orc, dim):
    """The exact (binary128) epsilon-quotient differs from the tangent by
    (eps/2) N''(v, v) + O(eps^2): the gap scales linearly in eps over six
    decades, and the double-precision literal quotient tracks it only while
    cancellation noise ~ eps_m/eps stays below it."""
    g, f, P = _problem(orc, nx=8, ny=12, dim=dim, nz=6 if dim == 3 else 1)
    q0 = si.perturbed_base_flow(g, f, seed=3)
    v = si.random_complex(4, g.n)
    jt = orc.core.jv(P, q0, v)
    gaps = []
    for eps in (1e-3, 1e-5, 1e-7, 1e-9):
        gaps.append(np.linalg.norm(orc.core.jv(P, q0, v, "quad", eps) - jt))
    slopes = np.diff(np.log10(gaps)) / -2.0
    assert np.all(np.abs(slopes - 1.0) < 0.02)
    lit = np.linalg.norm(orc.core.jv(P, q0, v, "literal", 1e-5) - jt)
    assert abs(lit / gaps[1] - 1.0) < 0.05


def test_quad_matches_double_rhs(orc):
    g, f, P = _problem(orc, nx=8, ny=12)
    q0 = si.perturbed_base_flow(g, f, seed=5)
    r1 = orc.core.rhs(P, q0)
    r2 = orc.core.rhs(P, q0, quad=True)
    assert np.linalg.norm(r1 - r2) < 1e-13 * np.linalg.norm(r2)


def test_dense_jacobian_columns_are_tangent(orc):
    g, f, P = _problem(orc, nx=8, ny=10)
    q0 = si.perturbed_base_flow(g, f, seed=9)
    J = orc.core.dense_jacobian(P, q0)
    v = si.random_complex(8, g.n)
    assert np.linalg.norm(J @ v - orc.core.jv(P, q0, v)) < 1e-13 * np.linalg.norm(J @ v)


@pytest.mark.parametrize("low", [0, 1])
@pytest.mark.parametrize("bulk", [0.0, 0.7])
def test_xz_fourier_symbol_of_uniform_3d_state(orc, bulk, low):
    """3-D pin of every viscous index: a uniform moving state (U, 0, W) with
    non-reference pressure and entropy (rho0, T0 != 1, so Sutherland's mu(T0)
    enters), perturbed by q' = (a + b y) exp(i (kx x + kz z)) on a uniform y
    grid (the bounded compact schemes differentiate a + b y exactly, closure
    rows included).  On interior rows J q' = E [S (a + b y) + Y b] with the
    5x5 matrices below, derived by hand from the linearised equations about a
    uniform state: convection -i(U k1x + W k1z); pressure gradient and
    divergence; mu (laplacian + d_i div / 3) + mu_v d_i div with pure second
    derivatives through the compact second-derivative symbols k2^2 and the
    mixed d_x d_z, d_x d_y, d_y d_z through products of first-derivative
    symbols; conduction lambda laplacian T' with T' = T0 ((1 - 1/gamma) p'/p0 +
    s'/c_p) in the p and s rows.  A transposed index in the 3-D viscous stress
    or a mixed derivative taken as a second derivative fails it.  The reduced
    operator (low: second-order explicit differences, which also differentiate
    a + b y exactly, end rows included) is pinned by the same symbol with its
    own modified wavenumbers."""
    nx, ny, nz = 8, 7, 6
    lx, lz = 3.0, 2.5
    g = si.Grid(3, nx, ny, nz, lx, -1.0, 2.0, lz, 0.0)
    f = si.Flow(0.6, 50.0, Pr=0.5)
    P = orc.Problem.from_inputs(g, f, bulk, low)
    gam, R = f.gamma, 1.0 / (f.gamma * f.Ma ** 2)
    cp = gam * R / (gam - 1)
    p0, s0, U, W = 1.3 * R, 0.3, 0.4, -0.7
    q0 = np.zeros((5, nz, ny, nx))
    q0[0], q0[1], q0[3], q0[4] = p0, U, W, s0
    rho0 = (p0 / R) ** (1 / gam) * math.exp(-s0 / cp)
    T0 = p0 / (rho0 * R)
    mu0 = (1 / f.Re) * T0 ** 1.5 * (1 + f.S) / (T0 + f.S)
    lam0, muv0 = mu0 * cp / f.Pr, bulk * mu0
    Tp, Ts = T0 * (gam - 1) / (gam * p0), T0 / cp  # T' = Tp p' + Ts s'
    mx, mz = 2, 1
    kx1, kx2 = _symbols(lx / nx, mx, nx, low)
    kz1, kz2 = _symbols(lz / nz, mz, nz, low)
    conv = -1j * (U * kx1 + W * kz1)
    lap = -(kx2 + kz2)  # second-derivative symbols (y part: d2/dy2 (a + b y) = 0)
    vd = (mu0 / 3 + muv0) / rho0  # coefficient of d_i div u
    S = np.zeros((5, 5), dtype=complex)
    S[0] = [conv + (gam - 1) * lam0 * lap * Tp, -gam * p0 * 1j * kx1, 0, -gam * p0 * 1j * kz1,
            (gam - 1) * lam0 * lap * Ts]
    S[1] = [-1j * kx1 / rho0, conv + mu0 / rho0 * lap + vd * (-kx2), 0, vd * (-kx1 * kz1), 0]
    S[2] = [0, 0, conv + mu0 / rho0 * lap, 0, 0]
    S[3] = [-1j * kz1 / rho0, vd * (-kz1 * kx1), 0, conv + mu0 / rho0 * lap + vd * (-kz2), 0]
    S[4] = [lam0 * lap * Tp / (rho0 * T0), 0, 0, 0, conv + lam0 * lap * Ts / (rho0 * T0)]
    Y = np.zeros((5, 5), dtype=complex)
    Y[0, 2] = -gam * p0
    Y[1, 2] = vd * 1j * kx1
    Y[2] = [-1 / rho0, vd * 1j * kx1, 0, vd * 1j * kz1, 0]
    Y[3, 2] = vd * 1j * kz1
    a = si.random_complex(21, 5)
    b = si.random_complex(22, 5)
    x = np.arange(nx) * lx / nx
    z = np.arange(nz) * lz / nz
    y = g.y()
    E = np.exp(1j * (2 * math.pi * mx / lx * x[None, None, :] + 2 * math.pi * mz / lz * z[:, None, None]))
    amp = a[:, None] + b[:, None] * y[None, :]                      # (5, ny)
    v = amp[:, None, :, None] * E[None]                             # (5, nz, ny, nx)
    expect = (S @ amp + (Y @ b)[:, None])[:, None, :, None] * E[None]
    jv = orc.core.jv(P, q0, v.reshape(-1)).reshape(5, nz, ny, nx)
    inner = slice(1, ny - 1)  # the non-reflective boundary rows have their own form
    err = np.abs(jv[:, :, inner] - expect[:, :, inner]).max()
    assert err < 1e-11 * np.abs(expect).max()
