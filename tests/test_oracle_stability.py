"""Physics and eigen pins of the oracle: growth rates of the tanh mixing
layer against the paper's Table validation_results, Cayley-IRAM on the
discretised operator against dense LAPACK, and the block-Jacobi blocks."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import stab_inputs as si

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "validation_results.json")))


def _beta_for_min_spacing(Ly: float, ny: int, dmin: float) -> float:
    """Stretching parameter of y(eta) = yc + (Ly/2) sinh(beta (2 eta - 1))/sinh(beta)
    whose smallest spacing (at the centre) is dmin."""
    from scipy.optimize import brentq
    return brentq(lambda b: Ly * b / math.sinh(b) / (ny - 1) - dmin, 1e-3, 40.0)


def _fourier_jacobian(orc, P, q0, m: int = 1) -> np.ndarray:
    """J restricted to the x-Fourier mode exp(2 pi i m x / Lx): the base state
    does not depend on x, so J commutes with x-shifts and its columns at x = 0
    give the whole mode, J_m = sum_x J[(., x), (., 0)] exp(-2 pi i m x / nx)."""
    nx, ny, npts = P.nx, P.ny, P.nx * P.ny
    cols = np.array([v * npts + j * nx for v in range(4) for j in range(ny)])
    Jc = orc.core.jacobian_columns(P, q0, cols).reshape(4, ny, nx, 4 * ny)
    ph = np.exp(-2j * np.pi * m * np.arange(nx) / nx)
    return np.einsum("vyxc,x->vyc", Jc, ph).reshape(4 * ny, 4 * ny)


def _kh_growth(J: np.ndarray) -> float:
    """Largest real part among the non-propagating eigenvalues (the tanh
    layer's Kelvin-Helmholtz mode has zero phase speed)."""
    lam = sla.eigvals(J)
    return float(lam[np.abs(lam.imag) < 1e-6].real.max())


# Reading of Table validation_config's Reynolds number (the paper does not
# give its reference length): an independent 1-D viscous solve of the same
# equations gives a maximum growth rate of 0.1396 at Re_delta = 1000 but
# 0.1269 at Re_delta = 100, where the table prints 0.1273 / 0.1270 and Mack
# 0.1271; the table's Re = 1000 is read as Re_delta = 100 (a reference length
# of ten half-thicknesses).
RE_TABLE_TO_DELTA = 0.1


def test_linstab1d_reproduces_literature():
    """The independent 1-D solver (tests/linstab1d.py) against published
    inviscid values: Michalke's incompressible tanh layer (maximum growth
    0.1897 at alpha 0.4446), Mack's compressible values of Table
    validation_results, and the paper's L1 = 15.83 = 2 pi / alpha_max at
    M = 0.5 (Sec. Numerical Experiments)."""
    pytest.importorskip("sympy")
    import linstab1d as L

    w, _ = L.kh_growth(0.4446, 0.4446, 0.01, None, N=200, Y=120, beta=5.0)
    assert abs(w - 0.1897) < 5e-4
    a05, w05 = L.alpha_max(0.5, None, N=160, Y=100, beta=5.0)
    assert abs(w05 - GOLD["cases"]["V02"]["mack"]) < 2e-3 * w05
    assert abs(2 * math.pi / a05 - GOLD["L1_numerical_experiments"]) < 2e-3 * GOLD["L1_numerical_experiments"]
    a09, w09 = L.alpha_max(0.9, None, N=160, Y=200, beta=5.0)
    assert abs(w09 - GOLD["cases"]["V03"]["mack"]) < 2e-3 * w09


@pytest.mark.parametrize("Ma,Re,Pr,bulk,a,Y,ny", [(0.5, None, 0.71, 0.0, 0.4, 50.0, 192),
                                                    (0.5, 100.0, 0.71, 0.0, 0.4, 50.0, 192),
                                                    (0.9, 300.0, 0.2, 0.6, 0.22, 150.0, 256)])
def test_oracle_fourier_mode_matches_independent_1d_solve(orc, Ma, Re, Pr, bulk, a, Y, ny):
    """Pin of the 2-D oracle's whole linearised operator (inviscid and
    viscous terms, conduction, bulk viscosity, Sutherland law) against the
    independent 1-D solver: the Kelvin-Helmholtz eigenvalue of the oracle's J
    restricted to one x-Fourier mode equals that of the 1-D symbolic
    linearisation evaluated with the same compact-scheme modified
    wavenumbers, to the y-discretisation error (< 2e-6 relative)."""
    pytest.importorskip("sympy")
    import linstab1d as L

    nx = 16
    g = si.Grid(2, nx, ny, 1, 2 * math.pi / a, -Y, Y, 1.0, 3.0 if Y < 100 else 4.5)
    f = si.Flow(Ma, Re if Re else 0.0, Pr=Pr)
    P = orc.Problem.from_inputs(g, f, bulk)
    w = _kh_growth(_fourier_jacobian(orc, P, si.tanh_base_flow(g, f)))
    hx = g.lx / nx
    w1, _ = L.kh_growth(L.lele_k1(a, hx), L.lele_k2(a, hx), Ma, Re, N=200 if Y < 100 else 240, Y=Y,
                        beta=4.0 if Y < 100 else 4.5, Pr=Pr, bulk=bulk)
    assert abs(w - w1) < 2e-6 * w1


@pytest.mark.slow
@pytest.mark.parametrize("case", ["V01", "V02", "V03", "V04", "V05", "V06", "V07", "V08"])
def test_growth_rates_against_paper_table(orc, case):
    """Table validation_results, every row: L1 = 2 pi / alpha_max of the
    least stable mode (alpha_max from the independent 1-D solve), y extent
    8 L1 stretched to a minimum spacing of 0.08 delta, the table's resolution;
    the oracle's growth rate (J restricted to the x-Fourier mode of one
    wavelength) is within 2 % of the paper's computed value and within 0.5 %
    of Mack's.  Re: see RE_TABLE_TO_DELTA."""
    pytest.importorskip("sympy")
    import linstab1d as L

    c = GOLD["cases"][case]
    Re = c["Re"] * RE_TABLE_TO_DELTA if c["Re"] else None
    a, w1 = L.alpha_max(c["Ma"], Re, N=160, Y=150.0 if c["Ma"] > 0.8 else 80.0, beta=5.0)
    L1 = 2 * math.pi / a
    nx, ny = c["res"]
    Ly = 8 * L1
    g = si.Grid(2, nx, ny, 1, L1, -Ly / 2, Ly / 2, 1.0, _beta_for_min_spacing(Ly, ny, GOLD["min_dy"]))
    f = si.Flow(c["Ma"], Re if Re else 0.0)
    P = orc.Problem.from_inputs(g, f)
    w = _kh_growth(_fourier_jacobian(orc, P, si.tanh_base_flow(g, f)))
    assert abs(w - c["omega"]) < 0.02 * c["omega"]
    assert abs(w - c["mack"]) < 0.005 * c["mack"]
    assert abs(w - w1) < 1e-3 * w1


def test_double_kh_eigenvalue_and_trends(orc):
    """On the 2-D grid the +-alpha Fourier pair makes the least stable mode a
    double eigenvalue of the dense J; viscosity and compressibility lower the
    growth rate."""
    def growth(Ma, Re):
        L1 = GOLD["L1_numerical_experiments"]
        g = si.Grid(2, 16, 48, 1, L1, -4 * L1, 4 * L1, 1.0, _beta_for_min_spacing(8 * L1, 48, 0.12))
        f = si.Flow(Ma, Re)
        P = orc.Problem.from_inputs(g, f)
        lam = sla.eigvals(orc.core.dense_jacobian(P, si.tanh_base_flow(g, f)))
        return np.sort(lam[np.abs(lam.imag) < 1e-6].real)[::-1]
    w05 = growth(0.5, 0.0)
    assert abs(w05[0] - w05[1]) < 1e-8 * w05[0]
    assert growth(0.5, 100.0)[0] < w05[0]
    assert growth(0.9, 0.0)[0] < w05[0] < growth(0.1, 0.0)[0]


def _c1_like(orc, nx=8, ny=16):
    g, f = si.mixing_layer_2d(nx, ny)
    P = orc.Problem.from_inputs(g, f)
    return g, f, P, si.tanh_base_flow(g, f)


def test_iram_on_operator_with_exact_cayley_matches_dense_lapack(orc):
    """Algorithm iram on C = (J - sigma I)^-1 (J - tau I) of the discretised
    operator, C applied by a dense LU: the k converged Ritz values map back to
    the k eigenvalues of J with the largest |theta| (dense LAPACK)."""
    g, f, P, q0 = _c1_like(orc)
    sigma, tau = 0.2j, -1 + 0.2j
    J = orc.core.dense_jacobian(P, q0)
    lu = sla.lu_factor(J - sigma * np.eye(g.n))
    res = orc.krylov.iram(lambda v: sla.lu_solve(lu, J @ v - tau * v), si.start_vector(0x5EED, g.n),
                          6, 30, 1e-12, sigma, tau)
    assert res.nconv == 6
    ref, _ = orc.stability.dense_reference(J, sigma, tau, 6)
    for l in res.lam:
        assert np.abs(ref - l).min() < 1e-12 * abs(l)
    for l in ref:
        assert np.abs(res.lam - l).min() < 1e-12 * abs(l)


@pytest.mark.slow
def test_cayley_iram_with_gmres_inner_solves(orc):
    """The full oracle path (inexact Cayley by GMRES on the matrix-free
    tangent) reaches the double Kelvin-Helmholtz eigenvalue of the dense J to
    1e-8 with true residual below 1e-8."""
    g, f, P, q0 = _c1_like(orc)
    J = orc.core.dense_jacobian(P, q0)
    lam_all = sla.eigvals(J)
    res, resid, counts = orc.stability.cayley_eigs(P, q0, 0.25, -1.0, nev=2, ncv=10, tol=1e-12, gmres_m=30,
                                                    gmres_tol=1e-12, v0=si.start_vector(0x5EED, g.n))
    assert res.nconv == 2
    for l in res.lam:
        assert np.abs(lam_all - l).min() < 1e-8 * abs(l)
        assert abs(l.real - 0.1065529227739) < 1e-8
    assert resid.max() < 1e-8


def test_block_jacobi_blocks_and_factorisation(orc):
    g, f, P, q0 = _c1_like(orc, 8, 16)
    sigma = 0.25
    J = orc.core.dense_jacobian(P, q0)
    tile = (4, 4)
    B = orc.stability.blocks_from_dense(J, P, tile, sigma)
    assert B.shape == (8, 64, 64)
    # blocks from columns agree with the dense principal submatrices
    for t in (0, 5):
        Bt = orc.stability.block_from_columns(P, q0, tile, t, sigma)
        assert np.abs(Bt - B[t]).max() < 1e-12 * np.abs(B[t]).max()
    # tiles partition the dofs
    idx = np.concatenate(orc.stability.tile_dofs(P, tile))
    assert np.array_equal(np.sort(idx), np.arange(g.n))
    # LU with partial pivoting reconstructs the block; the apply inverts it
    Pm, L, U = sla.lu(B[3])
    assert np.abs(Pm @ L @ U - B[3]).max() < 1e-13 * np.abs(B[3]).max()
    M = orc.stability.BlockJacobi(P, tile, B)
    x = si.random_complex(3, g.n)
    Mx = np.zeros_like(x)
    for d, Bt in zip(orc.stability.tile_dofs(P, tile), B):
        Mx[d] = Bt @ x[d]
    assert np.linalg.norm(M(Mx) - x) < 1e-10 * np.linalg.norm(x)


def test_block_jacobi_reduces_gmres_iterations(orc):
    g, f, P, q0 = _c1_like(orc, 16, 32)
    sigma = 0.25
    J = orc.core.dense_jacobian(P, q0)
    A = J - sigma * np.eye(g.n)
    b = si.random_complex(4, g.n)
    M = orc.stability.BlockJacobi(P, (8, 8), orc.stability.blocks_from_dense(J, P, (8, 8), sigma))
    _, st0 = orc.krylov.fgmres(lambda z: A @ z, b, None, m=40, tol=1e-8, max_restarts=200)
    _, st1 = orc.krylov.fgmres(lambda z: A @ z, b, M, m=40, tol=1e-8, max_restarts=200)
    assert st1.converged and st1.matvecs < st0.matvecs


@pytest.mark.parametrize("dim,shape,tile", [(2, (8, 12, 1), (4, 12)), (2, (16, 16, 1), (8, 8)),
                                            (3, (8, 8, 6), (4, 8, 2))])
def test_reduced_operator_tiles_are_block_tridiagonal_in_y_levels(orc, dim, shape, tile):
    """The structure the reduced-operator preconditioner's factorisation relies on (reading of the
    reduced operator: three-point stencils, four-point end rows): inside every tile, grouping the points in
    levels of two y lines, a level of J_low couples only to itself and its two neighbouring levels, the
    domain's y boundaries included.  The compact operator's tiles are dense along y (its derivatives are
    global on a line), so the same grouping has nonzero couplings two or more levels apart there."""
    nx, ny, nz = shape
    if dim == 2:
        g, f = si.mixing_layer_2d(nx, ny)
    else:
        g = si.Grid(3, nx, ny, nz, si.LX_04, -15, 15, si.LX_04)
        f = si.Flow(0.5, 800.0)
    q0 = si.tanh_base_flow(g, f)
    JL = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f, low_order=1), q0)
    J = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f), q0)
    npts = nx * ny * nz
    tx, ty = tile[0], tile[1]
    tz = tile[2] if dim == 3 else 1
    nlev = ty // 2
    for t, dofs in enumerate(orc.stability.tile_dofs(orc.Problem.from_inputs(g, f), tile[:dim])):
        pts = dofs % npts
        ylocal = (pts // nx) % ny % ty
        lev = ylocal // 2
        far = np.abs(lev[:, None] - lev[None, :]) > 1
        blk_low = JL[np.ix_(dofs, dofs)]
        assert np.all(blk_low[far] == 0.0), t
        if nlev > 2:
            assert np.abs(J[np.ix_(dofs, dofs)][far]).max() > 0.0
