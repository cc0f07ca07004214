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


def _validation_problem(orc, Ma, Re, nx=16, ny=64):
    L1 = GOLD["L1"]
    # 8 L1 in y, sinh stretching giving a minimum spacing of ~0.08 delta (Sec. Model problem)
    g = si.Grid(2, nx, ny, 1, L1, -4 * L1, 4 * L1, 1.0, 5.65)
    f = si.Flow(Ma, Re if Re else 0.0)
    return g, f, orc.Problem.from_inputs(g, f)


def _growth(orc, Ma, Re):
    g, f, P = _validation_problem(orc, Ma, Re)
    J = orc.core.dense_jacobian(P, si.tanh_base_flow(g, f))
    lam = sla.eigvals(J)
    real = lam[np.abs(lam.imag) < 1e-6].real
    return np.sort(real)[::-1]


@pytest.mark.slow
def test_growth_rates_against_paper_table(orc):
    """Least-stable stationary mode at alpha = 2 pi / L1: V05 (M 0.1) and V06
    (M 0.5) within 2 % of the paper's computed and Blumen's values; the mode
    is a double eigenvalue (the +-alpha Fourier pair); viscosity (Re 1000)
    lowers the growth rate; compressibility lowers it monotonically."""
    c = GOLD["cases"]
    w01 = _growth(orc, 0.1, None)
    w05 = _growth(orc, 0.5, None)
    w05v = _growth(orc, 0.5, 1000)
    w09 = _growth(orc, 0.9, None)
    assert abs(w01[0] - w01[1]) < 1e-8 * w01[0]  # double eigenvalue
    assert abs(w01[0] - c["V05"]["blumen"]) < 0.02 * c["V05"]["blumen"]
    assert abs(w01[0] - c["V05"]["omega"]) < 0.02 * c["V05"]["omega"]
    assert abs(w05[0] - c["V06"]["blumen"]) < 0.02 * c["V06"]["blumen"]
    assert abs(w05[0] - c["V06"]["omega"]) < 0.02 * c["V06"]["omega"]
    assert w05v[0] < w05[0]
    assert w09[0] < w05[0] < w01[0]


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
