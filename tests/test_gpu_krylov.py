"""GPU parity of the Krylov layer through the C ABI: CGS2 (Sec. Krylov
methods), GMRES (Sec. Iterative solvers) and Cayley-IRAM (Algorithm iram),
against the oracle and dense LAPACK."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import stab_inputs as si
from gpu_util import rel_err

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "c1_dense_eigs.json")


def _stab(nx, ny, **opts):
    from paper_1502_03701_gb300 import Stab
    g, f = si.mixing_layer_2d(nx, ny)
    q0 = si.tanh_base_flow(g, f)
    return Stab(q0, g, f.Ma, f.Re, f.Pr, **opts), g, f, q0


def test_cgs2_matches_oracle(orc):
    import torch
    S, g, f, q0 = _stab(16, 24)
    n = g.n
    rng = np.random.default_rng(3)
    for k in (0, 1, 7, 33):
        Vh = np.linalg.qr(rng.standard_normal((n, max(k, 1))) + 1j * rng.standard_normal((n, max(k, 1))))[0][:, :k]
        w = si.random_complex(40 + k, n)
        V = torch.from_numpy(np.ascontiguousarray(Vh.T)).cuda()  # column j contiguous
        wd = torch.from_numpy(w.copy()).cuda()
        h, nrm = S.orthogonalize(V, k, wd)
        # products are exact FP32 two-products of operands split to ~2^-47 (pair
        # arithmetic), so coefficients carry errors of order 2^-45 ||w||
        wn = np.linalg.norm(w)
        if k:
            href, wref = orc.krylov.cgs2(Vh, w)
            assert np.abs(h - href).max() < 1e-12 * wn
        else:
            wref = w
        assert rel_err(wd.cpu().numpy(), wref) < 1e-12
        assert abs(nrm - np.linalg.norm(wref)) < 1e-12 * wn
        if k:
            assert np.abs(Vh.conj().T @ wd.cpu().numpy()).max() < 1e-12 * wn
    S.close()


@pytest.mark.parametrize("sigma", [0.25, 0.1 + 0.3j])
def test_gmres_solution_against_dense_solve(orc, sigma):
    import torch
    S, g, f, q0 = _stab(8, 16, eps_mode=2, gmres_m=40, gmres_tol=1e-12, gmres_max_restarts=400)
    J = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f), q0)
    A = J - sigma * np.eye(g.n)
    b = si.random_complex(77, g.n)
    x = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    st, iters = S.solve(sigma, torch.from_numpy(b).cuda(), x)
    assert st == 0 and iters > 0
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xh) <= 1.05e-12 * np.linalg.norm(b)
    ref = sla.solve(A, b)
    assert rel_err(xh, ref) < 1e-7  # conditioning of J - sigma I times the tolerance
    S.close()


def test_eigs_match_dense_lapack_tiny(orc):
    """8 x 16 layer, real pole near the Kelvin-Helmholtz mode: the two wanted
    Ritz values (the double eigenvalue of the +-alpha pair) match dense LAPACK
    eigenvalues of J to 1e-8 relative with true residuals below 1e-8."""
    S, g, f, q0 = _stab(8, 16, eps_mode=2, gmres_m=30, gmres_tol=1e-12, gmres_max_restarts=400)
    J = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f), q0)
    lam_all = sla.eigvals(J)
    r = S.eigs(0.25, -1.0, nev=2, ncv=12, tol=1e-11, v0=None)
    assert r.status == 0 and r.nconv == 2
    for l in r.lam:
        assert np.abs(lam_all - l).min() < 1e-8 * abs(l)
    ref, _ = orc.stability.dense_reference(J, 0.25, -1.0, 2)
    for l in ref:
        assert np.abs(r.lam - l).min() < 1e-8 * abs(l)
    assert r.resid.max() < 1e-8
    assert r.stats["jv_calls"] > 0 and r.stats["gmres_solves"] > 0
    S.close()


def test_eigs_small_layer_against_stored_dense_eigenvalues():
    """32 x 64 layer (8,192 unknowns), sigma = 0.25, tau = -1: eigenvalues
    against the stored dense LAPACK values written by the oracle."""
    import torch
    gold = json.load(open(GOLD))
    ref = [complex(*l) for l in gold["sets"][1]["lambda"]]
    S, g, f, q0 = _stab(32, 64, eps_mode=2, gmres_m=30, gmres_tol=1e-12, gmres_max_restarts=2000)
    v0 = torch.from_numpy(si.start_vector(0x5EED, g.n)).cuda()
    r = S.eigs(0.25, -1.0, nev=2, ncv=12, tol=1e-10, v0=v0)
    assert r.status == 0 and r.nconv == 2
    for l in r.lam:
        assert np.abs(np.array(ref) - l).min() < 1e-8 * abs(l)
    assert r.resid.max() < 1e-8
    S.close()


def test_eigs_eps_mode_offset_is_small(orc):
    """With the epsilon-quotient (eps ~ 1e-7 per unit vector) the eigenvalues
    move from the tangent ones by O(eps); both are reported."""
    S0, g, f, q0 = _stab(8, 16, eps_mode=2, gmres_tol=1e-12, gmres_max_restarts=400)
    S1, _, _, _ = _stab(8, 16, eps_mode=0, gmres_tol=1e-12, gmres_max_restarts=400)
    a = S0.eigs(0.25, -1.0, nev=2, ncv=12, tol=1e-11)
    b = S1.eigs(0.25, -1.0, nev=2, ncv=12, tol=1e-11)
    assert a.nconv == 2 and b.nconv == 2
    assert np.abs(np.sort_complex(a.lam) - np.sort_complex(b.lam)).max() < 1e-5
    S0.close()
    S1.close()


def test_eigs_rejects_bad_arguments():
    from paper_1502_03701_gb300 import StabError
    S, g, f, q0 = _stab(8, 16)
    with pytest.raises(StabError, match="INVALID_ARG"):
        S.eigs(0.25, -1.0, nev=5, ncv=5, tol=1e-8)
    S.close()


def test_eigs_3d_mixed_precision_matches_dense_lapack(orc):
    """3-D layer (8 x 8 x 6, 1,920 unknowns), block-Jacobi over 4 x 4 x 2 tiles
    stored in FP32 inside the FP64 flexible GMRES (the mixed-precision path):
    the wanted Cayley eigenvalue (pole 0.5 right of the spectrum, so the inner
    solves converge: cond(J - 0.5 I) = 91; the least stable real mode has
    |theta| 2.026 against 2.002 next) matches dense LAPACK to 1e-8 relative,
    as the plain FP64 path does."""
    from paper_1502_03701_gb300 import Stab
    g = si.Grid(3, 8, 8, 6, si.LX_04, -15, 15, 6.0)
    f = si.Flow(0.4, 500.0)
    q0 = si.tanh_base_flow(g, f)
    J = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f), q0)
    ref, _ = orc.stability.dense_reference(J, 0.5, -1.0, 1)
    for prec in (32, 64):
        S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2, precond=1, tile=(4, 4, 2), precond_prec=prec, gmres_m=30,
                 gmres_tol=1e-12, gmres_max_restarts=400)
        r = S.eigs(0.5, -1.0, nev=1, ncv=20, tol=1e-10)
        assert r.status == 0 and r.nconv == 1, prec
        for l in ref:
            assert np.abs(r.lam - l).min() < 1e-8 * abs(l), (prec, r.lam, ref)
        assert r.resid.max() < 1e-8
        S.close()


@pytest.mark.parametrize("sigma", [0.25, 0.1 + 0.3j])
def test_fp32_basis_gmres_refines_to_fp64_tolerance(orc, sigma):
    """GMRES with an FP32 Krylov basis (J v, solution update and restart
    residuals in FP64): the restarts refine the solution to the FP64
    tolerance, checked against a dense solve."""
    import torch
    S, g, f, q0 = _stab(8, 16, eps_mode=2, gmres_m=40, gmres_tol=1e-12, gmres_max_restarts=400, gmres_basis_prec=32)
    J = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f), q0)
    A = J - sigma * np.eye(g.n)
    b = si.random_complex(77, g.n)
    x = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    st, iters = S.solve(sigma, torch.from_numpy(b).cuda(), x)
    assert st == 0 and iters > 0
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xh) <= 1.05e-12 * np.linalg.norm(b)
    assert rel_err(xh, sla.solve(A, b)) < 1e-7
    S.close()


def test_fp32_basis_preconditioned_gmres_and_eigs(orc):
    """FP32 basis with block-Jacobi (FP32 inverses) on 32 x 64: the same solution
    as the FP64 flexible GMRES to 1e-8; eigenvalues of the tiny layer match LAPACK."""
    import torch
    common = dict(eps_mode=2, precond=1, tile=(8, 8), precond_prec=32, gmres_m=50, gmres_tol=1e-10,
                  gmres_max_restarts=400)
    S64, g, f, q0 = _stab(32, 64, **common)
    S32, _, _, _ = _stab(32, 64, gmres_basis_prec=32, **common)
    b = torch.from_numpy(si.random_complex(5, g.n)).cuda()
    x64, x32 = torch.zeros_like(b), torch.zeros_like(b)
    st64, it64 = S64.solve(1.0, b, x64)
    st32, it32 = S32.solve(1.0, b, x32)
    assert st64 == 0 and st32 == 0 and it32 <= 1.5 * it64
    assert rel_err(x32.cpu().numpy(), x64.cpu().numpy()) < 1e-8
    S64.close()
    S32.close()
    S, g, f, q0 = _stab(8, 16, eps_mode=2, gmres_m=30, gmres_tol=1e-12, gmres_max_restarts=400, gmres_basis_prec=32)
    J = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f), q0)
    ref, _ = orc.stability.dense_reference(J, 0.25, -1.0, 2)
    r = S.eigs(0.25, -1.0, nev=2, ncv=12, tol=1e-11)
    assert r.status == 0 and r.nconv == 2
    for l in ref:
        assert np.abs(r.lam - l).min() < 1e-8 * abs(l)
    assert r.resid.max() < 1e-8
    S.close()


@pytest.mark.parametrize("sigma,k", [(0.25, 2), (0.1 + 0.3j, 4)])
def test_lgmres_solution_against_dense_solve_and_oracle(orc, sigma, k):
    """LGMRES (augmented restarts, Sec. Iterative solvers) on the 8 x 16
    layer: the solution meets the tolerance against the dense operator,
    equals the dense solve, and takes the oracle LGMRES's number of J v
    products (the augmentation steps take none)."""
    import torch
    m = 12
    S, g, f, q0 = _stab(8, 16, eps_mode=2, gmres_m=m, lgmres_k=k, gmres_tol=1e-12, gmres_max_restarts=2000)
    J = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f), q0)
    A = J - sigma * np.eye(g.n)
    b = si.random_complex(78, g.n)
    x = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    before = S.stats()["jv_calls"]
    st, iters = S.solve(sigma, torch.from_numpy(b).cuda(), x)
    jv = S.stats()["jv_calls"] - before
    S.close()
    assert st == 0 and iters > 0
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xh) <= 1.05e-12 * np.linalg.norm(b)
    assert rel_err(xh, sla.solve(A, b)) < 1e-7
    xo, so = orc.krylov.lgmres(lambda z: A @ z, b, None, m=m, k=k, tol=1e-12, max_restarts=2000)
    assert so.converged
    assert abs(jv - so.matvecs) <= max(m, so.matvecs // 20), (jv, so.matvecs)


def test_lgmres_preconditioned_above_16k_and_eigs(orc):
    """LGMRES with block-Jacobi on 64 x 64 (16,384 unknowns, selective
    reorthogonalisation): the true residual, measured with the oracle's
    tangent J v, meets the tolerance; Cayley-IRAM with LGMRES inner solves
    finds the dense LAPACK eigenvalues of the 8 x 16 layer."""
    import torch
    g, f = si.mixing_layer_2d(64, 64)
    from paper_1502_03701_gb300 import Stab
    q0 = si.tanh_base_flow(g, f)
    S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2, precond=1, tile=(8, 8), gmres_m=40, lgmres_k=3,
             gmres_tol=1e-10, gmres_max_restarts=400)
    b = si.random_complex(92, g.n)
    x = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    st, iters = S.solve(0.5 + 0.2j, torch.from_numpy(b).cuda(), x)
    S.close()
    assert st == 0
    xh = x.cpu().numpy()
    P = orc.Problem.from_inputs(g, f)
    r = b - (orc.core.jv(P, q0, xh, "tangent") - (0.5 + 0.2j) * xh)
    assert np.linalg.norm(r) <= 1.1e-10 * np.linalg.norm(b)
    S, g, f, q0 = _stab(8, 16, eps_mode=2, gmres_m=20, lgmres_k=2, gmres_tol=1e-12, gmres_max_restarts=400)
    J = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f), q0)
    ref, _ = orc.stability.dense_reference(J, 0.25, -1.0, 2)
    res = S.eigs(0.25, -1.0, nev=2, ncv=12, tol=1e-11)
    S.close()
    assert res.status == 0 and res.nconv == 2
    for l in ref:
        assert np.abs(res.lam - l).min() < 1e-8 * abs(l)
    assert res.resid.max() < 1e-8


def test_lgmres_option_checks():
    from paper_1502_03701_gb300 import StabError
    with pytest.raises(StabError, match="INVALID_ARG"):
        _stab(8, 16, gmres_m=4, lgmres_k=4)
    with pytest.raises(StabError, match="UNSUPPORTED"):
        _stab(8, 16, gmres_m=10, lgmres_k=2, gmres_basis_prec=32)


def test_nested_fp32_inner_gmres_under_fp64_fgmres(orc):
    """Mixed precision by nesting: FP64 flexible GMRES whose directions are
    FP32-basis inner GMRES(10) solves (block-Jacobi inside, FP32 inverses):
    the solution still meets the FP64 tolerance against the oracle's exact
    tangent and equals the flat FGMRES solution; Cayley-IRAM with the nested
    inner solver finds the dense LAPACK eigenvalues of the 8 x 16 layer."""
    import torch
    common = dict(eps_mode=2, precond=1, tile=(8, 8), precond_prec=32, gmres_tol=1e-10, gmres_max_restarts=400)
    S0, g, f, q0 = _stab(32, 64, gmres_m=50, **common)
    S1, _, _, _ = _stab(32, 64, gmres_m=20, gmres_inner_m=10, gmres_inner_tol=1e-3, **common)
    b = torch.from_numpy(si.random_complex(5, g.n)).cuda()
    x0, x1 = torch.zeros_like(b), torch.zeros_like(b)
    st0, it0 = S0.solve(1.0, b, x0)
    jv_before = S1.stats()["jv_calls"]
    st1, it1 = S1.solve(1.0, b, x1)
    jv1 = S1.stats()["jv_calls"] - jv_before
    assert st0 == 0 and st1 == 0
    assert jv1 > it1  # the inner solves' J v products are counted
    assert rel_err(x1.cpu().numpy(), x0.cpu().numpy()) < 1e-8
    xh, bh = x1.cpu().numpy(), b.cpu().numpy()
    P = orc.Problem.from_inputs(g, f)
    r = bh - (orc.core.jv(P, q0, xh, "tangent") - 1.0 * xh)
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(bh)
    S0.close()
    S1.close()
    S, g, f, q0 = _stab(8, 16, eps_mode=2, gmres_m=12, gmres_inner_m=8, gmres_tol=1e-12, gmres_max_restarts=400)
    J = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f), q0)
    ref, _ = orc.stability.dense_reference(J, 0.25, -1.0, 2)
    res = S.eigs(0.25, -1.0, nev=2, ncv=12, tol=1e-11)
    S.close()
    assert res.status == 0 and res.nconv == 2
    for l in ref:
        assert np.abs(res.lam - l).min() < 1e-8 * abs(l)
    assert res.resid.max() < 1e-8
    from paper_1502_03701_gb300 import StabError
    with pytest.raises(StabError, match="UNSUPPORTED"):
        _stab(8, 16, gmres_inner_m=4, gmres_basis_prec=32)
