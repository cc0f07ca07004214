"""GPU parity of the reduced-operator preconditioner (precond = 2; Sec.
Numerical experiments and Conclusions: block-Jacobi blocks built from a
non-compact, lower-order discretisation of N).  The tile blocks are the
principal submatrices of the oracle's tangent Jacobian of the second-order
explicit operator; they are factorised in block-tridiagonal form (levels of
two y lines), so the apply is checked against the oracle's dense LU of the
same blocks, and the preconditioned FGMRES against the oracle's FGMRES."""
import numpy as np
import pytest

import stab_inputs as si
from gpu_util import max_rel_err, rel_err

pytestmark = pytest.mark.gpu


def _make(g, f, general=False, **opts):
    from paper_1502_03701_gb300 import Stab
    q0 = si.perturbed_base_flow(g, f, seed=31) if general else si.tanh_base_flow(g, f)
    return Stab(q0, g, f.Ma, f.Re, f.Pr, precond=2, **opts), q0


BLOCK_CASES = [
    ("2d_visc", si.Grid(2, 16, 16, 1, si.LX_04, -15, 15), si.Flow(0.3, 1000.0), False, (4, 8, 1), (0, 3, 7)),
    ("2d_stretched_general_full_y", si.Grid(2, 12, 18, 1, si.LX_04, -15, 15, 1.0, 1.4), si.Flow(0.6, 300.0), True,
     (2, 18, 1), (0, 5)),
    ("2d_inviscid", si.Grid(2, 16, 12, 1, si.LX_04, -15, 15), si.Flow(0.9, 0.0), False, (8, 4, 1), (1, 5)),
    ("3d_visc", si.Grid(3, 8, 8, 6, si.LX_04, -15, 15, 6.0), si.Flow(0.4, 500.0), False, (4, 4, 2), (0, 7, 11)),
]


@pytest.mark.parametrize("name,g,f,general,tile,tiles", BLOCK_CASES, ids=[c[0] for c in BLOCK_CASES])
def test_reduced_blocks_match_oracle(orc, name, g, f, general, tile, tiles):
    """Assembled reduced-operator tile blocks (second-order explicit
    derivatives of the perturbation and of the base state) equal the oracle's
    principal submatrices of J_low - sigma I to 1e-11."""
    sigma = 0.2 + 0.1j
    S, q0 = _make(g, f, general, tile=tile)
    PL = orc.Problem.from_inputs(g, f, low_order=1)
    for t in tiles:
        got = S.precond_block(sigma, t)
        ref = orc.stability.block_from_columns(PL, q0, tile[:g.dim], t, sigma)
        assert max_rel_err(got, ref) < 1e-11, (name, t)
    S.close()


APPLY_CASES = [
    ("2d_tall_tiles", si.mixing_layer_2d(16, 32), (4, 32), 64, 1e-9),
    ("2d_tall_tiles_fp32", si.mixing_layer_2d(16, 32), (4, 32), 32, 1e-3),
    ("2d_square_tiles", si.mixing_layer_2d(16, 32), (8, 8), 64, 1e-9),
    ("3d", (si.Grid(3, 8, 8, 6, si.LX_04, -15, 15, si.LX_04), si.Flow(0.5, 800.0)), (2, 8, 2), 64, 1e-9),
]


@pytest.mark.parametrize("name,gf,tile,prec,tol", APPLY_CASES, ids=[c[0] for c in APPLY_CASES])
def test_reduced_apply_matches_oracle_lu(orc, name, gf, tile, prec, tol):
    """z = M^{-1} q by the block-tridiagonal factors equals the oracle's LU
    solve of the same tile blocks: to rounding with FP64 factors, to FP32
    roundoff times the blocks' conditioning with FP32 factors."""
    import torch
    g, f = gf
    S, q0 = _make(g, f, tile=tile, precond_prec=prec)
    sigma = 0.25 + 0.05j
    S.precond_build(sigma)
    PL = orc.Problem.from_inputs(g, f, low_order=1)
    J = orc.core.dense_jacobian(PL, q0)
    M = orc.stability.BlockJacobi(PL, tile, orc.stability.blocks_from_dense(J, PL, tile, sigma))
    for seed in (12, 13):
        q = si.random_complex(seed, g.n)
        z = torch.empty(g.n, dtype=torch.complex128, device="cuda")
        S.precond_apply(torch.from_numpy(q).cuda(), z)
        assert rel_err(z.cpu().numpy(), M(q)) < tol, name
    S.close()


def test_reduced_preconditioner_fgmres_against_oracle(orc):
    """FGMRES(50) to 1e-10 at sigma = 1 on the 32 x 64 layer with the reduced
    blocks over full-y tiles of 8 x 64 points (FP64 factors): the true
    residual, measured with the oracle's exact-tangent J v of the compact
    operator, meets the tolerance, and the iteration count equals the
    oracle's FGMRES with the same blocks within a few iterations."""
    import torch
    g, f = si.mixing_layer_2d(32, 64)
    tile = (8, 64)
    S, q0 = _make(g, f, tile=tile, precond_prec=64, eps_mode=2, gmres_m=50, gmres_tol=1e-10, gmres_max_restarts=40)
    sigma = 1.0
    b = si.random_complex(5, g.n)
    x = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    st, iters = S.solve(sigma, torch.from_numpy(b).cuda(), x)
    S.close()
    assert st == 0
    P = orc.Problem.from_inputs(g, f)
    PL = orc.Problem.from_inputs(g, f, low_order=1)
    xh = x.cpu().numpy()
    r = b - (orc.core.jv(P, q0, xh, "tangent") - sigma * xh)
    assert np.linalg.norm(r) <= 1.1e-10 * np.linalg.norm(b)
    J = orc.core.dense_jacobian(P, q0)
    JL = orc.core.dense_jacobian(PL, q0)
    M = orc.stability.BlockJacobi(PL, tile, orc.stability.blocks_from_dense(JL, PL, tile, sigma))
    _, sto = orc.krylov.fgmres(lambda z: J @ z - sigma * z, b, M, m=50, tol=1e-10, max_restarts=40)
    assert sto.converged
    assert abs(iters - sto.iterations) <= max(3, sto.iterations // 20), (iters, sto.iterations)


def test_reduced_preconditioner_eigs_match_lapack(orc):
    """Cayley-IRAM with reduced-operator inner preconditioning finds the
    eigenvalues of the compact operator (the preconditioner changes only
    the inner iterations): the two least-stable pairs of the 32 x 64 layer
    against the stored dense LAPACK eigenvalues."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c1_dense_eigs.json")))
    ref = np.array([complex(*l) for l in gold["sets"][1]["lambda"]])
    import torch
    g, f = si.mixing_layer_2d(32, 64)
    S, q0 = _make(g, f, tile=(8, 64), precond_prec=32, eps_mode=2, gmres_m=50, gmres_tol=1e-11,
                  gmres_max_restarts=400)
    v0 = torch.from_numpy(si.start_vector(0x5EED, g.n)).cuda()
    r = S.eigs(1.0, -1.0, nev=4, ncv=30, tol=1e-10, v0=v0)
    S.close()
    assert r.status == 0 and r.nconv == 4
    for l in r.lam:
        assert np.abs(ref - l).min() < 1e-8 * abs(l)
    assert r.resid.max() < 1e-8


def test_reduced_preconditioner_rejections():
    import torch
    from paper_1502_03701_gb300 import JvBatch, StabError
    g, f = si.mixing_layer_2d(16, 32)
    with pytest.raises(StabError, match="UNSUPPORTED"):
        _make(g, f, tile=(4, 8), precond_prec=16)
    S, _ = _make(g, f, tile=(4, 7))  # ty = 7 does not divide 32
    with pytest.raises(StabError, match="INVALID"):
        S.precond_build(0.5)
    S.close()
    S, _ = _make(g, f, tile=(16, 2))  # levels of 4 * 2 * 16 = 128 unknowns: fine
    S.precond_build(0.5)
    S.close()
    S, _ = _make(g, f, tile=(16, 1))  # odd ty
    with pytest.raises(StabError, match="INVALID"):
        S.precond_build(0.5)
    S.close()
    S, _ = _make(g, f, tile=(4, 8))
    S.precond_build(0.5)
    B = JvBatch([S])
    q = torch.from_numpy(si.random_complex(3, g.n)).cuda()
    with pytest.raises(StabError, match="UNSUPPORTED"):
        B.precond_apply([q], [torch.empty_like(q)])
    with pytest.raises(StabError, match="UNSUPPORTED"):
        B.solve([0.5], [q], [torch.zeros_like(q)])
    B.close()
    S.close()


@pytest.mark.parametrize("opts", [dict(gmres_basis_prec=32), dict(gmres_inner_m=10, gmres_inner_tol=1e-3),
                                  dict(lgmres_k=4)], ids=["fp32_basis", "nested_inner", "lgmres"])
def test_reduced_preconditioner_with_other_inner_solvers(orc, opts):
    """The reduced-operator preconditioner under the FP32-basis GMRES (FP32 input to the level sweeps),
    the nested FP32 inner GMRES and LGMRES: each solve meets 1e-10 against the oracle's exact-tangent
    J v."""
    import torch
    g, f = si.mixing_layer_2d(32, 64)
    S, q0 = _make(g, f, tile=(8, 64), precond_prec=32, eps_mode=2, gmres_m=30 if "gmres_inner_m" in opts else 50,
                  gmres_tol=1e-10, gmres_max_restarts=200, **opts)
    b = si.random_complex(6, g.n)
    x = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    st, iters = S.solve(1.0, torch.from_numpy(b).cuda(), x)
    S.close()
    assert st == 0 and iters > 0
    xh = x.cpu().numpy()
    r = b - (orc.core.jv(orc.Problem.from_inputs(g, f), q0, xh, "tangent") - xh)
    assert np.linalg.norm(r) <= 1.1e-10 * np.linalg.norm(b)
