"""GPU parity of the block-Jacobi preconditioner (Sec. Preconditioning)
through the C ABI: assembled tile blocks against the oracle's dense-Jacobian
principal submatrices, the inverse apply against the oracle's LU solves, and
the preconditioned GMRES / eigen solves."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import stab_inputs as si
from gpu_util import max_rel_err, rel_err

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "c1_dense_eigs.json")


def _make(g, f, general=False, **opts):
    from paper_1502_03701_gb300 import Stab
    q0 = si.perturbed_base_flow(g, f, seed=31) if general else si.tanh_base_flow(g, f)
    return Stab(q0, g, f.Ma, f.Re, f.Pr, **opts), q0


BLOCK_CASES = [
    ("2d_visc", si.Grid(2, 16, 16, 1, si.LX_04, -15, 15), si.Flow(0.3, 1000.0), False, (8, 8, 1), (0, 3)),
    ("2d_stretched_general", si.Grid(2, 12, 18, 1, si.LX_04, -15, 15, 1.0, 1.4), si.Flow(0.6, 300.0), True, (4, 6, 1), (0, 4, 8)),
    ("2d_inviscid", si.Grid(2, 16, 12, 1, si.LX_04, -15, 15), si.Flow(0.9, 0.0), False, (8, 4, 1), (1, 5)),
    ("3d_visc", si.Grid(3, 8, 8, 6, si.LX_04, -15, 15, 6.0), si.Flow(0.4, 500.0), False, (4, 4, 2), (0, 7, 11)),
]


@pytest.mark.parametrize("name,g,f,general,tile,tiles", BLOCK_CASES, ids=[c[0] for c in BLOCK_CASES])
def test_assembled_blocks_match_dense_jacobian(orc, name, g, f, general, tile, tiles):
    sigma = 0.2 + 0.1j
    S, q0 = _make(g, f, general, tile=tile)
    P = orc.Problem.from_inputs(g, f)
    for t in tiles:
        got = S.precond_block(sigma, t)
        ref = orc.stability.block_from_columns(P, q0, tile[:g.dim], t, sigma)
        assert max_rel_err(got, ref) < 1e-11, (name, t)
    S.close()


# FP64 inverse to rounding; FP32 / BF16 storage to their unit roundoff times the blocks' conditioning
@pytest.mark.parametrize("prec,tol", [(64, 1e-9), (32, 1e-3), (16, 3e-2)])
def test_apply_matches_oracle_lu(orc, prec, tol):
    import torch
    g, f = si.mixing_layer_2d(16, 32)
    S, q0 = _make(g, f, tile=(8, 8), precond_prec=prec)
    sigma = 0.25
    S.precond_build(sigma)
    P = orc.Problem.from_inputs(g, f)
    J = orc.core.dense_jacobian(P, q0)
    M = orc.stability.BlockJacobi(P, (8, 8), orc.stability.blocks_from_dense(J, P, (8, 8), sigma))
    q = si.random_complex(12, g.n)
    z = torch.empty(g.n, dtype=torch.complex128, device="cuda")
    S.precond_apply(torch.from_numpy(q).cuda(), z)
    assert rel_err(z.cpu().numpy(), M(q)) < tol
    S.close()


BF16_CASES = [
    ("2d_8x8", si.Grid(2, 16, 32, 1, si.LX_04, -15, 15), si.Flow(0.3, 1000.0), (8, 8)),      # 256 rows, one slice
    ("2d_4x4", si.Grid(2, 16, 32, 1, si.LX_04, -15, 15), si.Flow(0.3, 1000.0), (4, 4)),      # 64 rows, row slices
    ("3d_3x3x1", si.Grid(3, 12, 18, 6, si.LX_04, -15, 15, si.LX_04), si.Flow(0.5, 800.0), (3, 3, 1)),  # 45 rows
]


@pytest.mark.parametrize("name,g,f,tile", BF16_CASES, ids=[c[0] for c in BF16_CASES])
def test_bf16_apply_columns_are_the_rounded_fp32_inverse(name, g, f, tile):
    """Applied to unit vectors, the BF16 apply returns columns of the inverse
    exactly (products with 1 and 0 are exact): they must equal the FP32-storage
    apply's columns rounded to bfloat16 (nearest, ties to even), bit for bit.
    Pins the column-major layout, the four-rows-per-thread kernel (row counts
    divisible by four) and the one-row-per-thread kernel (45 rows)."""
    import torch
    S16, _ = _make(g, f, tile=tile, precond_prec=16)
    S32, _ = _make(g, f, tile=tile, precond_prec=32)
    S16.precond_build(0.25)
    S32.precond_build(0.25)
    rng = np.random.default_rng(5)
    for j in rng.choice(g.n, 6, replace=False):
        q = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
        q[int(j)] = 1.0
        z16, z32 = torch.empty_like(q), torch.empty_like(q)
        S16.precond_apply(q, z16)
        S32.precond_apply(q, z32)
        a = z32.cpu().numpy()
        parts = np.stack([a.real, a.imag]).astype(np.float32)
        bits = parts.view(np.uint32).astype(np.uint64)
        rounded = (((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16).astype(np.uint32).view(np.float32)
        b = z16.cpu().numpy()
        assert np.array_equal(np.stack([b.real, b.imag]), rounded.astype(np.float64)), int(j)
        assert np.count_nonzero(a) > 0
    S16.close()
    S32.close()


def test_preconditioned_gmres_and_eigs(orc):
    import torch
    gold = json.load(open(GOLD))
    ref = np.array([complex(*l) for l in gold["sets"][1]["lambda"]])
    g, f = si.mixing_layer_2d(32, 64)
    q0 = si.tanh_base_flow(g, f)
    from paper_1502_03701_gb300 import Stab
    common = dict(eps_mode=2, gmres_m=50, gmres_tol=1e-10, gmres_max_restarts=400)
    S0 = Stab(q0, g, f.Ma, f.Re, f.Pr, **common)
    S1 = Stab(q0, g, f.Ma, f.Re, f.Pr, precond=1, tile=(8, 8), precond_prec=32, **common)
    b = torch.from_numpy(si.random_complex(5, g.n)).cuda()
    x0, x1 = torch.zeros_like(b), torch.zeros_like(b)
    st0, it0 = S0.solve(1.0, b, x0)
    st1, it1 = S1.solve(1.0, b, x1)
    # the same counts as the oracle's FGMRES with the same blocks (570 and 197)
    assert st0 == 0 and st1 == 0 and it1 < it0 / 2
    assert rel_err(x1.cpu().numpy(), x0.cpu().numpy()) < 1e-8
    v0 = torch.from_numpy(si.start_vector(0x5EED, g.n)).cuda()
    S1.close()
    # pole right of the spectrum (inner solves of a few hundred iterations), the two least-stable pairs
    S1 = Stab(q0, g, f.Ma, f.Re, f.Pr, precond=1, tile=(8, 8), precond_prec=32, eps_mode=2, gmres_m=50,
              gmres_tol=1e-11, gmres_max_restarts=400)
    r = S1.eigs(1.0, -1.0, nev=4, ncv=30, tol=1e-10, v0=v0)
    assert r.status == 0 and r.nconv == 4
    for l in r.lam:
        assert np.abs(ref - l).min() < 1e-8 * abs(l)
    assert abs(r.lam[0].real - 0.169) < 1e-3 and abs(r.lam[2].real - 0.0955) < 1e-3
    assert r.resid.max() < 1e-8
    assert r.stats["precond_builds"] == 1
    S0.close()
    S1.close()


def test_bf16_inverses_keep_fgmres_accuracy():
    """BF16-stored block inverses inside FP64 flexible GMRES: the solve still
    reaches the FP64 tolerance (the preconditioner only changes the iteration
    count, which stays within 1.3x of FP32 storage)."""
    import torch
    from paper_1502_03701_gb300 import Stab
    g, f = si.mixing_layer_2d(32, 64)
    q0 = si.tanh_base_flow(g, f)
    b = torch.from_numpy(si.random_complex(5, g.n)).cuda()
    out = {}
    for prec in (32, 16):
        S = Stab(q0, g, f.Ma, f.Re, f.Pr, precond=1, tile=(8, 8), precond_prec=prec, eps_mode=2, gmres_m=50,
                 gmres_tol=1e-10, gmres_max_restarts=400)
        x = torch.zeros_like(b)
        st, it = S.solve(1.0, b, x)
        assert st == 0
        out[prec] = (it, x.cpu().numpy())
        S.close()
    assert out[16][0] <= 1.3 * out[32][0]
    assert rel_err(out[16][1], out[32][1]) < 1e-8


def test_full_size_blocks_invert_consistently():
    """256 x 512 layer with 8 x 8 tiles (2,048 blocks of 256 x 256): for
    sampled tiles, the assembled block times the FP64 preconditioner output
    returns the input on that tile."""
    import torch
    g, f = si.mixing_layer_2d(256, 512)
    S, q0 = _make(g, f, tile=(8, 8), precond_prec=64)
    sigma = 0.25
    S.precond_build(sigma)
    q = si.random_complex(3, g.n)
    z = torch.empty(g.n, dtype=torch.complex128, device="cuda")
    S.precond_apply(torch.from_numpy(q).cuda(), z)
    zh = z.cpu().numpy()
    import oracle
    P = oracle.Problem.from_inputs(g, f)
    idx = oracle.stability.tile_dofs(P, (8, 8))
    for t in (0, 777, 2047):
        B = S.precond_block(sigma, t)
        assert rel_err(B @ zh[idx[t]], q[idx[t]]) < 1e-9
    S.close()


def test_precond_rejects_bad_tile():
    from paper_1502_03701_gb300 import StabError
    g, f = si.mixing_layer_2d(16, 24)
    S, q0 = _make(g, f, tile=(5, 8))
    with pytest.raises(StabError, match="tile"):
        S.precond_build(0.25)
    S.close()


TC_CASES = [
    ("2d_8x8_b256", si.Grid(2, 16, 32, 1, si.LX_04, -15, 15), si.Flow(0.3, 1000.0), (8, 8)),
    ("2d_16x16_b1024", si.Grid(2, 32, 32, 1, si.LX_04, -15, 15), si.Flow(0.4, 800.0), (16, 16)),
    ("3d_3x3x1_b45", si.Grid(3, 12, 18, 6, si.LX_04, -15, 15, si.LX_04), si.Flow(0.5, 800.0), (3, 3, 1)),
]


@pytest.mark.parametrize("factor,tol", [(1, 1e-3), (2, 3e-2)])
@pytest.mark.parametrize("name,g,f,tile", TC_CASES, ids=[c[0] for c in TC_CASES])
def test_tensor_core_factorisation_matches_oracle_lu(orc, name, g, f, tile, factor, tol):
    """Blocked Gauss-Jordan with the panels' trailing updates as batched
    tensor-core GEMMs (precond_factor 1: FP32 accuracy by BF16x9 emulation;
    2: TF32): the apply matches the oracle's LU solve of the dense-Jacobian
    tiles to the storage precision times the blocks' conditioning, for block
    sizes 256, 1,024 (64-column panels) and 45 (a ragged last panel), and
    equals the CUDA-core Gauss-Jordan's result to the same precision."""
    import torch
    S, q0 = _make(g, f, tile=tile, precond_prec=32, precond_factor=factor)
    R, _ = _make(g, f, tile=tile, precond_prec=32)
    sigma = 0.3 + 0.1j
    S.precond_build(sigma)
    R.precond_build(sigma)
    P = orc.Problem.from_inputs(g, f)
    J = orc.core.dense_jacobian(P, q0)
    M = orc.stability.BlockJacobi(P, tile[:g.dim], orc.stability.blocks_from_dense(J, P, tile[:g.dim], sigma))
    q = si.random_complex(13, g.n)
    z = torch.empty(g.n, dtype=torch.complex128, device="cuda")
    zr = torch.empty_like(z)
    S.precond_apply(torch.from_numpy(q).cuda(), z)
    R.precond_apply(torch.from_numpy(q).cuda(), zr)
    assert rel_err(z.cpu().numpy(), M(q)) < tol
    assert rel_err(z.cpu().numpy(), zr.cpu().numpy()) < tol
    S.close()
    R.close()


def test_tensor_core_factorisation_keeps_fgmres_iterations():
    """The FP32-accurate tensor-core factorisation leaves the preconditioned
    FGMRES iteration count and solution of the CUDA-core factorisation
    unchanged (within two iterations, 1e-8)."""
    import torch
    from paper_1502_03701_gb300 import Stab
    g, f = si.mixing_layer_2d(32, 64)
    q0 = si.tanh_base_flow(g, f)
    b = torch.from_numpy(si.random_complex(5, g.n)).cuda()
    out = {}
    for fac in (0, 1):
        S = Stab(q0, g, f.Ma, f.Re, f.Pr, precond=1, tile=(16, 16), precond_prec=32, precond_factor=fac,
                 eps_mode=2, gmres_m=50, gmres_tol=1e-10, gmres_max_restarts=400)
        x = torch.zeros_like(b)
        st, it = S.solve(1.0, b, x)
        assert st == 0
        out[fac] = (it, x.cpu().numpy())
        S.close()
    assert abs(out[1][0] - out[0][0]) <= 2
    assert rel_err(out[1][1], out[0][1]) < 1e-8
