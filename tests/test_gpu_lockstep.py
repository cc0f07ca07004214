"""Solver-level batching (stab_jv_batch_solve, stab_jv_batch_eigs): GMRES and
Cayley-IRAM of uneven instances in lockstep, every phase one launch for all
instances, converged instances dropping out through device-side gates.
Checked against each instance's lone solve, the oracle's exact-tangent
residual and dense LAPACK eigenvalues."""
import numpy as np
import pytest

import stab_inputs as si
from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def _handles(specs):
    from paper_1502_03701_gb300 import Stab
    out = []
    for (g, f), opts in specs:
        q0 = si.tanh_base_flow(g, f)
        out.append((Stab(q0, g, f.Ma, f.Re, f.Pr, **opts), g, f, q0))
    return out


SOLVE_SPECS = [
    (si.mixing_layer_2d(16, 32), dict(eps_mode=2, gmres_m=30, gmres_tol=1e-10, precond=1, tile=(8, 8))),
    (si.mixing_layer_2d(8, 16, Ma=0.6), dict(eps_mode=2, gmres_m=20, gmres_tol=1e-12)),
    ((si.Grid(2, 24, 20, 1, si.LX_04, -15, 15, 1.0, 1.5), si.Flow(0.5, 500.0)),
     dict(eps_mode=0, gmres_m=25, gmres_tol=1e-10, precond=1, tile=(4, 4), precond_prec=64)),
    ((si.Grid(3, 8, 12, 6, si.LX_04, -15, 15, si.LX_04), si.Flow(0.4, 800.0)),
     dict(eps_mode=2, gmres_m=30, gmres_tol=1e-10, precond=1, tile=(4, 4, 2))),
]


def test_lockstep_solve_equals_lone_solves_bit_for_bit(orc):
    """Below 16,384 unknowns the lockstep GMRES runs the lone cycle's
    kernels with the same arithmetic: every solution equals the instance's
    own stab_solve bit for bit, with the same iteration count, and its
    residual meets the tolerance against the oracle's exact tangent."""
    import torch
    from paper_1502_03701_gb300 import JvBatch
    inst = _handles(SOLVE_SPECS)
    sig = [0.25, 0.3 + 0.2j, 1.0, 0.5]
    bs = [torch.from_numpy(si.random_complex(200 + i, S.n)).cuda() for i, (S, *_) in enumerate(inst)]
    lone = []
    for (S, g, f, q0), s, b in zip(inst, sig, bs):
        x = torch.zeros_like(b)
        st, it = S.solve(s, b, x)
        assert st == 0
        lone.append((x, it))
    B = JvBatch([S for S, *_ in inst])
    xs = [torch.full_like(b, float("nan")) for b in bs]
    st, its = B.solve(sig, bs, xs)
    assert st == 0
    for i, ((x1, it1), x2, it2) in enumerate(zip(lone, xs, its)):
        assert it1 == it2, (i, it1, it2)
        assert torch.equal(x1, x2), (i, float((x1 - x2).abs().max()))
    S, g, f, q0 = inst[1]
    xh = xs[1].cpu().numpy()
    bh = bs[1].cpu().numpy()
    P = orc.Problem.from_inputs(g, f)
    r = bh - (orc.core.jv(P, q0, xh, "tangent") - sig[1] * xh)
    assert np.linalg.norm(r) <= 1.05e-12 * np.linalg.norm(bh)
    B.close()
    for S, *_ in inst:
        S.close()


def test_lockstep_solve_above_16k_against_oracle(orc):
    """An instance of 16,384 unknowns next to a small one: the lockstep solve
    (CGS2 at every size) meets the tolerance against the oracle's tangent J v
    and agrees with the lone solve (selective reorthogonalisation) to the
    tolerance times the conditioning."""
    import torch
    from paper_1502_03701_gb300 import JvBatch
    specs = [(si.mixing_layer_2d(64, 64), dict(eps_mode=2, gmres_m=40, gmres_tol=1e-10, precond=1, tile=(8, 8))),
             (si.mixing_layer_2d(16, 32, Ma=0.7), dict(eps_mode=2, gmres_m=30, gmres_tol=1e-10))]
    inst = _handles(specs)
    sig = [0.5 + 0.2j, 1.0]
    bs = [torch.from_numpy(si.random_complex(300 + i, S.n)).cuda() for i, (S, *_) in enumerate(inst)]
    B = JvBatch([S for S, *_ in inst])
    xs = [torch.zeros_like(b) for b in bs]
    st, its = B.solve(sig, bs, xs)
    assert st == 0 and all(i > 0 for i in its)
    for (S, g, f, q0), s, b, x in zip(inst, sig, bs, xs):
        P = orc.Problem.from_inputs(g, f)
        xh, bh = x.cpu().numpy(), b.cpu().numpy()
        r = bh - (orc.core.jv(P, q0, xh, "tangent") - s * xh)
        assert np.linalg.norm(r) <= 1.1e-10 * np.linalg.norm(bh)
        x1 = torch.zeros_like(b)
        S.solve(s, b, x1)
        assert rel_err(xh, x1.cpu().numpy()) < 1e-7
    B.close()
    for S, *_ in inst:
        S.close()


def test_lockstep_eigs_match_lone_solves_and_lapack(orc):
    """Cayley-IRAM of uneven instances with different nev, ncv, poles and
    preconditioners in lockstep: each instance's eigenvalues and residuals
    equal its lone stab_eigs (to 1e-12; the same kernels in the same order),
    the tiny layers' eigenvalues match dense LAPACK to 1e-8, and the J v
    counts equal the lone solves'."""
    import torch
    from paper_1502_03701_gb300 import JvBatch
    specs = [
        (si.mixing_layer_2d(8, 16), dict(eps_mode=2, gmres_m=30, gmres_tol=1e-12, gmres_max_restarts=400)),
        (si.mixing_layer_2d(16, 32, Ma=0.6), dict(eps_mode=2, gmres_m=30, gmres_tol=1e-10, precond=1, tile=(8, 8),
                                                   max_restarts=60)),
        ((si.Grid(2, 8, 12, 1, si.LX_04, -12, 12), si.Flow(0.5, 800.0)),
         dict(eps_mode=2, gmres_m=20, gmres_tol=1e-12, gmres_max_restarts=400)),
    ]
    jobs = [(0.25, -1.0, 2, 12, 1e-11), (1.0, -1.0, 2, 12, 1e-10), (0.3, -1.0, 3, 16, 1e-11)]
    inst = _handles(specs)
    lone = []
    for (S, *_), a in zip(inst, jobs):
        r = S.eigs(*a)
        assert r.status == 0 and r.nconv == a[2]
        lone.append(r)
    B = JvBatch([S for S, *_ in inst])
    vecs = [torch.zeros((a[2], S.n), dtype=torch.complex128, device="cuda") for (S, *_), a in zip(inst, jobs)]
    res = B.eigs(jobs, vecs=vecs)
    for i, (r, l, a) in enumerate(zip(res, lone, jobs)):
        assert r.status == 0 and r.nconv == a[2], (i, r.status, r.nconv)
        assert np.max(np.abs(r.lam - l.lam) / np.abs(l.lam)) <= 1e-12, (i, r.lam, l.lam)
        assert r.resid.max() < 1e-8
        assert r.stats["jv_calls"] == l.stats["jv_calls"], (i, r.stats, l.stats)
        assert np.allclose(np.linalg.norm(vecs[i].cpu().numpy(), axis=1), 1.0, atol=1e-12)
    for idx in (0, 2):
        S, g, f, q0 = inst[idx]
        J = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f), q0)
        ref, _ = orc.stability.dense_reference(J, jobs[idx][0], jobs[idx][1], jobs[idx][2])
        for l in ref:
            assert np.abs(res[idx].lam - l).min() < 1e-8 * abs(l)
    B.close()
    for S, *_ in inst:
        S.close()


def test_lockstep_rejects_fp32_basis_and_lgmres():
    from paper_1502_03701_gb300 import JvBatch, StabError
    inst = _handles([(si.mixing_layer_2d(8, 16), dict(gmres_basis_prec=32)),
                     (si.mixing_layer_2d(8, 16), dict(gmres_m=10, lgmres_k=2))])
    for S, *_ in inst:
        B = JvBatch([S])
        with pytest.raises(StabError, match="UNSUPPORTED"):
            B.eigs([(0.25, -1.0, 2, 12, 1e-10)])
        B.close()
        S.close()
