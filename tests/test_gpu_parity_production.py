"""GPU parity on the paths the production configurations run, checked
directly against the oracle: GMRES above 16,384 unknowns (Gram-Schmidt with
selective reorthogonalisation decided on the device), eigenspaces of the
double Kelvin-Helmholtz eigenvalue (principal angles), the batched J v,
block-Jacobi apply and CGS2 over uneven instances, and a served request."""
import numpy as np
import pytest
import scipy.linalg as sla

import stab_inputs as si
from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def _stab(g, f, **opts):
    from paper_1502_03701_gb300 import Stab
    q0 = si.tanh_base_flow(g, f)
    return Stab(q0, g, f.Ma, f.Re, f.Pr, **opts), q0


@pytest.mark.parametrize("nx,ny,sigma,precond", [(64, 64, 1.0, 0), (48, 96, 2.0 + 0.5j, 1)])
def test_gmres_above_16k_unknowns_against_oracle(orc, nx, ny, sigma, precond):
    """Sec. Iterative solvers at n >= 16,384, where the FP64 GMRES basis is
    orthogonalised by classical Gram-Schmidt with selective
    reorthogonalisation: the solution's true residual, measured with the
    oracle's exact-tangent J v, meets the tolerance; without preconditioner
    the solution equals the oracle's own matrix-free GMRES solution."""
    import torch
    g, f = si.mixing_layer_2d(nx, ny)
    assert g.n >= 16384
    opts = dict(eps_mode=2, gmres_m=50, gmres_tol=1e-10, gmres_max_restarts=200, precond=precond)
    if precond:
        opts.update(tile=(16, 16), precond_prec=32)
    S, q0 = _stab(g, f, **opts)
    P = orc.Problem.from_inputs(g, f)
    b = si.random_complex(91, g.n)
    x = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    st, iters = S.solve(sigma, torch.from_numpy(b).cuda(), x)
    S.close()
    assert st == 0 and iters > 0
    xh = x.cpu().numpy()
    r = b - (orc.core.jv(P, q0, xh, "tangent") - sigma * xh)
    assert np.linalg.norm(r) <= 1.1e-10 * np.linalg.norm(b)
    if not precond:
        xo, sto = orc.krylov.fgmres(lambda z: orc.core.jv(P, q0, z, "tangent") - sigma * z, b, None, m=50,
                                    tol=1e-10, max_restarts=200)
        assert sto.converged
        assert rel_err(xh, xo) < 1e-7
        assert abs(iters - sto.iterations) <= max(5, sto.iterations // 10)


def test_double_eigenvalue_eigenspace_principal_angles(orc):
    """The tanh layer's Kelvin-Helmholtz eigenvalue is double (the +-alpha
    pair), so eigenvectors are not unique: the GPU's two eigenvectors span the
    same space as dense LAPACK's, principal angles below 1e-6."""
    import torch
    g, f = si.mixing_layer_2d(8, 16)
    S, q0 = _stab(g, f, eps_mode=2, gmres_m=30, gmres_tol=1e-12, gmres_max_restarts=400)
    vecs = torch.zeros((2, g.n), dtype=torch.complex128, device="cuda")
    r = S.eigs(0.25, -1.0, nev=2, ncv=12, tol=1e-12, vecs=vecs)
    S.close()
    assert r.status == 0 and r.nconv == 2
    J = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f), q0)
    lam, X = sla.eig(J)
    pick = np.argsort(np.abs(lam - r.lam[0]))[:2]
    assert np.abs(lam[pick] - r.lam[0]).max() < 1e-8 * abs(r.lam[0])
    Vg = vecs.cpu().numpy().T
    ang = sla.subspace_angles(Vg, X[:, pick])
    assert ang.max() < 1e-6
    assert np.allclose(np.linalg.norm(Vg, axis=0), 1.0, atol=1e-12)


def _batch_instances():
    specs = [
        (si.mixing_layer_2d(16, 32), dict(tile=(8, 8))),
        ((si.Grid(2, 24, 20, 1, si.LX_04, -15, 15, 1.0, 1.5), si.Flow(0.6, 500.0)), dict(tile=(4, 4))),
        ((si.Grid(2, 16, 24, 1, si.LX_04, -15, 15), si.Flow(0.8, 0.0)), dict(tile=(8, 8))),
        ((si.Grid(3, 8, 12, 6, si.LX_04, -15, 15, si.LX_04), si.Flow(0.5, 800.0)), dict(tile=(4, 4, 2))),
    ]
    return specs


def test_batched_jv_apply_and_cgs2_against_oracle(orc):
    """stab_jv_batch_* over uneven instances compared with the oracle, not
    with the single-handle path: each batched J v - shift v with the exact
    epsilon-quotient in binary128 (1e-10), each batched block-Jacobi apply
    (FP64 inverses) with the oracle's LU of the dense-Jacobian tiles (1e-9),
    each batched CGS2 with the oracle's CGS2 (1e-12 ||w||)."""
    import torch
    from paper_1502_03701_gb300 import JvBatch, Stab
    hs, probs = [], []
    for (g, f), opts in _batch_instances():
        q0 = si.tanh_base_flow(g, f)
        hs.append(Stab(q0, g, f.Ma, f.Re, f.Pr, precond=1, precond_prec=64, **opts))
        probs.append((g, f, q0, opts["tile"]))
    shifts = [0.0, -1 + 0.2j, 0.5j, 2.0]
    vs = [si.random_complex(300 + i, S.n) for i, S in enumerate(hs)]
    B = JvBatch(hs)
    dv = [torch.from_numpy(v).cuda() for v in vs]
    outs = [torch.empty_like(v) for v in dv]
    B.apply(dv, outs, shifts)
    torch.cuda.synchronize()
    for S, (g, f, q0, tile), v, o, z in zip(hs, probs, vs, outs, shifts):
        P = orc.Problem.from_inputs(g, f)
        ref = orc.core.jv(P, q0, v, "quad", S.last_eps()) - z * v
        assert rel_err(o.cpu().numpy(), ref) < 1e-10, (g, f)
    sig = [0.25, 0.3 + 0.1j, 0.5, 0.2]
    for S, s in zip(hs, sig):
        S.precond_build(s)
    zs = [torch.empty_like(v) for v in dv]
    B.precond_apply(dv, zs)
    torch.cuda.synchronize()
    for (g, f, q0, tile), v, z, s in zip(probs, vs, zs, sig):
        P = orc.Problem.from_inputs(g, f)
        J = orc.core.dense_jacobian(P, q0)
        M = orc.stability.BlockJacobi(P, tile, orc.stability.blocks_from_dense(J, P, tile, s))
        assert rel_err(z.cpu().numpy(), M(v)) < 1e-9, (g, f)
    ks = [3, 7, 1, 12]
    Vs, Vh = [], []
    for i, (S, k) in enumerate(zip(hs, ks)):
        rng = np.random.default_rng(70 + i)
        Q, _ = np.linalg.qr(rng.standard_normal((S.n, k)) + 1j * rng.standard_normal((S.n, k)))
        Vh.append(Q)
        Vs.append(torch.from_numpy(np.ascontiguousarray(Q.T)).cuda())
    ws = [torch.from_numpy(v.copy()).cuda() for v in vs]
    hc, nr = B.orthogonalize(Vs, ks, ws)
    for Q, v, w, h, nrm in zip(Vh, vs, ws, hc, nr):
        href, wref = orc.krylov.cgs2(Q, v)
        wn = np.linalg.norm(v)
        assert np.abs(h - href).max() < 1e-12 * wn
        assert np.abs(w.cpu().numpy() - wref).max() < 1e-12 * wn
        assert abs(nrm - np.linalg.norm(wref)) < 1e-12 * wn
    B.close()
    for S in hs:
        S.close()


def test_served_request_against_dense_lapack(orc):
    """One request through the continuous-batching server, in a mix with two
    others: its eigenvalues equal the oracle's dense LAPACK eigenvalues of J
    with the largest Cayley |theta| to 1e-8, true residuals below 1e-8."""
    from paper_1502_03701_gb300 import Server
    g, f = si.mixing_layer_2d(8, 16)
    q0 = si.tanh_base_flow(g, f)
    J = orc.core.dense_jacobian(orc.Problem.from_inputs(g, f), q0)
    ref, _ = orc.stability.dense_reference(J, 0.25, -1.0, 2)
    opts = dict(eps_mode=2, gmres_m=30, gmres_tol=1e-12, gmres_max_restarts=400)
    srv = Server(slots=3, mem_budget_bytes=4 << 30)
    others = []
    for nx, ny, Ma in ((16, 32, 0.5), (16, 24, 0.7)):
        g2, f2 = si.mixing_layer_2d(nx, ny, Ma=Ma)
        others.append(srv.submit(si.tanh_base_flow(g2, f2), g2, f2.Ma, f2.Re, f2.Pr, 1.0, -1.0, 2, 12, 1e-10,
                                 eps_mode=2, precond=1, tile=(8, 8)))
    rid = srv.submit(q0, g, f.Ma, f.Re, f.Pr, 0.25, -1.0, 2, 12, 1e-12, **opts)
    assert srv.wait(rid, 120.0)
    lam, res, info = srv.result(rid)
    for o in others:
        srv.wait(o, 120.0)
    srv.close()
    assert info["nconv"] == 2
    for l in ref:
        assert np.abs(lam - l).min() < 1e-8 * abs(l)
    assert res.max() < 1e-8
