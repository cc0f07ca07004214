"""Many problems on one GPU: stab_eigs_batch and the continuous-batching
server give every solve the same eigenvalues as the solve alone (identical
kernels and reduction orders, so equal to rounding; checked at 1e-12
relative, far inside the 1e-8 eigenvalue tolerance), admit requests by their
memory estimate, and overlap requests on the device."""
import numpy as np
import pytest

import stab_inputs as si

pytestmark = pytest.mark.gpu
OPTS = dict(eps_mode=2, precond=1, tile=(8, 8), precond_prec=32, gmres_m=30, gmres_tol=1e-10, max_restarts=60)
EIG = (1.0, -1.0, 2, 12, 1e-10)  # sigma, tau, nev, ncv, tol
PROBLEMS = [(16, 32, 0.3, 1000.0), (16, 48, 0.6, 500.0), (24, 32, 0.45, 2000.0), (16, 32, 0.8, 800.0)]


def _problem(nx, ny, Ma, Re):
    g, f = si.mixing_layer_2d(nx, ny, Ma=Ma)
    f = si.Flow(Ma, Re)
    return g, f, si.tanh_base_flow(g, f)


def _alone():
    from paper_1502_03701_gb300 import Stab
    out = []
    for p in PROBLEMS:
        g, f, q0 = _problem(*p)
        S = Stab(q0, g, f.Ma, f.Re, f.Pr, **OPTS)
        r = S.eigs(*EIG)
        S.close()
        assert r.nconv == EIG[2], p
        assert np.all(r.resid < 1e-8), p
        out.append((r.lam, r.resid))
    return out


@pytest.fixture(scope="module")
def alone():
    return _alone()


def _close(a, b):
    return np.max(np.abs(a - b) / np.abs(b)) <= 1e-12


def _same(lam, res, ref):
    """eigenvalues to 1e-12 relative; residuals to 1e-3 relative (they are ~1e-10 themselves)"""
    return _close(lam, ref[0]) and np.all(np.abs(res - ref[1]) <= 1e-3 * ref[1] + 1e-14)


def test_batch_equals_alone(alone):
    from paper_1502_03701_gb300 import Stab, eigs_batch
    hs = []
    for p in PROBLEMS:
        g, f, q0 = _problem(*p)
        hs.append(Stab(q0, g, f.Ma, f.Re, f.Pr, **OPTS))
    res = eigs_batch(hs, [EIG] * len(hs), concurrency=len(hs))
    for r, ref, p in zip(res, alone, PROBLEMS):
        assert r.status == 0 and r.nconv == EIG[2], p
        assert _same(r.lam, r.resid, ref), (p, r.lam, ref)
    # the handles are usable on their own streams afterwards
    r2 = hs[0].eigs(*EIG)
    assert _same(r2.lam, r2.resid, alone[0])
    for h in hs:
        h.close()


def test_server_same_alone_and_in_mix(alone):
    from paper_1502_03701_gb300 import Server
    srv = Server(slots=4, mem_budget_bytes=8 << 30)
    ids = []
    for i, p in enumerate(PROBLEMS):
        g, f, q0 = _problem(*p)
        ids.append(srv.submit(q0, g, f.Ma, f.Re, f.Pr, *EIG, vectors=(i == 0), **OPTS))
    for rid, ref, p in zip(ids, alone, PROBLEMS):
        assert srv.wait(rid, 600.0)
        got, res, info = srv.result(rid)
        assert info["status"] == 0 and info["nconv"] == EIG[2], p
        assert _same(got, res, ref), (p, got, ref)
        assert info["latency_s"] >= info["run_s"] > 0 and info["est_bytes"] > 0
        if "vecs" in info:  # unit eigenvectors with the reported residual ||J x - lambda x||
            from paper_1502_03701_gb300 import Stab
            import torch
            g, f, q0 = _problem(*p)
            S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2)
            for q in range(EIG[2]):
                x = torch.from_numpy(info["vecs"][q].copy()).cuda()
                jx = torch.empty_like(x)
                S.apply_J(x, jx, got[q])
                assert abs(float(torch.linalg.vector_norm(x)) - 1.0) < 1e-12
                assert float(torch.linalg.vector_norm(jx)) == pytest.approx(res[q], rel=1e-3, abs=1e-13)
            S.close()
    st = srv.stats()
    assert st["peak_running"] >= 2          # requests overlapped on the device
    assert st["running"] == 0 and st["queued"] == 0
    srv.close()


def test_server_admits_by_memory(alone):
    from paper_1502_03701_gb300 import Server, StabError, estimate_bytes
    sizes = []
    for p in PROBLEMS[:3]:
        g, f, q0 = _problem(*p)
        sizes.append(estimate_bytes(g, EIG[2], EIG[3], True, **OPTS))
    budget = int(max(sizes) * 1.5)          # room for one request at a time
    srv = Server(slots=4, mem_budget_bytes=budget)
    ids = []
    for p in PROBLEMS[:3]:
        g, f, q0 = _problem(*p)
        ids.append(srv.submit(q0, g, f.Ma, f.Re, f.Pr, *EIG, **OPTS))
    for rid, ref in zip(ids, alone):
        assert srv.wait(rid, 600.0)
        got, res, info = srv.result(rid)
        assert _same(got, res, ref)
    st = srv.stats()
    assert st["peak_bytes"] <= budget and st["peak_running"] == 1
    g, f, q0 = _problem(64, 128, 0.3, 1000.0)
    with pytest.raises(StabError):           # larger than the whole budget
        srv.submit(q0, g, f.Ma, f.Re, f.Pr, *EIG, **OPTS)
    with pytest.raises(StabError):
        srv.wait(12345, 0.0)
    srv.close()


def test_server_lockstep_cohort_same_as_alone(alone):
    """With lockstep cohorts, one worker takes all four queued requests and
    solves them together (stab_jv_batch_eigs: every phase one launch for the
    cohort); each result equals the request's lone solve to 1e-12."""
    from paper_1502_03701_gb300 import Server
    srv = Server(slots=1, mem_budget_bytes=8 << 30, cohort=4)
    ids = []
    for i, p in enumerate(PROBLEMS):
        g, f, q0 = _problem(*p)
        ids.append(srv.submit(q0, g, f.Ma, f.Re, f.Pr, *EIG, vectors=(i == 1), **OPTS))
    for rid, ref, p in zip(ids, alone, PROBLEMS):
        assert srv.wait(rid, 600.0)
        got, res, info = srv.result(rid)
        assert info["status"] == 0 and info["nconv"] == EIG[2], p
        assert _same(got, res, ref), (p, got, ref)
        if "vecs" in info:
            assert np.allclose(np.linalg.norm(info["vecs"], axis=1), 1.0, atol=1e-12)
    st = srv.stats()
    assert st["peak_running"] >= 2  # the cohort's requests ran together on the one worker
    srv.close()
