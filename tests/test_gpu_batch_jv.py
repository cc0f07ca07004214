"""Batched J v and block-Jacobi apply (stab_jv_batch_*): one launch per phase
for several problems of uneven size.  Each instance's result must equal its handle's own stab_apply_J
bit for bit (same kernels, same per-instance launch shapes and summation
order); the single-handle path is the one the parity tests check against the
oracle."""
import numpy as np
import pytest

import stab_inputs as si

pytestmark = pytest.mark.gpu


def _instances():
    from paper_1502_03701_gb300 import Stab
    specs = [
        (si.mixing_layer_2d(32, 64), {}),
        (si.mixing_layer_2d(64, 128, Ma=0.6), dict(eps_mode=2)),
        ((si.Grid(2, 48, 40, 1, si.LX_04, -15, 15), si.Flow(0.3, 500.0)), dict(stencil_prec=48)),
        ((si.Grid(2, 70, 67, 1, si.LX_04, -15, 15, 1.0, 1.7), si.Flow(0.6, 500.0)), {}),   # stretched, ragged
        ((si.Grid(2, 24, 40, 1, si.LX_04, -15, 15), si.Flow(0.9, 0.0)), {}),                 # inviscid
        ((si.Grid(3, 12, 16, 8, si.LX_04, -15, 15, si.LX_04), si.Flow(0.5, 800.0)), {}),     # 3-D
        ((si.Grid(3, 16, 20, 6, si.LX_04, -15, 15, si.LX_04), si.Flow(0.4, 300.0)), dict(eps_mode=2, stencil_prec=48)),
    ]
    out = []
    for (g, f), opts in specs:
        S = Stab(si.tanh_base_flow(g, f), g, f.Ma, f.Re, f.Pr, **opts)
        out.append((S, g))
    # launch shapes: one instance in the compact mode, one side by side, one tuned
    out[0][0].set_line_config(1, 16, 4, 3)
    out[0][0].set_line_config(0, 16, 2, 2)
    out[3][0].autotune()
    out[5][0].set_line_config(2, 16, 2, 3)
    out[2][0].set_line_config(1, 16, 2, 3)  # compact mode with pair right-hand sides
    return out


def test_batch_equals_each_handle_bit_for_bit():
    import torch
    from paper_1502_03701_gb300 import JvBatch
    inst = _instances()
    vs = [torch.from_numpy(si.random_complex(500 + i, S.n)).cuda() for i, (S, g) in enumerate(inst)]
    shifts = [0.0, -1 + 0.2j, 0.5j, 0.0, 2.0, -0.25, 1 - 1j]
    ref, eps_ref = [], []
    for (S, g), v, z in zip(inst, vs, shifts):
        o = torch.empty_like(v)
        S.apply_J(v, o, z)
        ref.append(o)
        eps_ref.append(S.last_eps())
    B = JvBatch([S for S, g in inst])
    for rep in range(3):  # repeated calls reuse the staging and parameter buffers
        outs = [torch.full_like(v, float("nan")) for v in vs]
        B.apply(vs, outs, shifts)
        torch.cuda.synchronize()
        for i, (o, r) in enumerate(zip(outs, ref)):
            assert torch.equal(o, r), (rep, i, float((o - r).abs().max() / r.abs().max()))
        assert [S.last_eps() for S, g in inst] == eps_ref
    # without shifts: J v itself
    outs = [torch.empty_like(v) for v in vs]
    B.apply(vs, outs)
    for (S, g), v, o in zip(inst, vs, outs):
        r = torch.empty_like(v)
        S.apply_J(v, r)
        assert torch.equal(o, r)
    B.close()
    for S, g in inst:
        S.close()


def test_batch_rejects_bad_handles_and_vectors():
    import torch
    from paper_1502_03701_gb300 import JvBatch, Stab, StabError
    g, f = si.mixing_layer_2d(16, 32)
    S = Stab(si.tanh_base_flow(g, f), g, f.Ma, f.Re, f.Pr)
    G = Stab(si.perturbed_base_flow(g, f, seed=3), g, f.Ma, f.Re, f.Pr)   # base varies in x: not batched
    with pytest.raises(StabError, match="INVALID_ARG"):
        JvBatch([S, S])
    with pytest.raises(StabError, match="UNSUPPORTED"):
        JvBatch([S, G])
    B = JvBatch([S])
    v = torch.zeros(S.n, dtype=torch.complex128, device="cuda")
    with pytest.raises(StabError, match="overlapping"):
        B.apply([v], [v])
    with pytest.raises(ValueError):
        B.apply([v, v], [v])
    B.close()
    S.close()
    G.close()


def test_batch_precond_apply_equals_each_handle_bit_for_bit():
    """Batched block-Jacobi apply over handles with every inverse storage layout:
    FP64 and FP32 rows, BF16 four rows per thread (256 and 64 rows, one and
    several row slices), BF16 one row per thread (45 rows)."""
    import torch
    from paper_1502_03701_gb300 import JvBatch, Stab, StabError
    specs = [
        (si.mixing_layer_2d(16, 32), dict(tile=(8, 8), precond_prec=64)),
        (si.mixing_layer_2d(32, 64), dict(tile=(8, 8), precond_prec=32)),
        (si.mixing_layer_2d(16, 32, Ma=0.6), dict(tile=(4, 4), precond_prec=16)),
        ((si.Grid(3, 12, 18, 6, si.LX_04, -15, 15, si.LX_04), si.Flow(0.5, 800.0)), dict(tile=(3, 3, 1), precond_prec=16)),
        ((si.Grid(2, 24, 40, 1, si.LX_04, -15, 15), si.Flow(0.4, 600.0)), dict(tile=(8, 8), precond_prec=16)),
    ]
    hs = []
    for i, ((g, f), opts) in enumerate(specs):
        S = Stab(si.tanh_base_flow(g, f), g, f.Ma, f.Re, f.Pr, eps_mode=2, precond=1, **opts)
        hs.append(S)
    B = JvBatch(hs)
    qs = [torch.from_numpy(si.random_complex(700 + i, S.n)).cuda() for i, S in enumerate(hs)]
    with pytest.raises(StabError, match="no preconditioner"):
        B.precond_apply(qs, [torch.empty_like(q) for q in qs])
    for i, S in enumerate(hs):
        S.precond_build(0.25 + 0.1 * i)
    ref = []
    for S, q in zip(hs, qs):
        z = torch.empty_like(q)
        S.precond_apply(q, z)
        ref.append(z)
    for rep in range(2):
        zs = [torch.full_like(q, float("nan")) for q in qs]
        B.precond_apply(qs, zs)
        torch.cuda.synchronize()
        for i, (z, r) in enumerate(zip(zs, ref)):
            assert torch.equal(z, r), (rep, i)
    # J v and the apply interleaved on the same batch (parameter buffer reused)
    outs = [torch.empty_like(q) for q in qs]
    B.apply(qs, outs)
    zs = [torch.empty_like(q) for q in qs]
    B.precond_apply(outs, zs)
    for S, q, z in zip(hs, qs, zs):
        a, b = torch.empty_like(q), torch.empty_like(q)
        S.apply_J(q, a)
        S.precond_apply(a, b)
        assert torch.equal(z, b)
    B.close()
    for S in hs:
        S.close()


def test_batch_orthogonalize_equals_each_handle_bit_for_bit():
    """Batched CGS2 over uneven problems and column counts (one column: fewer
    columns than warps; 40: more) against each handle's stab_orthogonalize."""
    import torch
    from paper_1502_03701_gb300 import JvBatch, Stab, StabError
    specs = [si.mixing_layer_2d(32, 64), (si.Grid(2, 48, 40, 1, si.LX_04, -15, 15), si.Flow(0.3, 500.0)),
             (si.Grid(3, 12, 16, 8, si.LX_04, -15, 15, si.LX_04), si.Flow(0.5, 800.0)), si.mixing_layer_2d(64, 128)]
    ks = [1, 5, 11, 40]
    hs = [Stab(si.tanh_base_flow(g, f), g, f.Ma, f.Re, f.Pr) for g, f in specs]
    Vs, ws = [], []
    for i, (S, k) in enumerate(zip(hs, ks)):
        rng = np.random.default_rng(40 + i)
        A = rng.standard_normal((S.n, k)) + 1j * rng.standard_normal((S.n, k))
        Q, _ = np.linalg.qr(A)
        Vs.append(torch.from_numpy(np.ascontiguousarray(Q.T)).cuda())  # column j at V + j n
        ws.append(torch.from_numpy(si.random_complex(60 + i, S.n)).cuda())
    single = []
    for S, V, k, w in zip(hs, Vs, ks, ws):
        w1 = w.clone()
        h1, n1 = S.orthogonalize(V, k, w1)
        single.append((w1, h1, n1))
    B = JvBatch(hs)
    w2 = [w.clone() for w in ws]
    hcs, nrs = B.orthogonalize(Vs, ks, w2)
    for i, ((w1, h1, n1), w_b, h_b, n_b) in enumerate(zip(single, w2, hcs, nrs)):
        assert torch.equal(w1, w_b), i
        assert np.array_equal(h1, h_b), i
        assert n1 == n_b, i
    # the result is an orthogonalisation: w is orthogonal to the columns afterwards
    for V, k, w in zip(Vs, ks, w2):
        assert float((V.conj() @ w).abs().max()) < 1e-12 * float(w.abs().max())
    with pytest.raises(StabError, match="1 <= k"):
        B.orthogonalize(Vs, [0, 5, 11, 40], w2)
    B.close()
    for S in hs:
        S.close()
