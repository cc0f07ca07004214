"""Parity of the CUDA J(q0) v (Eq. frechet) with the oracle, through the C ABI.

Tolerances: the cancellation-free epsilon-quotient matches the binary128
value of the same quotient to 1e-10 relative (element by element, scaled by
the largest entry, and in the 2-norm); the exact-tangent mode matches the
complex-step tangent to 1e-10 as well."""
import numpy as np
import pytest

import stab_inputs as si
from gpu_util import max_rel_err, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _gpu(q0, g, f, v, shift=0.0, **opts):
    import torch
    from paper_1502_03701_gb300 import Stab
    S = Stab(q0, g, f.Ma, f.Re, f.Pr, **opts)
    dv = torch.from_numpy(np.ascontiguousarray(v)).cuda()
    out = torch.empty_like(dv)
    S.apply_J(dv, out, shift)
    torch.cuda.synchronize()
    eps = S.last_eps()
    res = out.cpu().numpy()
    S.close()
    return res, eps


CASES = [
    # name, grid, flow, general base?
    ("small2d_visc", si.Grid(2, 32, 64, 1, si.LX_04, -15, 15), si.Flow(0.3, 1000.0), False),
    ("ragged2d_visc_stretched", si.Grid(2, 70, 67, 1, si.LX_04, -15, 15, 1.0, 1.7), si.Flow(0.6, 500.0), False),
    ("general2d_inviscid", si.Grid(2, 24, 40, 1, si.LX_04, -15, 15), si.Flow(0.9, 0.0), True),
    ("general2d_visc", si.Grid(2, 16, 20, 1, si.LX_04, -15, 15, 1.0, 1.2), si.Flow(0.3, 200.0), True),
    ("small3d_visc", si.Grid(3, 12, 16, 8, si.LX_04, -15, 15, si.LX_04), si.Flow(0.5, 800.0), False),
    ("general3d_visc", si.Grid(3, 8, 10, 7, si.LX_04, -15, 15, 5.0, 0.8), si.Flow(0.4, 300.0), True),
]


@pytest.mark.parametrize("stencil_prec", [64, 48])
@pytest.mark.parametrize("name,g,f,general", CASES, ids=[c[0] for c in CASES])
def test_jv_eps_quotient_matches_quad_oracle(orc, name, g, f, general, stencil_prec):
    q0 = si.perturbed_base_flow(g, f, seed=21) if general else si.tanh_base_flow(g, f)
    v = si.random_complex(101, g.n)
    got, eps = _gpu(q0, g, f, v, stencil_prec=stencil_prec)
    assert eps > 0
    P = orc.Problem.from_inputs(g, f)
    ref = orc.core.jv(P, q0, v, "quad", eps)
    assert abs(eps - orc.core.knoll_keyes_eps(q0, v)) < 1e-12 * eps
    assert max_rel_err(got, ref) < TOL, name
    assert rel_err(got, ref) < TOL, name


@pytest.mark.parametrize("stencil_prec", [64, 48])
@pytest.mark.parametrize("name,g,f,general", CASES, ids=[c[0] for c in CASES])
def test_jv_tangent_matches_complex_step(orc, name, g, f, general, stencil_prec):
    q0 = si.perturbed_base_flow(g, f, seed=22) if general else si.tanh_base_flow(g, f)
    v = si.random_complex(102, g.n)
    got, eps = _gpu(q0, g, f, v, eps_mode=2, stencil_prec=stencil_prec)
    assert eps == 0.0
    ref = orc.core.jv(orc.Problem.from_inputs(g, f), q0, v, "tangent")
    assert max_rel_err(got, ref) < TOL, name
    assert rel_err(got, ref) < TOL, name


def test_jv_shift_fixed_eps_and_bulk_viscosity(orc):
    g, f = si.mixing_layer_2d(16, 32)
    q0 = si.tanh_base_flow(g, f)
    v = si.random_complex(5, g.n)
    tau = -1 + 0.2j
    got, eps = _gpu(q0, g, f, v, shift=tau, eps=1e-6, bulk_visc_ratio=0.7)
    assert eps == 1e-6
    P = orc.Problem.from_inputs(g, f, bulk=0.7)
    ref = orc.core.jv(P, q0, v, "quad", 1e-6) - tau * v
    assert max_rel_err(got, ref) < TOL


def test_jv_zero_vector_and_determinism(orc):
    import torch
    from paper_1502_03701_gb300 import Stab
    g, f = si.mixing_layer_2d(32, 64)
    S = Stab(si.tanh_base_flow(g, f), g, f.Ma, f.Re, f.Pr)
    z = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    out = torch.full_like(z, 7.0)
    S.apply_J(z, out)
    assert torch.count_nonzero(out).item() == 0 and S.last_eps() == 0.0
    v = torch.from_numpy(si.random_complex(9, g.n)).cuda()
    a, b = torch.empty_like(v), torch.empty_like(v)
    S.apply_J(v, a)
    S.apply_J(v, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    S.close()


def test_invalid_arguments_fail_loudly():
    import torch
    from paper_1502_03701_gb300 import Stab, StabError
    g, f = si.mixing_layer_2d(16, 16)
    S = Stab(si.tanh_base_flow(g, f), g, f.Ma, f.Re, f.Pr)
    v = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    with pytest.raises(StabError, match="overlap"):
        S.apply_J(v, v)
    S.close()
    with pytest.raises(StabError, match="UNSUPPORTED"):
        Stab(si.tanh_base_flow(g, f), g, f.Ma, f.Re, f.Pr, eps_mode=1)
    bad = si.tanh_base_flow(g, f)
    bad[0, 0, 3, 3] = -1.0
    with pytest.raises(StabError, match="positive pressure"):
        Stab(bad, g, f.Ma, f.Re, f.Pr)


@pytest.mark.parametrize("stencil_prec", [64, 48])
@pytest.mark.parametrize("mode", ["tangent", "quad"])
def test_jv_full_size_256x512(orc, mode, stencil_prec):
    """The 256 x 512 layer (524,288 unknowns): every element against the oracle."""
    g, f = si.mixing_layer_2d(256, 512)
    q0 = si.tanh_base_flow(g, f)
    v = si.random_complex(2024, g.n)
    got, eps = _gpu(q0, g, f, v, eps_mode=2 if mode == "tangent" else 0, stencil_prec=stencil_prec)
    ref = orc.core.jv(orc.Problem.from_inputs(g, f), q0, v, mode, eps if mode == "quad" else None)
    assert max_rel_err(got, ref) < TOL


def test_jv_full_size_3d_128x256x64(orc):
    """The 128 x 256 x 64 three-dimensional layer (10,485,760 unknowns), exact
    tangent against the complex-step oracle on every element."""
    g, f = si.mixing_layer_3d(128, 256, 64)
    q0 = si.tanh_base_flow(g, f)
    v = si.random_complex(303, g.n)
    got, eps = _gpu(q0, g, f, v, eps_mode=2)
    ref = orc.core.jv(orc.Problem.from_inputs(g, f), q0, v, "tangent")
    assert max_rel_err(got, ref) < TOL
    assert rel_err(got, ref) < TOL


def test_phase_timing_records_every_launch_group():
    """stab_timing: one interval per phase per J v, none when disabled."""
    import torch
    from paper_1502_03701_gb300 import Stab
    for g, f, expect_z in ((si.Grid(2, 32, 64, 1, si.LX_04, -15, 15), si.Flow(0.3, 1000.0), 0),
                           (si.Grid(3, 12, 16, 8, si.LX_04, -15, 15, si.LX_04), si.Flow(0.5, 800.0), 1)):
        q0 = si.tanh_base_flow(g, f)
        S = Stab(q0, g, f.Ma, f.Re, f.Pr)
        v = torch.from_numpy(si.random_complex(7, g.n)).cuda()
        out = torch.empty_like(v)
        S.timing(True)
        for _ in range(5):
            S.apply_J(v, out)
        ph = S.timing_read()
        for k in ("eps", "temperature", "line_y", "line_x", "pointwise"):
            assert ph[k][1] == 5 and ph[k][0] > 0, k
        assert ph["line_z"][1] == 5 * expect_z
        assert ph["cgs2"][1] == 0 and ph["dropped"] == 0
        S.timing(False)
        S.apply_J(v, out)
        ph = S.timing_read()
        assert all(ph[k][1] == 0 for k in ph if k != "dropped")
        S.close()


@pytest.mark.parametrize("scale_exp", [-40, 0, 40])
def test_pair_stencil_scales_exactly(scale_exp):
    """The pair right-hand sides work on exponent-shifted copies of each CTA's
    input, so J(2^k v) = 2^k J v (exact tangent, linear in v) to rounding, and the
    pair-stencil J v agrees with the FP64-stencil J v to ~1e-13."""
    import torch
    from paper_1502_03701_gb300 import Stab
    g, f = si.mixing_layer_2d(32, 48)
    q0 = si.tanh_base_flow(g, f)
    v = torch.from_numpy(si.random_complex(77, g.n)).cuda()
    S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2, stencil_prec=48)
    S64 = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2)
    a, b, c = torch.empty_like(v), torch.empty_like(v), torch.empty_like(v)
    S.apply_J(v, a)
    S64.apply_J(v, c)
    s = 2.0 ** scale_exp
    S.apply_J(v * s, b)
    torch.cuda.synchronize()
    ref = c.cpu().numpy()
    assert max_rel_err(a.cpu().numpy(), ref) < 1e-12
    assert max_rel_err(b.cpu().numpy() / s, ref) < 1e-12
    S.close()
    S64.close()
