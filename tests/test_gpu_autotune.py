"""Line-pass launch shapes (stab_set_line_config, stab_autotune): every
admissible shape gives the same J v as the oracle (1e-10 relative, as the
other J v parity tests), and the tuner's cache is shared by handles of one shape."""
import numpy as np
import pytest

import stab_inputs as si
from gpu_util import max_rel_err, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10

CASES = [
    ("ragged2d_stretched", si.Grid(2, 70, 67, 1, si.LX_04, -15, 15, 1.0, 1.7), si.Flow(0.6, 500.0)),
    ("small3d", si.Grid(3, 12, 16, 8, si.LX_04, -15, 15, si.LX_04), si.Flow(0.5, 800.0)),
    # 33 points in y: chunks of 16 and 32 end one point before the wall (t1 = n - 1)
    ("ragged_y33", si.Grid(2, 20, 33, 1, si.LX_04, -15, 15), si.Flow(0.4, 700.0)),
]


@pytest.mark.parametrize("stencil_prec", [64, 48])
@pytest.mark.parametrize("name,g,f", CASES, ids=[c[0] for c in CASES])
def test_every_line_shape_matches_oracle(orc, name, g, f, stencil_prec):
    import torch
    from paper_1502_03701_gb300 import Stab, StabError
    q0 = si.tanh_base_flow(g, f)
    v = si.random_complex(301, g.n)
    S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2, stencil_prec=stencil_prec)
    P = orc.Problem.from_inputs(g, f)
    ref = orc.core.jv(P, q0, v, "tangent")
    dv = torch.from_numpy(v).cuda()
    out = torch.empty_like(dv)
    tried = 0
    for kinds in (1, 2, 3):
        for C in (16, 32, 64):
            for L in (1, 3, 8, 32):
                ok = True
                for ax in range(g.dim):
                    try:
                        S.set_line_config(ax, C, L, kinds)
                    except StabError:
                        ok = False
                if not ok:
                    continue
                S.apply_J(dv, out)
                got = out.cpu().numpy()
                assert max_rel_err(got, ref) < TOL, (C, L, kinds)
                assert rel_err(got, ref) < TOL, (C, L, kinds)
                tried += 1
    assert tried >= 14
    with pytest.raises(StabError):
        S.set_line_config(0, 24, 1, 1)
    with pytest.raises(StabError):
        S.set_line_config(0, 32, 1, 4)
    with pytest.raises(StabError):
        S.set_line_config(0, 16, 33, 3)
    S.close()


def test_autotune_picks_a_shape_and_shares_it(orc):
    import torch
    from paper_1502_03701_gb300 import Stab
    g, f = CASES[0][1], CASES[0][2]
    q0 = si.tanh_base_flow(g, f)
    S = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2)
    res = S.autotune(force=True)
    assert set(res) == {"x", "y"}
    for C, L, kinds, ms in res.values():
        assert C in (16, 32, 64) and 1 <= L <= 32 and kinds in (1, 2, 3) and ms > 0
    v = si.random_complex(302, g.n)
    dv = torch.from_numpy(v).cuda()
    out = torch.empty_like(dv)
    S.apply_J(dv, out)
    ref = orc.core.jv(orc.Problem.from_inputs(g, f), q0, v, "tangent")
    assert max_rel_err(out.cpu().numpy(), ref) < TOL
    S2 = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2)
    res2 = S2.autotune(force=False)
    for ax in res:
        assert res2[ax][:3] == res[ax][:3] and res2[ax][3] == -1.0
    # the cached shape is applied at creation: identical results bit for bit
    out2 = torch.empty_like(dv)
    S3 = Stab(q0, g, f.Ma, f.Re, f.Pr, eps_mode=2)
    S3.apply_J(dv, out2)
    assert torch.equal(out, out2)
    for s in (S, S2, S3):
        s.close()
