"""The allocation-free CGS2 entry point (for callers that cannot allocate
device memory, so cannot create a handle) against the handle-based one,
through the C ABI, on two calls in a row.  Collected last on purpose."""
import numpy as np
import pytest

import stab_inputs as si

pytestmark = pytest.mark.gpu


def test_noalloc_orthogonalize_matches_handle_version():
    import torch
    from paper_1502_03701_gb300 import Stab, StabError, binding
    g, f = si.mixing_layer_2d(16, 24)
    S = Stab(si.tanh_base_flow(g, f), g, f.Ma, f.Re, f.Pr)
    n = g.n
    rng = np.random.default_rng(9)
    for call, k in enumerate((13, 40)):  # two calls in a row, the second larger
        Vh = np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))[0]
        V = torch.from_numpy(np.ascontiguousarray(Vh.T)).cuda()
        w0 = si.random_complex(500 + call, n)
        wa = torch.from_numpy(w0.copy()).cuda()
        wb = torch.from_numpy(w0.copy()).cuda()
        ha, na = S.orthogonalize(V, k, wa)
        hb, nb = binding.orthogonalize_noalloc(V, k, n, wb, torch.cuda.current_stream())
        torch.cuda.synchronize()
        # the handle path forms its products in FP32-pair arithmetic (~2^-47 operand
        # splits), this one in FP64: they agree to the pair precision relative to ||w||
        wn = float(np.linalg.norm(w0))
        assert np.abs(ha - hb).max() <= 1e-12 * wn
        assert abs(na - nb) <= 1e-12 * wn
        assert torch.allclose(wa, wb, rtol=0, atol=1e-12 * wn)
    with pytest.raises(StabError, match="k <= 128"):
        binding.orthogonalize_noalloc(V, 129, n, wb)
    S.close()
