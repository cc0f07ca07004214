"""Writes the stored expected values of the eigen-parity tests.

Calls only the oracle: the dense tangent Jacobian of the 32 x 64 mixing layer
(8,192 unknowns, Ma 0.3, Re 1000) assembled column by column by the complex
step, and its eigenvalues from LAPACK (scipy.linalg.eigvals).  Stores the
eigenvalues with the largest Cayley magnitude |theta| = |lambda - tau| /
|lambda - sigma| for two Cayley parameter pairs.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np
import scipy.linalg as sla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import stab_inputs as si  # noqa: E402


def main():
    g, f = si.mixing_layer_2d(32, 64)
    P = oracle.Problem.from_inputs(g, f)
    q0 = si.tanh_base_flow(g, f)
    J = oracle.core.dense_jacobian(P, q0)
    lam = sla.eigvals(J)
    out = {"source": "oracle: dense complex-step Jacobian of the 32x64 layer (Ma 0.3, Re 1000, y in [-15, 15], "
                     "Lx = 2 pi / 0.4) and LAPACK eigenvalues; sorted by decreasing Cayley |theta|",
           "grid": [32, 64], "Ma": 0.3, "Re": 1000.0, "sets": []}
    for sigma, tau in ((0.2j, -1 + 0.2j), (0.25, -1.0)):
        th = (lam - tau) / (lam - sigma)
        o = np.argsort(-np.abs(th), kind="stable")[:16]
        out["sets"].append({"sigma": [sigma.real if isinstance(sigma, complex) else sigma, complex(sigma).imag],
                            "tau": [complex(tau).real, complex(tau).imag],
                            "lambda": [[float(l.real), float(l.imag)] for l in lam[o]],
                            "abs_theta": [float(abs(t)) for t in th[o]]})
    with open(os.path.join(HERE, "c1_dense_eigs.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
