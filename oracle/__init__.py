"""CPU oracle for the stability path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, independent restatement of what the GPU library computes:
the discretised right-hand side N(q) (Eq. navier_stokes), the three forms of
J(q0) v (Eq. frechet), the dense Jacobian, CGS2, GMRES, the Cayley map and
the implicitly restarted Arnoldi method (Algorithm iram), and the block-Jacobi
preconditioner.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the library never does.
"""
from . import core, krylov, stability  # noqa: F401
from .core import Problem, build  # noqa: F401
