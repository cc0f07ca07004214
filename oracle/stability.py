"""Stability driver of the oracle (test infrastructure only): Cayley-IRAM with
inexact GMRES inner solves and the local block-Jacobi preconditioner
(Sec. "Preconditioning", after Hegland 1991), on top of the C++ J(q0) v.

Block-Jacobi reading: one block per tile of tx x ty (x tz) grid points with
all variables; the block is the principal submatrix of (J - sigma I) over the
tile's dofs, J the exact tangent; LU with partial pivoting; applied on the
right.  Dof order inside a tile: [var][lz][ly][lx], lx fastest.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import core
from .krylov import cayley_lambda, cayley_theta, fgmres, iram


def tile_dofs(P: core.Problem, tile) -> list[np.ndarray]:
    """Global dof indices of every tile, tiles ordered (tz, ty, tx), tx fastest."""
    tx, ty = tile[0], tile[1]
    tz = tile[2] if P.dim == 3 else 1
    assert P.nx % tx == 0 and P.ny % ty == 0 and P.nz % tz == 0
    nv = P.dim + 2
    out = []
    for bz in range(P.nz // tz):
        for by in range(P.ny // ty):
            for bx in range(P.nx // tx):
                z = bz * tz + np.arange(tz)
                y = by * ty + np.arange(ty)
                x = bx * tx + np.arange(tx)
                pts = ((z[:, None, None] * P.ny + y[None, :, None]) * P.nx + x[None, None, :]).reshape(-1)
                out.append((np.arange(nv)[:, None] * P.npts + pts[None, :]).reshape(-1))
    return out


def blocks_from_dense(J: np.ndarray, P: core.Problem, tile, sigma) -> np.ndarray:
    """Principal submatrices of (J - sigma I) over the tiles, shape (ntiles, b, b)."""
    idx = tile_dofs(P, tile)
    return np.stack([J[np.ix_(d, d)] - sigma * np.eye(d.size) for d in idx])


def block_from_columns(P: core.Problem, q0, tile, t: int, sigma) -> np.ndarray:
    """One tile's block computed from J's columns at the tile's dofs."""
    d = tile_dofs(P, tile)[t]
    cols = core.jacobian_columns(P, q0, d)
    return cols[d, :] - sigma * np.eye(d.size)


class BlockJacobi:
    """z = M^{-1} q with M = blockdiag of the tile blocks, LU-factored."""

    def __init__(self, P: core.Problem, tile, blocks: np.ndarray):
        self.idx = tile_dofs(P, tile)
        self.lu = [sla.lu_factor(B) for B in blocks]

    def __call__(self, q: np.ndarray) -> np.ndarray:
        z = np.empty_like(q, dtype=np.complex128)
        for d, lu in zip(self.idx, self.lu):
            z[d] = sla.lu_solve(lu, q[d])
        return z


def cayley_eigs(P: core.Problem, q0, sigma, tau, nev: int, ncv: int, tol: float,
                gmres_m: int, gmres_tol: float, v0, precond=None, mode: str = "tangent",
                max_restarts: int = 300, gmres_max_restarts: int = 200):
    """Eigenvalues of J(q0) nearest the Cayley-selected region (Alg. iram on
    C = (J - sigma I)^-1 (J - tau I), Eqs. cayley_transform, cayley_arnoldi)."""
    q0 = np.asarray(q0, dtype=np.float64).reshape(-1)
    counts = {"jv": 0, "gmres_it": 0}

    def J(v):
        counts["jv"] += 1
        return core.jv(P, q0, v, mode=mode)

    def C(v):
        b = J(v) - tau * v
        x, st = fgmres(lambda z: J(z) - sigma * z, b, precond, gmres_m, gmres_tol, gmres_max_restarts)
        counts["gmres_it"] += st.iterations
        return x

    res = iram(C, np.asarray(v0), nev, ncv, tol, sigma, tau, max_restarts)
    resid = np.array([np.linalg.norm(core.jv(P, q0, x, "tangent") - lam * x) / np.linalg.norm(x)
                      for lam, x in zip(res.lam, res.vectors.T)])
    return res, resid, counts


def dense_reference(J: np.ndarray, sigma, tau, count: int):
    """Eigenvalues of the dense J (LAPACK) sorted by decreasing |theta|."""
    lam = sla.eigvals(J)
    th = cayley_theta(lam, sigma, tau)
    order = np.argsort(-np.abs(th), kind="stable")
    return lam[order[:count]], th[order[:count]]


__all__ = ["tile_dofs", "blocks_from_dense", "block_from_columns", "BlockJacobi", "cayley_eigs",
           "dense_reference", "cayley_lambda", "cayley_theta"]
