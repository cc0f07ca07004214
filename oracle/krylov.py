"""Krylov side of the oracle (test infrastructure only): CGS2, restarted
right-preconditioned (flexible) GMRES, the Cayley map and the implicitly
restarted Arnoldi method, in plain NumPy/SciPy complex128.

Readings where the paper is silent (listed in the design notes):
 * Gram-Schmidt variant: classical Gram-Schmidt applied twice (CGS2);
 * GMRES (Sec. "Iterative solvers", Saad-Schultz): x0 = 0, right
   preconditioning in flexible form, stop when ||b - A x|| <= tol ||b||;
 * Cayley transform (Eq. cayley_transform): sigma is the pole, tau the zero,
   C = (J - sigma I)^-1 (J - tau I), theta = (lambda - tau)/(lambda - sigma);
 * IRAM (Algorithm iram): wanted = the k Ritz values of largest |theta|, the
   p = m - k others are the exact shifts; f_k = (V_m Q)e_{k+1} beta_k + f_m
   sigma_k and H_k = the leading k x k block of the shifted H_m;
 * Ritz estimate (Eq. ritz_estimate) with the Frobenius norm of H_m.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

EPS_M = np.finfo(np.float64).eps


def cgs2(V: np.ndarray, w: np.ndarray):
    """Orthogonalise w against the orthonormal columns of V, twice (CGS2).
    Returns (h, w_perp) with w = V h + w_perp."""
    h1 = V.conj().T @ w
    w = w - V @ h1
    h2 = V.conj().T @ w
    w = w - V @ h2
    return h1 + h2, w


def cayley_theta(lam, sigma, tau):
    """theta = (lambda - tau) / (lambda - sigma) (Eq. cayley_transform, sigma = pole)."""
    return (lam - tau) / (lam - sigma)


def cayley_lambda(theta, sigma, tau):
    """Inverse map: lambda = (sigma theta - tau) / (theta - 1)."""
    return (sigma * theta - tau) / (theta - 1.0)


@dataclass
class GmresStats:
    matvecs: int = 0
    iterations: int = 0
    restarts: int = 0
    converged: bool = False
    history: list = field(default_factory=list)


def fgmres(A, b, M=None, m: int = 30, tol: float = 1e-10, max_restarts: int = 200):
    """Restarted GMRES(m) (Saad & Schultz 1986) with right preconditioning in
    flexible form (Z_j = M v_j kept), x0 = 0.  The small least-squares problem
    is solved with a library least-squares routine at every step."""
    n = b.size
    st = GmresStats()
    x = np.zeros(n, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        st.converged = True
        return x, st
    r = b.astype(np.complex128).copy()
    beta = bnorm
    for cycle in range(max_restarts):
        V = np.zeros((n, m + 1), dtype=np.complex128)
        Z = np.zeros((n, m), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        V[:, 0] = r / beta
        y = None
        jend = 0
        for j in range(m):
            Z[:, j] = V[:, j] if M is None else M(V[:, j])
            w = A(Z[:, j])
            st.matvecs += 1
            st.iterations += 1
            h, w = cgs2(V[:, :j + 1], w)
            H[:j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w)
            e1 = np.zeros(j + 2, dtype=np.complex128)
            e1[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
            res = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)
            st.history.append(res / bnorm)
            jend = j + 1
            if res <= tol * bnorm or H[j + 1, j] == 0.0:
                break
            V[:, j + 1] = w / H[j + 1, j]
        x = x + Z[:, :jend] @ y
        r = b - A(x)
        st.matvecs += 1
        beta = np.linalg.norm(r)
        st.restarts = cycle + 1
        if beta <= tol * bnorm:
            st.converged = True
            break
    return x, st


def lgmres(A, b, M=None, m: int = 30, k: int = 2, tol: float = 1e-10, max_restarts: int = 200,
           cycle_check=None):
    """Restarted GMRES with augmented restarts, LGMRES (Baker, Jessup and
    Manteuffel 2005; the paper's Sec. "Iterative solvers" and Table
    comparison_overall use it next to GMRES).

    Every cycle spans the same number m of directions as GMRES(m): m - a
    Krylov directions of the current residual (right-preconditioned, kept in
    flexible form) followed by the a <= k most recent error approximations
    z_c = x_{c+1} - x_c of earlier cycles (newest first), each stored with
    A z_c so that it enters the Arnoldi process without a matrix-vector
    product.  A z_c is the difference of the true residuals before and after
    the cycle.  The stored pairs are scaled to unit ||z||.  x0 = 0; stop when
    ||b - A x|| <= tol ||b||.  With k = 0 this is ``fgmres``.
    ``cycle_check(W, x_old, x_new)`` is called after every cycle with the
    cycle's search directions (for the minimisation pin of the tests)."""
    n = b.size
    st = GmresStats()
    x = np.zeros(n, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        st.converged = True
        return x, st
    r = b.astype(np.complex128).copy()
    beta = bnorm
    aug = []  # (z, A z) pairs, newest first
    for cycle in range(max_restarts):
        nkry = m - len(aug)
        V = np.zeros((n, m + 1), dtype=np.complex128)
        Z = np.zeros((n, m), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        V[:, 0] = r / beta
        y = None
        jend = 0
        for j in range(m):
            if j < nkry:
                Z[:, j] = V[:, j] if M is None else M(V[:, j])
                w = A(Z[:, j])
                st.matvecs += 1
            else:
                Z[:, j], w = aug[j - nkry]
                w = w.copy()
            st.iterations += 1
            h, w = cgs2(V[:, :j + 1], w)
            H[:j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w)
            e1 = np.zeros(j + 2, dtype=np.complex128)
            e1[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
            res = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)
            st.history.append(res / bnorm)
            jend = j + 1
            if res <= tol * bnorm or H[j + 1, j] == 0.0:
                break
            V[:, j + 1] = w / H[j + 1, j]
        dz = Z[:, :jend] @ y
        if cycle_check is not None:
            cycle_check(Z[:, :jend].copy(), x.copy(), x + dz)
        x = x + dz
        r_new = b - A(x)
        st.matvecs += 1
        dn = np.linalg.norm(dz)
        if k > 0 and dn > 0.0:
            aug.insert(0, (dz / dn, (r - r_new) / dn))
            del aug[k:]
        r = r_new
        beta = np.linalg.norm(r)
        st.restarts = cycle + 1
        if beta <= tol * bnorm:
            st.converged = True
            break
    return x, st


def _wanted_order(theta, sigma, tau):
    """Indices sorted by decreasing |theta|, ties by larger Re lambda, then Im lambda."""
    lam = cayley_lambda(theta, sigma, tau)
    return np.lexsort((-lam.imag, -lam.real, -np.abs(theta)))


@dataclass
class IramResult:
    theta: np.ndarray
    lam: np.ndarray
    vectors: np.ndarray
    estimates: np.ndarray
    nconv: int
    restarts: int
    ops: int
    H: np.ndarray = None
    V: np.ndarray = None
    f: np.ndarray = None


def iram(apply_C, v0, k: int, m: int, tol: float, sigma=0.0, tau=0.0, max_restarts: int = 300,
         arnoldi_check=None):
    """Implicitly restarted Arnoldi (Algorithm iram, after Sorensen) on the
    operator apply_C, wanted = k Ritz values of largest magnitude.
    ``arnoldi_check(V, H, f)`` is called after every restart (for the
    Arnoldi-relation invariant tests)."""
    n = v0.size
    V = np.zeros((n, m), dtype=np.complex128)
    H = np.zeros((m, m), dtype=np.complex128)
    f = np.asarray(v0, dtype=np.complex128) / np.linalg.norm(v0)
    ops = 0
    j0 = 0
    first = True
    for restart in range(max_restarts + 1):
        # extend the factorisation from j0 to m steps
        for j in range(j0, m):
            beta = np.linalg.norm(f)
            if not first or j > 0:
                H[j, j - 1] = beta
            V[:, j] = f / beta
            w = apply_C(V[:, j])
            ops += 1
            h, f = cgs2(V[:, :j + 1], w)
            H[:j + 1, j] = h
        first = False
        if arnoldi_check is not None:
            arnoldi_check(V, H, f)
        # spectrum of H_m, wanted / unwanted split, Ritz estimates
        theta, Y = sla.eig(H)
        Y = Y / np.linalg.norm(Y, axis=0)
        order = _wanted_order(theta, sigma, tau)
        want, shifts = order[:k], order[k:]
        fnorm = np.linalg.norm(f)
        est = fnorm * np.abs(Y[m - 1, want])
        bound = np.maximum(EPS_M * np.linalg.norm(H), tol * np.abs(theta[want]))
        conv = est <= bound
        if conv.all() or restart == max_restarts:
            x = V @ Y[:, want]
            return IramResult(theta[want], cayley_lambda(theta[want], sigma, tau), x, est,
                              int(conv.sum()), restart, ops, H.copy(), V.copy(), f.copy())
        # implicit QR shifts with the unwanted Ritz values
        Q = np.eye(m, dtype=np.complex128)
        for mu in theta[shifts]:
            Qj, _ = np.linalg.qr(H - mu * np.eye(m))
            H = Qj.conj().T @ H @ Qj
            Q = Q @ Qj
        beta_k = H[k, k - 1]
        sigma_k = Q[m - 1, k - 1]
        f = (V @ Q[:, k]) * beta_k + f * sigma_k
        V[:, :k] = V @ Q[:, :k]
        V[:, k:] = 0.0
        H[k:, :] = 0.0
        H[:, k:] = 0.0
        j0 = k
    raise AssertionError("unreachable")
