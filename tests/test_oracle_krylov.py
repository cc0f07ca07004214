"""Pins of the oracle's Krylov layer: CGS2, GMRES (Sec. Iterative solvers),
the Cayley map (Eq. cayley_transform) and IRAM (Algorithm iram, Eq. arnoldi,
Eq. ritz_estimate), against LAPACK and the algebra they must satisfy."""
import numpy as np
import pytest
import scipy.linalg as sla

import stab_inputs as si


def _nonnormal(n, seed):
    rng = np.random.default_rng(seed)
    lam = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = np.eye(n) + 0.3 * rng.standard_normal((n, n))
    return X @ np.diag(lam) @ np.linalg.inv(X)


def test_cgs2_orthogonality(orc):
    rng = np.random.default_rng(0)
    n, m = 500, 40
    V = np.zeros((n, m), dtype=complex)
    w = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    V[:, 0] = w / np.linalg.norm(w)
    for j in range(1, m):
        w = V[:, j - 1] + 1e-9 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))  # nearly dependent
        h, w2 = orc.krylov.cgs2(V[:, :j], w)
        assert np.linalg.norm(V[:, :j] @ h + w2 - w) < 1e-14 * np.linalg.norm(w)
        V[:, j] = w2 / np.linalg.norm(w2)
    assert np.abs(V.conj().T @ V - np.eye(m)).max() < 1e-13


def test_cayley_round_trip_and_reciprocal_form(orc):
    rng = np.random.default_rng(1)
    lam = rng.standard_normal(100) + 1j * rng.standard_normal(100)
    sigma, tau = 0.2j, -1 + 0.2j
    th = orc.krylov.cayley_theta(lam, sigma, tau)
    assert np.abs(orc.krylov.cayley_lambda(th, sigma, tau) - lam).max() < 1e-13 * np.abs(lam).max()
    mu = (lam - sigma) / (lam - tau)  # the reciprocal form of the same map
    assert np.abs(mu * th - 1).max() < 1e-14


def test_cayley_spectrum_of_dense_operator(orc):
    A = _nonnormal(30, 2)
    sigma, tau = 0.3 + 0.1j, -1.0
    C = np.linalg.solve(A - sigma * np.eye(30), A - tau * np.eye(30))
    th = np.linalg.eigvals(C)
    lam = np.linalg.eigvals(A)
    back = orc.krylov.cayley_lambda(th, sigma, tau)
    for l in lam:
        assert np.abs(back - l).min() < 1e-9 * (1 + abs(l))


@pytest.mark.parametrize("precond", [False, True])
def test_gmres_matches_direct_solve(orc, precond):
    rng = np.random.default_rng(3)
    n = 120
    A = _nonnormal(n, 3) + 4 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    M = None
    if precond:
        Dinv = 1 / np.diag(A)
        M = lambda q: Dinv * q  # noqa: E731
    x, st = orc.krylov.fgmres(lambda z: A @ z, b, M, m=15, tol=1e-12, max_restarts=100)
    ref = sla.solve(A, b)
    assert st.converged
    assert np.linalg.norm(x - ref) < 1e-9 * np.linalg.norm(ref)
    assert np.linalg.norm(b - A @ x) <= 1.01e-12 * np.linalg.norm(b)


def test_gmres_residual_monotone_within_cycle(orc):
    A = _nonnormal(80, 4) + 2 * np.eye(80)
    b = np.ones(80, dtype=complex)
    _, st = orc.krylov.fgmres(lambda z: A @ z, b, None, m=80, tol=1e-14, max_restarts=1)
    h = np.array(st.history)
    h = h[h > 1e-11]  # above the rounding floor of the small least-squares solve
    assert h.size > 20 and np.all(np.diff(h) <= 1e-15)


def test_iram_matches_lapack_and_keeps_arnoldi_relation(orc):
    n = 200
    A = _nonnormal(n, 5)
    sigma, tau = 0.5 + 0.5j, -2.0
    C = np.linalg.solve(A - sigma * np.eye(n), A - tau * np.eye(n))
    checks = []

    def check(V, H, f):
        m = V.shape[1]
        E = C @ V - V @ H
        E[:, -1] -= f
        checks.append(np.linalg.norm(E) / np.linalg.norm(C @ V))
        checks.append(np.abs(V.conj().T @ V - np.eye(m)).max())

    v0 = si.start_vector(0x5EED, n)
    res = orc.krylov.iram(lambda v: C @ v, v0, k=6, m=20, tol=1e-12, sigma=sigma, tau=tau,
                          arnoldi_check=check)
    assert res.nconv == 6
    assert max(checks) < 1e-12
    lam = np.linalg.eigvals(A)
    th = orc.krylov.cayley_theta(lam, sigma, tau)
    want = lam[np.argsort(-np.abs(th))[:6]]
    for l in res.lam:
        assert np.abs(want - l).min() < 1e-9 * abs(l)
    # Ritz estimate is the true residual of the Ritz pair for C
    for t, x in zip(res.theta, res.vectors.T):
        assert np.linalg.norm(C @ x - t * x) < 1e-10 * abs(t)


def test_splitmix64_vectorised_matches_reference_loop():
    import stab_inputs
    raw = stab_inputs.splitmix64_stream(12345, 64)
    u = stab_inputs.splitmix64_uniform(12345, 64)
    ref = (raw >> np.uint64(11)).astype(np.float64) / 2.0 ** 53 - 0.5
    assert np.array_equal(u, ref)
    assert -0.5 <= u.min() and u.max() < 0.5


@pytest.mark.parametrize("precond", [False, True])
def test_lgmres_matches_direct_solve(orc, precond):
    """LGMRES (augmented restarts) solves a non-normal system to the
    tolerance and agrees with LAPACK."""
    n = 240
    if precond:  # convection-diffusion stencil, block-Jacobi over blocks of 24
        A = (np.diag(np.full(n, 2.0)) + np.diag(np.full(n - 1, -1.6), -1) + np.diag(np.full(n - 1, -0.4), 1)
             + 0.05j * np.eye(n))
    else:
        A = _nonnormal(n, 7) + 4.0 * np.eye(n)
    b = si.random_complex(5, n)
    M = None
    if precond:
        lu = [sla.lu_factor(A[i:i + 24, i:i + 24]) for i in range(0, n, 24)]

        def M(v):
            return np.concatenate([sla.lu_solve(f, v[i:i + 24]) for f, i in zip(lu, range(0, n, 24))])
    x, st = orc.krylov.lgmres(lambda v: A @ v, b, M, m=12, k=3, tol=1e-11, max_restarts=500)
    assert st.converged
    assert np.linalg.norm(b - A @ x) <= 1.01e-11 * np.linalg.norm(b)
    assert np.linalg.norm(x - sla.solve(A, b)) < 1e-8 * np.linalg.norm(x)


def test_lgmres_without_augmentation_is_fgmres(orc):
    n = 150
    A = _nonnormal(n, 3) + 3.0 * np.eye(n)
    b = si.random_complex(6, n)
    x0, s0 = orc.krylov.fgmres(lambda v: A @ v, b, None, m=10, tol=1e-10, max_restarts=300)
    x1, s1 = orc.krylov.lgmres(lambda v: A @ v, b, None, m=10, k=0, tol=1e-10, max_restarts=300)
    assert s0.matvecs == s1.matvecs and s0.iterations == s1.iterations
    assert np.array_equal(x0, x1)


def test_lgmres_cycle_minimises_true_residual_over_its_space(orc):
    """Every cycle's new iterate minimises ||b - A x|| over x_old + span(W),
    W = the cycle's Krylov and augmentation directions: so the stored A z of
    the augmentation vectors (residual differences) is exact, and the flexible
    Arnoldi relation holds on them."""
    n = 300
    A = _nonnormal(n, 11) + 4.0 * np.eye(n)
    b = si.random_complex(8, n)
    seen = []

    def check(W, x_old, x_new):
        r_old = b - A @ x_old
        y = np.linalg.lstsq(A @ W, r_old, rcond=None)[0]
        best = np.linalg.norm(r_old - A @ W @ y)
        got = np.linalg.norm(b - A @ x_new)
        seen.append(W.shape[1])
        assert got <= best * (1 + 1e-8) + 1e-13 * np.linalg.norm(b)
    x, st = orc.krylov.lgmres(lambda v: A @ v, b, None, m=8, k=2, tol=1e-10, max_restarts=400, cycle_check=check)
    assert st.converged and len(seen) >= 3
