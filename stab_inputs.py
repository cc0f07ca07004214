"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle glue.

This module holds no arithmetic of the stability method itself: only the grid
coordinates, the analytic base flow of the model problem (a tanh mixing layer,
Sec. "Model problem", Eq. tanh), the workload definitions and a counter-based
random generator (splitmix64) for start vectors and perturbation directions.

Layout convention everywhere: a state or perturbation vector is stored as
``[var][z][y][x]`` with x fastest; 2-D problems have nz = 1 and the variables
(p, u, v, s); 3-D problems have (p, u, v, w, s).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = 1.4
# Sutherland constant 110.4 K over a 273.15 K reference temperature.
SUTHERLAND_S = 110.4 / 273.15

_MASK64 = (1 << 64) - 1


def splitmix64_stream(seed: int, count: int) -> np.ndarray:
    """``count`` outputs of splitmix64 (Steele, Lea and Flood, OOPSLA 2014).

    The state advances by the golden-ratio increment; each output is the
    state passed through the published two-multiply finaliser.
    """
    out = np.empty(count, dtype=np.uint64)
    state = seed & _MASK64
    for i in range(count):
        state = (state + 0x9E3779B97F4A7C15) & _MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        out[i] = z ^ (z >> 31)
    return out


def splitmix64_uniform(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [-1/2, 1/2) from the top 53 bits of splitmix64."""
    if count <= 0:
        return np.zeros(0)
    # vectorised splitmix64: state_i = seed + (i+1)*golden (mod 2^64)
    idx = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0) - 0.5


def random_complex(seed: int, n: int) -> np.ndarray:
    """Complex vector with Re and Im uniform in [-1/2, 1/2) (interleaved draws)."""
    u = splitmix64_uniform(seed, 2 * n)
    return u[0::2] + 1j * u[1::2]


def start_vector(seed: int, n: int) -> np.ndarray:
    """Normalised complex start vector for the Arnoldi iteration."""
    v = random_complex(seed, n)
    return v / np.linalg.norm(v)


@dataclasses.dataclass(frozen=True)
class Grid:
    """Cartesian grid: x (and z) periodic, y bounded on [ly0, ly1].

    ``stretch`` = 0 gives uniform y; beta > 0 clusters points at the centre
    of the y range through y(eta) = y_c + (L/2) sinh(beta (2 eta - 1)) / sinh(beta),
    eta uniform on [0, 1].
    """
    dim: int
    nx: int
    ny: int
    nz: int
    lx: float
    ly0: float
    ly1: float
    lz: float = 1.0
    stretch: float = 0.0

    @property
    def nvars(self) -> int:
        return self.dim + 2

    @property
    def npts(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n(self) -> int:
        return self.nvars * self.npts

    def y(self) -> np.ndarray:
        eta = np.arange(self.ny) / (self.ny - 1)
        if self.stretch == 0.0:
            return self.ly0 + (self.ly1 - self.ly0) * eta
        b = self.stretch
        yc = 0.5 * (self.ly0 + self.ly1)
        half = 0.5 * (self.ly1 - self.ly0)
        return yc + half * np.sinh(b * (2.0 * eta - 1.0)) / math.sinh(b)


@dataclasses.dataclass(frozen=True)
class Flow:
    Ma: float
    Re: float  # <= 0 means inviscid (Re -> infinity)
    Pr: float = 0.71
    gamma: float = GAMMA
    S: float = SUTHERLAND_S


def tanh_base_flow(grid: Grid, flow: Flow) -> np.ndarray:
    """Base state q0 of the mixing layer: u = tanh(y), other velocities 0,
    uniform pressure 1/(gamma Ma^2) (unit density and temperature) and s = 0.
    Returns float64 of shape (nvars, nz, ny, nx)."""
    q = np.zeros((grid.nvars, grid.nz, grid.ny, grid.nx))
    q[0] = 1.0 / (flow.gamma * flow.Ma ** 2)
    q[1] = np.tanh(grid.y())[None, :, None]
    return q


def perturbed_base_flow(grid: Grid, flow: Flow, seed: int, amp: float = 1e-2) -> np.ndarray:
    """A base state that varies in every direction (tanh layer plus a seeded,
    smooth-in-nothing random perturbation of relative size ``amp``) for tests
    of the general (non-homogeneous) base path."""
    q = tanh_base_flow(grid, flow)
    r = splitmix64_uniform(seed, q.size).reshape(q.shape)
    scale = np.array([q[0].max()] + [1.0] * (grid.nvars - 1))[:, None, None, None]
    return q + amp * scale * r


# ---------------------------------------------------------------------------
# Workloads (the configurations the library is measured on)
# ---------------------------------------------------------------------------
LX_04 = 2.0 * math.pi / 0.4


def mixing_layer_2d(nx: int, ny: int, Ma: float = 0.3, Re: float = 1000.0) -> tuple[Grid, Flow]:
    return Grid(2, nx, ny, 1, LX_04, -15.0, 15.0), Flow(Ma, Re)


def mixing_layer_3d(nx: int, ny: int, nz: int, Ma: float = 0.3, Re: float = 1000.0) -> tuple[Grid, Flow]:
    return Grid(3, nx, ny, nz, LX_04, -15.0, 15.0, LX_04), Flow(Ma, Re)


# 32 x 64 2-D layer, 8,192 dofs; Cayley pole 0.2i, zero -1+0.2i; 6 of 30.
SMALL_2D = dict(nx=32, ny=64, Ma=0.3, Re=1000.0, sigma=0.2j, tau=-1 + 0.2j,
                nev=6, ncv=30, gmres_m=30, gmres_tol=1e-10)
# 256 x 512 2-D layer, 524,288 dofs; block-Jacobi over 8 x 8-point tiles.
LARGE_2D = dict(nx=256, ny=512, Ma=0.3, Re=1000.0, nev=10, ncv=60, gmres_m=50,
                tile=(8, 8), mach_sweep=(0.3, 0.6, 0.9))
# 128 x 256 x 64 3-D layer, 10,485,760 dofs.
LARGE_3D = dict(nx=128, ny=256, nz=64, Ma=0.3, Re=1000.0, nev=8, ncv=40, tile=(4, 4, 4))


def batched_instances(count: int = 64, seed: int = 1234, nxs=(32, 64, 128, 256),
                      nys=(64, 128, 256, 512)) -> list[dict]:
    """Uneven 2-D instances: Nx and Ny drawn uniformly from the sets (by default
    {32..256} and {64..512}), Ma ~ U[0.1, 0.9], Re log-uniform on [500, 5000]."""
    u = splitmix64_uniform(seed, 4 * count) + 0.5
    out = []
    for i in range(count):
        out.append(dict(nx=nxs[min(len(nxs) - 1, int(u[4 * i] * len(nxs)))],
                        ny=nys[min(len(nys) - 1, int(u[4 * i + 1] * len(nys)))],
                        Ma=0.1 + 0.8 * u[4 * i + 2],
                        Re=math.exp(math.log(500.0) + (math.log(5000.0) - math.log(500.0)) * u[4 * i + 3])))
    return out


def poisson_arrivals(count: int, rate: float, seed: int = 4321) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: exponential gaps of mean 1/rate."""
    u = splitmix64_uniform(seed, count) + 0.5          # [0, 1)
    gaps = -np.log1p(-u) / rate
    return np.cumsum(gaps)
