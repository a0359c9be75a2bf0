"""Seeded synthetic workloads for the coupled Allen–Cahn/Cahn–Hilliard time step.

This module holds no arithmetic of the method.  It only says which grid,
coefficients, solver settings and initial fields a run uses, and draws the
initial fields from a seeded NumPy PCG64 generator.  Both the CPU oracle and the
CUDA path are fed from here, so the two sides always see the same inputs.

Initial fields follow the paper's random-perturbation recipe (Sec. 4.1 A and B:
a constant state plus uniform noise on u and v); the amplitudes, seeds, grid
sizes and coefficients are those of the five named workloads below.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import Tuple

import numpy as np

BC_PERIODIC = 0
BC_NEUMANN = 1
DT_FIXED = 0
DT_ADAPTIVE = 1
RAS_LEFT = 0
RAS_AS = 1
RAS_RIGHT = 2
PREC_FP64 = 0
PREC_MIXED = 1
JAC_MATFREE = 0
JAC_ASSEMBLED = 1
SUB_ILU0 = 0
SUB_ILU1 = 1
SUB_ILU2 = 2
SUB_LU = 3


@dataclass
class Params:
    """Problem and solver settings (field names follow the C struct acac_params)."""

    dim: int = 2
    n: Tuple[int, int, int] = (64, 64, 1)        # Nx, Ny, Nz
    L: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    bc: int = BC_PERIODIC
    alpha: float = 3.0
    beta: float = 1.0
    theta: float = 0.3
    gamma: float = 1e-3
    rho: float = 1.0
    taylor_S: int = 10
    dt_mode: int = DT_FIXED
    dt0: float = 1e-3
    dt_min: float = 1e-5
    dt_max: float = 1e-1
    eta0: float = 1e4
    newton_rtol: float = 1e-8
    newton_atol: float = 1e-13
    newton_maxit: int = 20
    gmres_rtol: float = 1e-6
    gmres_atol: float = 1e-14
    gmres_restart: int = 30
    gmres_maxit: int = 500
    ras_parts: Tuple[int, int, int] = (4, 4, 1)
    ras_overlap: int = 1
    ras_type: int = RAS_LEFT
    ilu_reuse: int = 1
    precision: int = PREC_FP64
    jac_mode: int = JAC_MATFREE
    batch: int = 1
    cgs_refine: int = 1          # 1: CGS2 (two passes), 0: single classical pass
    graphs: int = 1              # 1: GMRES iterations replayed from captured CUDA graphs
    ras_window: int = 0          # 2D Schwarz apply: 0 choose, 1 level window, 2 whole box vector
    subdomain_solver: int = SUB_ILU0   # ILU(0), ILU(1), ILU(2) or LU (Sec. 4.2, Table 2)

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)

    @property
    def shape(self) -> Tuple[int, ...]:
        """Array shape of one field, slowest axis first (x is the last axis)."""
        nx, ny, nz = self.n
        return (ny, nx) if self.dim == 2 else (nz, ny, nx)

    @property
    def ncells(self) -> int:
        return int(np.prod(self.shape))


def initial_fields(p: Params, seed: int, u_mean: float, amp: float):
    """u = u_mean + amp*U(-1,1), v = amp*U(-1,1), drawn u then v from PCG64(seed)."""
    rng = np.random.default_rng(seed)
    noise = rng.uniform(-1.0, 1.0, size=(2,) + p.shape)
    u = u_mean + amp * noise[0]
    v = amp * noise[1]
    return np.ascontiguousarray(u), np.ascontiguousarray(v)


def perturbed_pair(p: Params, seed: int, u_mean: float = 0.5, amp: float = 0.05,
                   step_amp: float = 1e-3):
    """Two nearby admissible states (U1, U0) for residual / Jacobian parity checks.

    U0 is drawn as initial_fields(seed); U1 = U0 + step_amp*U(-1,1) (seed+1).
    """
    u0, v0 = initial_fields(p, seed, u_mean, amp)
    rng = np.random.default_rng(seed + 1)
    d = rng.uniform(-1.0, 1.0, size=(2,) + p.shape)
    return (u0 + step_amp * d[0], v0 + step_amp * d[1]), (u0, v0)


def near_pure_pair(p: Params, seed: int, frac: float = 0.5, eps_range=(1e-8, 1e-3),
                   ratio_max: float = 0.7):
    """Two admissible states (U1, U0) for parity checks near pure phases and at large
    series ratios (the regime of Lemma 2.2's series where the logarithms and the
    truncation of the sum matter most).

    Works in the variables p = u + v and q = u - v of Eq. D2-1, each of which must lie
    in (0, 1), through their midpoints zeta and half changes sigma.  zeta: a background
    0.45 +- 0.05; in a seeded fraction `frac` of the cells one of zeta_p, zeta_q (or
    both) is put at eps or 1 - eps with log10(eps) uniform over eps_range, so that
    u +- v lies within about 1e-8..1e-3 of 0 or 1 (and v near +-1/2 where p and q sit at
    opposite ends).  sigma = r min(zeta, 1 - zeta) with r uniform over (-ratio_max,
    ratio_max), so that max(|sigma/zeta|, |sigma/(1 - zeta)|) = |r|.  The end states
    are zeta -+ sigma.  Returns ((u1, v1), (u0, v0)) in the shape of one field."""
    rng = np.random.default_rng(seed)
    shape = p.shape
    zeta = 0.45 + 0.05 * rng.uniform(-1.0, 1.0, size=(2,) + shape)
    pick = rng.uniform(0.0, 1.0, size=shape) < frac
    which = rng.integers(0, 3, size=shape)                  # 0: p, 1: q, 2: both
    lo, hi = np.log10(eps_range[0]), np.log10(eps_range[1])
    eps = 10.0 ** rng.uniform(lo, hi, size=(2,) + shape)
    side = rng.integers(0, 2, size=(2,) + shape)              # 0: near 0, 1: near 1
    for a in range(2):
        sel = pick & ((which == a) | (which == 2))
        zeta[a] = np.where(sel, np.where(side[a] == 0, eps[a], 1.0 - eps[a]), zeta[a])
    r = rng.uniform(-ratio_max, ratio_max, size=(2,) + shape)
    sigma = r * np.minimum(zeta, 1.0 - zeta)
    pq0, pq1 = zeta - sigma, zeta + sigma
    u0, v0 = 0.5 * (pq0[0] + pq0[1]), 0.5 * (pq0[0] - pq0[1])
    u1, v1 = 0.5 * (pq1[0] + pq1[1]), 0.5 * (pq1[0] - pq1[1])
    return ((np.ascontiguousarray(u1), np.ascontiguousarray(v1)),
            (np.ascontiguousarray(u0), np.ascontiguousarray(v0)))


def near_pure_state(p: Params, seed: int, eps_p: float, eps_q: float, spread: float = 0.5,
                    flip: bool = False):
    """A start state close to the pure phase p = u + v -> 0, q = u - v -> 1 (so u near
    1/2 and v near -1/2): p = eps_p exp(spread U(-1,1)), 1 - q = eps_q exp(spread U(-1,1)),
    drawn p then q from PCG64(seed).  flip = True exchanges the roles (p near 1, q near 0,
    v near +1/2).  Returns (u, v) in the shape of one field."""
    rng = np.random.default_rng(seed)
    a = eps_p * np.exp(spread * rng.uniform(-1.0, 1.0, size=p.shape))
    b = 1.0 - eps_q * np.exp(spread * rng.uniform(-1.0, 1.0, size=p.shape))
    pp, qq = (1.0 - a, 1.0 - b) if flip else (a, b)
    return np.ascontiguousarray(0.5 * (pp + qq)), np.ascontiguousarray(0.5 * (pp - qq))


def random_vector(p: Params, seed: int):
    """A seeded direction (wu, wv) with entries U(-1,1)."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(-1.0, 1.0, size=(2,) + p.shape)
    return np.ascontiguousarray(w[0]), np.ascontiguousarray(w[1])


def sinusoidal_fields(p: Params):
    """The smooth initial state of the paper's 2D convergence test (Sec. 4.1 A):
    u = 0.4 (sin^2(2 pi x) + cos^2(2 pi y)) + 0.1, v = 0.4 (sin^2(2 pi x) - cos^2(2 pi y)),
    at the cell centres x_i = (i + 1/2) dx, y_j = (j + 1/2) dy."""
    nx, ny = p.n[0], p.n[1]
    x = (np.arange(nx) + 0.5) * (p.L[0] / nx)
    y = (np.arange(ny) + 0.5) * (p.L[1] / ny)
    sx = np.sin(2.0 * np.pi * x)[None, :] ** 2
    cy = np.cos(2.0 * np.pi * y)[:, None] ** 2
    return np.ascontiguousarray(0.4 * (sx + cy) + 0.1), np.ascontiguousarray(0.4 * (sx - cy))


# Coefficients and solver tolerances of the paper's numerical section (Sec. 4: S = 10,
# eps_r = 1e-6, eps_a = 1e-13, xi_r = 1e-8, xi_a = 1e-14; Sec. 4.1: alpha = 4, beta = 2,
# gamma = 0.005, theta = 0.1, rho = 0.001).
PAPER_COEF = dict(alpha=4.0, beta=2.0, gamma=0.005, theta=0.1, rho=0.001, taylor_S=10)
PAPER_TOL = dict(newton_rtol=1e-6, newton_atol=1e-13, gmres_rtol=1e-8, gmres_atol=1e-14)


@dataclass
class Workload:
    name: str
    params: Params
    steps: int
    seed: int
    u_mean: float
    amp: float

    def fields(self):
        return initial_fields(self.params, self.seed, self.u_mean, self.amp)


_COEF = dict(alpha=3.0, beta=1.0, theta=0.3, gamma=1e-3, rho=1.0)

# 2D 64x64 periodic, FP64, fixed dt=1e-3, 10 steps, RAS 4x4 overlap 1, ILU(0).
C1 = Workload(
    "2d-64x64-periodic-fp64-fixed-dt1e-3",
    Params(dim=2, n=(64, 64, 1), bc=BC_PERIODIC, dt_mode=DT_FIXED, dt0=1e-3,
           ras_parts=(4, 4, 1), ras_overlap=1, **_COEF),
    steps=10, seed=0, u_mean=0.5, amp=0.01)

# The 1024^2 and 2048^2 workloads keep the mesh spacing of the 64^2 unit-square
# workload, h = 1/64, so their domains are [0, N/64]^2.  (On the unit square the
# radius-2 operator at h = 1/1024 or 1/2048 is so stiff at every allowed dt that
# natural-order ILU(0) of the 68^2 / 132^2 subdomain boxes amplifies by 1e11-1e17
# and GMRES stagnates; those variants are kept below as *_UNIT for reference.)
H64 = 1.0 / 64.0

# 2D 1024x1024 periodic, FP64, adaptive dt from 1e-4 in [1e-5, 1e-1], 100 steps,
# RAS 16x16 overlap 2, ILU(0).
C2 = Workload(
    "2d-1024x1024-periodic-fp64-adaptive",
    Params(dim=2, n=(1024, 1024, 1), L=(1024 * H64, 1024 * H64, 1.0), bc=BC_PERIODIC,
           dt_mode=DT_ADAPTIVE, dt0=1e-4,
           dt_min=1e-5, dt_max=1e-1, eta0=1e4, ras_parts=(16, 16, 1), ras_overlap=2,
           **_COEF),
    steps=100, seed=1, u_mean=0.4, amp=0.05)

# 2D 2048x2048 periodic, mixed precision (FP32 Krylov / Jacobian / RAS-ILU), adaptive,
# 50 steps, RAS 17x17 overlap 2: boxes of 124-125 cells per direction, whose wavefront levels
# hold at most 63 cells (four warps of two threads per cell), 289 boxes for 152 SMs (measured
# fastest for the FP64 and the mixed form together among 16..32 boxes per direction).
C3 = Workload(
    "2d-2048x2048-periodic-mixed-adaptive",
    Params(dim=2, n=(2048, 2048, 1), L=(2048 * H64, 2048 * H64, 1.0), bc=BC_PERIODIC,
           dt_mode=DT_ADAPTIVE, dt0=1e-4,
           dt_min=1e-5, dt_max=1e-1, eta0=1e4, ras_parts=(17, 17, 1), ras_overlap=2,
           precision=PREC_MIXED, **_COEF),
    steps=50, seed=2, u_mean=0.4, amp=0.05)

# 3D 128^3 homogeneous Neumann on the unit cube (the paper's 3D test, Sec. 4.1 B), FP64
# residual with FP32 Krylov / Jacobian / ILU, RAS 8x8x8 overlap 1 (boxes truncated at the
# walls), adaptive dt from 1e-4 in [1e-5, 1e-1], seed 3, initial state as the 2D runs.
C4 = Workload(
    "3d-128x128x128-neumann-mixed-adaptive",
    Params(dim=3, n=(128, 128, 128), L=(1.0, 1.0, 1.0), bc=BC_NEUMANN, dt_mode=DT_ADAPTIVE, dt0=1e-4,
           dt_min=1e-5, dt_max=1e-1, eta0=100.0, ras_parts=(8, 8, 8), ras_overlap=1,
           precision=PREC_MIXED, **_COEF),
    steps=50, seed=3, u_mean=0.4, amp=0.05)
C4_FP64 = Workload("3d-128x128x128-neumann-fp64-adaptive", C4.params.replace(precision=PREC_FP64),
                   steps=50, seed=3, u_mean=0.4, amp=0.05)

# Unit-square variants of C2 and C3 (see the note above H64).
C2_UNIT = Workload("2d-1024x1024-unit-square-periodic-fp64-adaptive",
                   C2.params.replace(L=(1.0, 1.0, 1.0)), steps=100, seed=1, u_mean=0.4, amp=0.05)
C3_UNIT = Workload("2d-2048x2048-unit-square-periodic-mixed-adaptive",
                   C3.params.replace(L=(1.0, 1.0, 1.0)), steps=50, seed=2, u_mean=0.4, amp=0.05)

# C3 in FP64, the reference point of the mixed-precision speed-up.
C3_FP64 = Workload("2d-2048x2048-periodic-fp64-adaptive", C3.params.replace(precision=PREC_FP64),
                   steps=50, seed=2, u_mean=0.4, amp=0.05)



@dataclass
class EnsembleWorkload(Workload):
    """B independent members of one grid: member m starts from
    initial_fields(seed * 1000 + m) and has theta_m = lo + (hi - lo) * U(0, 1), the B
    values drawn from PCG64(seed); the other coefficients are shared."""

    theta_range: Tuple[float, float] = (0.25, 0.35)

    @property
    def members(self) -> int:
        return self.params.batch

    def member_params(self, m: int) -> Params:
        return self.params.replace(batch=1, theta=float(self.thetas()[m]))

    def thetas(self) -> np.ndarray:
        lo, hi = self.theta_range
        return lo + (hi - lo) * np.random.default_rng(self.seed).uniform(0.0, 1.0, size=self.members)

    def member_fields(self, m: int):
        one = self.params.replace(batch=1)
        return initial_fields(one, self.seed * 1000 + m, self.u_mean, self.amp)

    def fields(self):
        """(u, v) of shape (B,) + grid shape, member-major."""
        us, vs = zip(*(self.member_fields(m) for m in range(self.members)))
        return np.ascontiguousarray(np.stack(us)), np.ascontiguousarray(np.stack(vs))


# 32 members of 256^2 periodic (h = 1/64, so [0, 4]^2), theta ~ U(0.25, 0.35) per member,
# FP64 residual with FP32 Krylov / Jacobian / ILU, adaptive dt from 1e-4.  RAS 3x3 boxes
# (85-86 owned cells per direction) with overlap 1: the partition acac_autotune picks for the
# whole ensemble, all members solved in lockstep.
E32 = EnsembleWorkload(
    "2d-ensemble-32x256x256-periodic-mixed-adaptive",
    Params(dim=2, n=(256, 256, 1), L=(256 * H64, 256 * H64, 1.0), bc=BC_PERIODIC, dt_mode=DT_ADAPTIVE,
           dt0=1e-4, dt_min=1e-5, dt_max=1e-1, eta0=1e4, ras_parts=(3, 3, 1), ras_overlap=1,
           precision=PREC_MIXED, batch=32, **_COEF),
    steps=50, seed=3, u_mean=0.4, amp=0.05)



@dataclass
class AdjointWorkload(Workload):
    """K fixed-dt steps from initial_fields(seed), then the loss
    L = w_energy E~(U^K) + (w_misfit/2) sum |U^K - U*|^2 dx dy against the target
    U* = initial_fields(target_seed) (same mean and amplitude); checkpoint every
    `every` steps."""

    target_seed: int = 0
    every: int = 5
    w_energy: float = 1.0
    w_misfit: float = 1.0

    def target(self):
        return initial_fields(self.params, self.target_seed, self.u_mean, self.amp)


# 2D 512x512 periodic, FP64, 20 steps at dt = 1e-3, checkpoint every 5; loss = final
# energy + misfit to the seeded target; gradients in u0, v0, alpha..gamma.  Mesh spacing
# h = 1/64 as the other large workloads ([0, 8]^2): on the unit square the forward GMRES
# stagnates at the first step (the same ILU(0) instability as the *_UNIT workloads).
C5 = AdjointWorkload(
    "2d-512x512-periodic-fp64-adjoint",
    Params(dim=2, n=(512, 512, 1), L=(512 * H64, 512 * H64, 1.0), bc=BC_PERIODIC, dt_mode=DT_FIXED, dt0=1e-3,
           ras_parts=(8, 8, 1), ras_overlap=1, **_COEF),
    steps=20, seed=4, u_mean=0.4, amp=0.05, target_seed=104, every=5)

WORKLOADS = {w.name: w for w in (C1, C2, C3, C3_FP64, C4, C4_FP64, C2_UNIT, C3_UNIT, E32, C5)}
