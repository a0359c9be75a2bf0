"""CPU FP64 oracle for the per-time-step Newton–Krylov–Schwarz solve of the
energy-stable DVD scheme for the coupled Allen–Cahn/Cahn–Hilliard system
(Huang, Yang & Wei, "Parallel energy-stable solver for a coupled Allen–Cahn and
Cahn–Hilliard system", arXiv 2007.04560).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline / reference leg may import or run anything in this package.  The
CUDA library shares no code with it.

Everything is plain NumPy / SciPy in float64 and follows the paper's definitions
in the paper's order; library primitives (sparse products, a dense solve, a
triangular solve) serve as steps.  The subdomain ILU(0) is the plain C routine in
ilu0.c.  Where the paper is silent or garbled the reading taken is stated at the
function that uses it:

  * Lemma 2.2 / Eq. (D2-1): the printed phi^S = f_S(zeta,sigma)+f_S(1-zeta,-sigma)
    is wrong in sign; the series of [Phi(z+s)-Phi(z-s)]/(2s) is
    ln(z/(1-z)) - sum_k [(s/z)^{2k} - (s/(1-z))^{2k}] / (2k(2k+1)).
  * The mobility inside A~ is evaluated at the midpoint state (U1+U0)/2, so that
    the scheme is second order in time (Sec. 2, "trapezoidal rule at the
    half-time level"); an explicit-in-time variant is kept for the order test.
  * The series is always used with S terms (Sec. 4: S = 10).
  * GMRES stops on its Arnoldi residual estimate; restart 30; classical
    Gram–Schmidt with one re-orthogonalisation pass (CGS2).
  * Line search: lambda = 1, halving, Armijo factor 1e-4 on ||F||^2, trial point
    must lie in the admissible set; failure below lambda = 2^-10.
  * Mass: the Newton direction is shifted by a constant in its u part so that the
    full step restores sum(u) = sum(u^n), which the exact Newton step does.
  * RAS subdomains: boxes of near-equal size (the first N mod P boxes one cell
    larger), extended by delta mesh layers (wrapped when periodic, clipped at
    Neumann walls); each subdomain matrix is ordered lexicographically in the
    box's own coordinates, x fastest, u before v; ILU(0) is taken on the full
    2x2-block pattern of the radius-2 stencil.
  * Subdomain solvers of Sec. 4.2 (Table 2): ILU(1) and ILU(2) keep the entries
    whose level of fill is at most 1 or 2 (the usual recursive definition, in the
    same natural order) and run the same elimination on that pattern; LU is the
    exact solve with A_k.

Parity pins for every function live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg
import scipy.sparse as sp
from scipy.special import xlogy

OK = 0
E_ARG = -1
E_DOMAIN = -3
E_DIVERGED = -4
E_DT_UNDERFLOW = -5

BC_PERIODIC = 0
BC_NEUMANN = 1
SUB_ILU0, SUB_ILU1, SUB_ILU2, SUB_LU = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


# --------------------------------------------------------------------------- C part
def build_lib(force: bool = False) -> str:
    """Compile ilu0.c into oracle/_ilu0.so with gcc (plain C, no GPU)."""
    so = os.path.join(_HERE, "_ilu0.so")
    src = os.path.join(_HERE, "ilu0.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build_lib())
        ip = ctypes.POINTER(ctypes.c_int)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_ilu0_factor.argtypes = [ctypes.c_int, ip, ip, dp, ip]
        lib.oracle_ilu0_factor.restype = ctypes.c_int
        lib.oracle_ilu0_solve.argtypes = [ctypes.c_int, ip, ip, dp, ip, dp, dp]
        lib.oracle_ilu0_solve.restype = None
        _LIB = lib
    return _LIB


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------- grid
class Grid:
    """Cell-centred uniform mesh (Sec. 2): x_i = (i-1/2)dx, dx = Lx/Nx, and the
    difference operators of Sec. 2 as sparse matrices on the flattened field
    (C order, x fastest).  Direction d = 0, 1, 2 is x, y, z.

    Per direction: Df (faces x cells) gives phi_{i+1} - phi_i on every face,
    Af gives (phi_i + phi_{i+1})/2 on every face, Dv = -Df^T maps a face flux to
    flux_{i+1/2} - flux_{i-1/2}.  Periodic: N faces (wrapping).  Homogeneous
    Neumann: the N-1 interior faces only, i.e. zero flux through the wall, which
    is the ghost rule phi_0 = phi_1, phi_{N+1} = phi_N of Sec. 2.
    """

    def __init__(self, p):
        self.p = p
        self.dim = p.dim
        self.shape = p.shape
        self.N = int(np.prod(self.shape))
        self.h = [p.L[d] / p.n[d] for d in range(p.dim)]
        self.periodic = p.bc == BC_PERIODIC
        self.Df, self.Af, self.Dv = [], [], []
        for d in range(p.dim):
            df1, af1 = self._ops1(p.n[d])
            self.Df.append(self._embed(df1, d))
            self.Af.append(self._embed(af1, d))
            self.Dv.append(self._embed(-df1.T.tocsr(), d))
        # discrete Laplacian  Delta = sum_d D_d D_d  (Sec. 2, [Delta phi] = [div grad phi])
        lap = sp.csr_matrix((self.N, self.N))
        for d in range(p.dim):
            lap = lap + self.Dv[d] @ self.Df[d] / self.h[d] ** 2
        self.Lap = lap.tocsr()

    def _ops1(self, n):
        if self.periodic:
            i = np.arange(n)
            df = sp.csr_matrix((np.r_[-np.ones(n), np.ones(n)],
                                (np.r_[i, i], np.r_[i, (i + 1) % n])), shape=(n, n))
            af = sp.csr_matrix((np.full(2 * n, 0.5),
                                (np.r_[i, i], np.r_[i, (i + 1) % n])), shape=(n, n))
        else:
            i = np.arange(n - 1)
            df = sp.csr_matrix((np.r_[-np.ones(n - 1), np.ones(n - 1)],
                                (np.r_[i, i], np.r_[i, i + 1])), shape=(n - 1, n))
            af = sp.csr_matrix((np.full(2 * (n - 1), 0.5),
                                (np.r_[i, i], np.r_[i, i + 1])), shape=(n - 1, n))
        return df, af

    def _embed(self, op1, d):
        """Apply a 1D operator along direction d of the C-ordered field."""
        axis = self.dim - 1 - d
        out = None
        for a in range(self.dim):
            f = op1 if a == axis else sp.identity(self.shape[a], format="csr")
            out = f if out is None else sp.kron(out, f, format="csr")
        return out.tocsr()

    # field-level helpers (arrays of self.shape)
    def lap(self, phi):
        return (self.Lap @ phi.ravel()).reshape(self.shape)

    def mob_div(self, c, G):
        """[D_x c~ D_x G] + [D_y c~ D_y G] (+ z): face mobility c~ = (c_i + c_{i+1})/2."""
        out = np.zeros(self.N)
        cf, gf = c.ravel(), G.ravel()
        for d in range(self.dim):
            flux = (self.Af[d] @ cf) * (self.Df[d] @ gf) / self.h[d]
            out += self.Dv[d] @ flux / self.h[d]
        return out.reshape(self.shape)

    @property
    def cell_volume(self):
        return float(np.prod(self.h))


_GRIDS = {}


def grid_for(p) -> Grid:
    key = (p.dim, tuple(p.n), tuple(p.L), p.bc)
    g = _GRIDS.get(key)
    if g is None:
        if len(_GRIDS) > 8:
            _GRIDS.clear()
        g = _GRIDS[key] = Grid(p)
    return g


# --------------------------------------------------------------------------- model
def mobility(u, v):
    """c(u, v) = u(1-u)(1/4 - v^2)  (Sec. 1, after Eq. 1)."""
    return u * (1.0 - u) * (0.25 - v * v)


def Phi(z, omz=None):
    """Phi(z) = z ln z + (1-z) ln(1-z), with 0 ln 0 = 0  (Sec. 1, Eq. 2).  omz: 1 - z when
    the caller has it more accurately than 1.0 - z (near z -> 1)."""
    omz = 1.0 - z if omz is None else omz
    return xlogy(z, z) + xlogy(omz, omz)


def admissible(u, v):
    """u in (0,1), v in (-1/2,1/2), u+v and u-v in (0,1)  (Sec. 2, after Eq. neq:01).
    The last two conditions imply the first two."""
    p, q = u + v, u - v
    return bool(np.all(p > 0.0) and np.all(p < 1.0) and np.all(q > 0.0) and np.all(q < 1.0))


def phi_S(zeta, sigma, S, omz=None):
    """Series form of [Phi(zeta+sigma) - Phi(zeta-sigma)] / (2 sigma)  (Lemma 2.2,
    Eq. D2-1), with the sign of the printed combination corrected:
        ln zeta - ln(1-zeta) - sum_{k=1..S} [(sigma/zeta)^{2k} - (sigma/(1-zeta))^{2k}] / ((2k+1) 2k).
    omz: 1 - zeta as formed by _pq (accurate near zeta -> 1); 1.0 - zeta when not given.
    """
    omz = 1.0 - zeta if omz is None else omz
    a = sigma / zeta
    b = sigma / omz
    out = np.log(zeta) - np.log(omz)
    for k in range(1, S + 1):
        out = out - (a ** (2 * k) - b ** (2 * k)) / ((2 * k + 1) * (2 * k))
    return out


def dphi_S(zeta, sigma, S, omz=None):
    """(d phi^S / d zeta, d phi^S / d sigma), differentiated term by term (omz as in phi_S)."""
    omz = 1.0 - zeta if omz is None else omz
    a = sigma / zeta
    b = sigma / omz
    dz = 1.0 / zeta + 1.0 / omz
    ds = np.zeros_like(zeta * sigma)
    for k in range(1, S + 1):
        dz = dz + (a ** (2 * k) / zeta + b ** (2 * k) / omz) / (2 * k + 1)
        ds = ds - (a ** (2 * k - 1) / zeta - b ** (2 * k - 1) / omz) / (2 * k + 1)
    return dz, ds


def exact_quotient(z1, z0):
    """[Phi(z1) - Phi(z0)] / (z1 - z0)  (Eq. D2); only for |z1 - z0| not tiny."""
    return (Phi(z1) - Phi(z0)) / (z1 - z0)


def _pq(u1, v1, u0, v0):
    """zeta, sigma of p = u+v and q = u-v (Sec. 2, after Eq. D2-1), and 1 - zeta of each:
    (zeta_p, sigma_p, zeta_q, sigma_q, 1 - zeta_p, 1 - zeta_q).

    zeta comes from the end values p1, p0 (each sum of u and v rounds relative to its own
    value); 1 - zeta from the end values 1 - p and 1 - q formed by one_minus_pq, not from
    1.0 - zeta after zeta has been rounded; sigma from the differences of whichever end
    values lie nearer zero (p1 - p0 where zeta < 1/2, (1 - p0) - (1 - p1) above).  Near a pure
    phase (zeta or 1 - zeta -> 0 at the edge of the admissible set) each of them then
    keeps its relative accuracy; 1.0 - zeta would carry an absolute error of ~1e-16, a
    relative error of ~1e-8 at 1 - zeta = 1e-8, and so would the logarithms."""
    p1, p0, q1, q0 = u1 + v1, u0 + v0, u1 - v1, u0 - v0
    mp1, mq1 = one_minus_pq(u1, v1)
    mp0, mq0 = one_minus_pq(u0, v0)
    zp, zq = (p1 + p0) / 2, (q1 + q0) / 2
    # sigma from the end values nearer zero: p1 - p0 below zeta = 1/2, (1 - p0) - (1 - p1) above
    sp_ = np.where(zp < 0.5, p1 - p0, mp0 - mp1) / 2
    sq = np.where(zq < 0.5, q1 - q0, mq0 - mq1) / 2
    return zp, sp_, zq, sq, (mp1 + mp0) / 2, (mq1 + mq0) / 2


def one_minus_pq(u, v):
    """1 - (u + v) and 1 - (u - v), each correctly rounded from the double inputs: 1 - u is
    split into its rounded value s and the rounding error e (s + e = 1 - u exactly, the
    two-sum of 1 and -u), and s -+ v is exact wherever the result is small (s and v then
    lie within a factor 2 of each other), so that only the final addition of e rounds."""
    s = 1.0 - u
    e = -u - (s - 1.0)
    return (s - v) + e, (s + v) + e


def G_tilde(p, g, u1, v1, u0, v0, exact=False):
    """Discrete variational derivative G~^S = G1 + G2^S + G3  (Sec. 2, Eqs. dvds-2,
    D2-1, dvds-1).  exact=True uses the rational G2 of Eq. D2 instead of the series.
    Returns (G_u, G_v)."""
    # G1 from e1 = alpha/2 u(1-u) - beta/2 v^2
    G1u = -0.5 * p.alpha * (u1 + u0 - 1.0)
    G1v = -0.5 * p.beta * (v1 + v0)
    # G2 from e2 = theta (Phi(u+v) + Phi(u-v))
    zp, sp_, zq, sq, omp, omq = _pq(u1, v1, u0, v0)
    if exact:
        phi = exact_quotient(u1 + v1, u0 + v0)
        psi = exact_quotient(u1 - v1, u0 - v0)
    else:
        phi = phi_S(zp, sp_, p.taylor_S, omp)
        psi = phi_S(zq, sq, p.taylor_S, omq)
    G2u = p.theta * (phi + psi)
    G2v = p.theta * (phi - psi)
    # G3 from e3 = gamma/2 (|grad u|^2 + |grad v|^2)
    G3u = -0.5 * p.gamma * (g.lap(u1) + g.lap(u0))
    G3v = -0.5 * p.gamma * (g.lap(v1) + g.lap(v0))
    return G1u + G2u + G3u, G1v + G2v + G3v


def mobility_state(u1, v1, u0, v0, mode="midpoint"):
    """Mobility field used in A~: at the midpoint state (default) or at U^n."""
    if mode == "midpoint":
        return mobility(0.5 * (u1 + u0), 0.5 * (v1 + v0))
    return mobility(u0, v0)


def residual(p, X1, X0, dt, mode="midpoint", g=None):
    """F(X) of scheme NSOA-1:  (U1 - U0)/dt + A~ G~^S = 0  with
    A~ = diag(-div c grad, c/rho)  (Sec. 2, Eqs. system-1, NSOA-1), i.e.
        F_u = (u1 - u0)/dt - [div c~ grad G_u],   F_v = (v1 - v0)/dt + c G_v / rho.
    X1, X0 are (u, v) pairs of arrays of p.shape.  Returns (F_u, F_v)."""
    g = g or grid_for(p)
    u1, v1 = X1
    u0, v0 = X0
    Gu, Gv = G_tilde(p, g, u1, v1, u0, v0)
    c = mobility_state(u1, v1, u0, v0, mode)
    Fu = (u1 - u0) / dt - g.mob_div(c, Gu)
    Fv = (v1 - v0) / dt + c * Gv / p.rho
    return Fu, Fv


def _dplus_dminus(phi, p, d):
    """[D^+ phi], [D^- phi] along direction d with the ghost rule of Sec. 2
    (periodic wrap, or phi_0 = phi_1 and phi_{N+1} = phi_N)."""
    axis = p.dim - 1 - d
    h = p.L[d] / p.n[d]
    if p.bc == BC_PERIODIC:
        nxt = np.roll(phi, -1, axis=axis)
        prv = np.roll(phi, 1, axis=axis)
    else:
        n = phi.shape[axis]
        idx_n = np.minimum(np.arange(n) + 1, n - 1)
        idx_p = np.maximum(np.arange(n) - 1, 0)
        nxt = np.take(phi, idx_n, axis=axis)
        prv = np.take(phi, idx_p, axis=axis)
    return (nxt - phi) / h, (phi - prv) / h


def energy_density(p, u, v):
    """Local discrete energy [e~]_ij of Eq. relations: e1 + e2 + gamma/2 sum_d
    ((D^+ phi)^2 + (D^- phi)^2)/2 for phi = u, v."""
    e = 0.5 * p.alpha * u * (1.0 - u) - 0.5 * p.beta * v * v
    mp, mq = one_minus_pq(u, v)
    e = e + p.theta * (Phi(u + v, mp) + Phi(u - v, mq))
    for phi in (u, v):
        for d in range(p.dim):
            dp, dm = _dplus_dminus(phi, p, d)
            e = e + 0.5 * p.gamma * 0.5 * (dp * dp + dm * dm)
    return e


def energy(p, u, v):
    """Discrete free energy E~ = <[e~]> = sum e~ dx dy (Eq. freeenergy)."""
    vol = float(np.prod([p.L[d] / p.n[d] for d in range(p.dim)]))
    return float(np.sum(energy_density(p, u, v)) * vol)


def mass(p, u):
    """sum u dx dy (dz)."""
    vol = float(np.prod([p.L[d] / p.n[d] for d in range(p.dim)]))
    return float(np.sum(u) * vol)


# --------------------------------------------------------------------------- Jacobian
def stencil_offsets(dim):
    """Offsets of the radius-2 stencil of F: all integer o with |o|_1 <= 2
    (13 in 2D, 25 in 3D), as (dx, dy, dz)."""
    out = []
    r = range(-2, 3)
    for dz in (r if dim == 3 else [0]):
        for dy in r:
            for dx in r:
                if abs(dx) + abs(dy) + abs(dz) <= 2:
                    out.append((dx, dy, dz))
    return out


def _interleave_perm(N):
    """Interleaved unknown index 2c + dof  ->  blocked index dof*N + c (Sec. 3.1:
    X = (u_00, v_00, u_10, v_10, ...))."""
    perm = np.empty(2 * N, dtype=np.int64)
    perm[0::2] = np.arange(N)
    perm[1::2] = N + np.arange(N)
    return perm


def linearization(p, X1, X0, g=None):
    """Per-cell quantities of dF/dX1: c, dc/du1, dc/dv1, G_u, G_v and
    theta*dphi/dp1, theta*dpsi/dq1 (p1 = u1+v1, q1 = u1-v1)."""
    g = g or grid_for(p)
    u1, v1 = X1
    u0, v0 = X0
    ub, vb = 0.5 * (u1 + u0), 0.5 * (v1 + v0)
    c = mobility(ub, vb)
    cu = 0.5 * (1.0 - 2.0 * ub) * (0.25 - vb * vb)     # d c(ub, vb) / d u1
    cv = 0.5 * ub * (1.0 - ub) * (-2.0 * vb)            # d c(ub, vb) / d v1
    Gu, Gv = G_tilde(p, g, u1, v1, u0, v0)
    zp, sp_, zq, sq, omp, omq = _pq(u1, v1, u0, v0)
    dzp, dsp = dphi_S(zp, sp_, p.taylor_S, omp)
    dzq, dsq = dphi_S(zq, sq, p.taylor_S, omq)
    A = p.theta * 0.5 * (dzp + dsp)     # theta d phi / d p1  (zeta, sigma both move by 1/2)
    B = p.theta * 0.5 * (dzq + dsq)     # theta d psi / d q1
    return dict(c=c, cu=cu, cv=cv, Gu=Gu, Gv=Gv, A=A, B=B)


def jacobian_blocks(p, X1, X0, dt, g=None):
    """dF/dX1 as four N x N sparse blocks (Juu, Juv, Jvu, Jvv), by the chain rule
    on residual():  F_u = (u1-u0)/dt - sum_d Dv_d[(Af_d c)(Df_d G_u)/h_d]/h_d and
    F_v = (v1-v0)/dt + c G_v/rho."""
    g = g or grid_for(p)
    lin = linearization(p, X1, X0, g)
    N = g.N
    I = sp.identity(N, format="csr")
    diag = lambda a: sp.diags(np.asarray(a).ravel(), format="csr")
    A, B = lin["A"].ravel(), lin["B"].ravel()
    dGu_du = diag(-0.5 * p.alpha + A + B) - 0.5 * p.gamma * g.Lap
    dGu_dv = diag(A - B)
    dGv_du = diag(A - B)
    dGv_dv = diag(-0.5 * p.beta + A + B) - 0.5 * p.gamma * g.Lap
    c, cu, cv = lin["c"].ravel(), lin["cu"].ravel(), lin["cv"].ravel()
    Gu, Gv = lin["Gu"].ravel(), lin["Gv"].ravel()
    Juu = I / dt
    Juv = sp.csr_matrix((N, N))
    for d in range(p.dim):
        h = g.h[d]
        gradG = diag(g.Df[d] @ Gu / h)          # face gradient of G_u
        cface = diag(g.Af[d] @ c)               # face mobility
        Juu = Juu - g.Dv[d] @ (gradG @ g.Af[d] @ diag(cu) + cface @ g.Df[d] @ dGu_du / h) / h
        Juv = Juv - g.Dv[d] @ (gradG @ g.Af[d] @ diag(cv) + cface @ g.Df[d] @ dGu_dv / h) / h
    Jvu = (diag(Gv * cu) + diag(c) @ dGv_du) / p.rho
    Jvv = I / dt + (diag(Gv * cv) + diag(c) @ dGv_dv) / p.rho
    return Juu.tocsr(), Juv.tocsr(), Jvu.tocsr(), Jvv.tocsr()


def block_pattern(p):
    """CSR pattern (ones) of the full 2x2-block radius-2 stencil in interleaved
    ordering: every (dof, dof') pair of every stencil neighbour inside the domain
    (periodic: wrapped)."""
    shape = p.shape
    N = int(np.prod(shape))
    idx = np.arange(N).reshape(shape)
    rows, cols = [], []
    for (dx, dy, dz) in stencil_offsets(p.dim):
        off = {p.dim - 1: dx, p.dim - 2: dy}
        if p.dim == 3:
            off[0] = dz
        nb = idx
        valid = np.ones(shape, dtype=bool)
        for axis, o in off.items():
            if o == 0:
                continue
            if p.bc == BC_PERIODIC:
                nb = np.roll(nb, -o, axis=axis)
            else:
                n = shape[axis]
                pos = np.arange(n) + o
                ok = (pos >= 0) & (pos < n)
                sl = [None] * p.dim
                sl[axis] = slice(None)
                valid = valid & ok[tuple(sl)]
                nb = np.take(nb, np.clip(pos, 0, n - 1), axis=axis)
        r = idx[valid]
        cc = nb[valid]
        for a in range(2):
            for b in range(2):
                rows.append(2 * r + a)
                cols.append(2 * cc + b)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    pat = sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(2 * N, 2 * N))
    pat.sum_duplicates()
    pat.sort_indices()
    return pat


def jacobian(p, X1, X0, dt, g=None):
    """Assembled Jacobian J = dF/dX1 in the interleaved ordering of Sec. 3.1, stored
    on the full 2x2-block stencil pattern (explicit zeros kept)."""
    g = g or grid_for(p)
    Juu, Juv, Jvu, Jvv = jacobian_blocks(p, X1, X0, dt, g)
    N = g.N
    Jb = sp.bmat([[Juu, Juv], [Jvu, Jvv]], format="csr")
    perm = _interleave_perm(N)
    Ji = Jb[perm][:, perm].tocsr()
    Ji.sum_duplicates()
    Ji.sort_indices()
    pat = block_pattern(p)
    n2 = 2 * N
    kJ = np.repeat(np.arange(n2, dtype=np.int64), np.diff(Ji.indptr)) * n2 + Ji.indices
    kP = np.repeat(np.arange(n2, dtype=np.int64), np.diff(pat.indptr)) * n2 + pat.indices
    pos = np.searchsorted(kP, kJ)
    ok = (pos < kP.size)
    ok[ok] = kP[pos[ok]] == kJ[ok]
    if not np.all(ok | (Ji.data == 0.0)):
        raise AssertionError("Jacobian has entries outside the radius-2 block stencil")
    data = np.zeros(kP.size)
    data[pos[ok]] = Ji.data[ok]
    return sp.csr_matrix((data, pat.indices.copy(), pat.indptr.copy()), shape=(n2, n2))


def interleave(u, v):
    x = np.empty(2 * u.size)
    x[0::2] = u.ravel()
    x[1::2] = v.ravel()
    return x


def deinterleave(x, shape):
    return x[0::2].reshape(shape).copy(), x[1::2].reshape(shape).copy()


# --------------------------------------------------------------------------- Schwarz
@dataclass
class Subdomain:
    cells: np.ndarray      # global cell index of every box cell, local lexicographic order
    owned: np.ndarray      # bool mask over box cells: inside the non-overlapping part
    box: tuple             # box widths (Wx, Wy[, Wz])
    idx: np.ndarray = None         # interleaved unknown indices
    indptr: np.ndarray = None
    indices: np.ndarray = None
    data: np.ndarray = None
    diag: np.ndarray = None


def partition_1d(n, parts):
    """[start, end) of `parts` near-equal boxes; the first n % parts get one extra cell."""
    base, rem = divmod(n, parts)
    out, s = [], 0
    for k in range(parts):
        w = base + (1 if k < rem else 0)
        out.append((s, s + w))
        s += w
    return out


def subdomains(p):
    """Overlapping decomposition Omega = U Omega_k^delta (Sec. 3.1): non-overlapping
    boxes extended by delta mesh layers per direction; periodic boxes wrap, Neumann
    boxes are clipped at the wall.  Subdomains ordered x fastest."""
    dim, d = p.dim, p.ras_overlap
    ranges = []
    for a in range(dim):
        n, P = p.n[a], p.ras_parts[a]
        if P < 1 or P > n:
            raise ValueError("bad ras_parts")
        rs = []
        for (s, e) in partition_1d(n, P):
            if p.bc == BC_PERIODIC:
                lo, hi = s - d, e + d
                if P < 2 or hi - lo > n - 2:
                    raise ValueError("periodic subdomain box wraps onto itself")
            else:
                lo, hi = max(0, s - d), min(n, e + d)
            coords = np.arange(lo, hi) % n
            own = (np.arange(lo, hi) >= s) & (np.arange(lo, hi) < e)
            rs.append((coords, own))
        ranges.append(rs)
    shape = p.shape
    out = []
    parts = list(p.ras_parts[:dim])
    for kz in range(parts[2] if dim == 3 else 1):
        for ky in range(parts[1]):
            for kx in range(parts[0]):
                cx, ox = ranges[0][kx]
                cy, oy = ranges[1][ky]
                if dim == 2:
                    cells = (cy[:, None] * shape[1] + cx[None, :]).ravel()
                    own = (oy[:, None] & ox[None, :]).ravel()
                    box = (cx.size, cy.size)
                else:
                    cz, oz = ranges[2][kz]
                    cells = ((cz[:, None, None] * shape[1] + cy[None, :, None]) * shape[2]
                             + cx[None, None, :]).ravel()
                    own = (oz[:, None, None] & oy[None, :, None] & ox[None, None, :]).ravel()
                    box = (cx.size, cy.size, cz.size)
                out.append(Subdomain(cells=cells, owned=own, box=box))
    return out


def fill_levels(indptr, indices, p=None):
    """Pattern of ILU(p) for a sparse matrix given by its CSR pattern (sorted rows):
    entries of A have level 0; eliminating row i in natural order, every entry
    (i, k) left of the diagonal whose level is at most p, taken in increasing k,
    gives the entries (i, j), j > k, of the upper part of row k the candidate level
    lev(i, k) + lev(k, j) + 1, and lev(i, j) is the smallest candidate (Sec. 4.2,
    "ILU factorizations with 0, 1 and 2 levels of fill-in").  Entries of level
    <= p are kept; p = None keeps every fill entry (the pattern of LU).  Returns
    (indptr, indices, levels) of the kept pattern, rows sorted."""
    import heapq
    n = len(indptr) - 1
    cap = math.inf if p is None else p
    rows = []                  # final {column: level} of each row
    for i in range(n):
        lev = {int(j): 0 for j in indices[indptr[i]:indptr[i + 1]]}
        heap = [j for j in lev if j < i]
        heapq.heapify(heap)
        done = set()
        while heap:
            k = heapq.heappop(heap)
            if k in done:
                continue
            done.add(k)
            lik = lev[k]
            for j, lkj in rows[k].items():
                if j <= k:
                    continue
                cand = lik + lkj + 1
                if cand > cap:
                    continue
                if j not in lev or cand < lev[j]:
                    lev[j] = cand
                    if j < i and j not in done:
                        heapq.heappush(heap, j)
        rows.append(lev)
    out_ptr = np.zeros(n + 1, dtype=np.int64)
    cols, levs = [], []
    for i, lev in enumerate(rows):
        js = sorted(lev)
        cols.extend(js)
        levs.extend(lev[j] for j in js)
        out_ptr[i + 1] = len(cols)
    return out_ptr, np.asarray(cols, dtype=np.int64), np.asarray(levs, dtype=np.int64)


def ilu_factor(A, p=0):
    """ILU(p) of the CSR matrix A in natural order: the IKJ elimination of ilu0.c on
    the pattern of fill_levels(A, p) (A's values there, explicit zeros at the fill
    entries).  Returns the factors as a CSR matrix (L strictly below the diagonal
    with unit diagonal implied, U on and above) and the diagonal positions."""
    A = A.tocsr()
    A.sort_indices()
    if p == 0:
        ip, ind = A.indptr.astype(np.int64), A.indices.astype(np.int64)
    else:
        ip, ind, _ = fill_levels(A.indptr, A.indices, p)
    n = A.shape[0]
    data = np.zeros(ind.size)
    for i in range(n):
        cols = ind[ip[i]:ip[i + 1]]
        a_cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        pos = np.searchsorted(cols, a_cols)
        data[ip[i] + pos] = A.data[A.indptr[i]:A.indptr[i + 1]]
    F = sp.csr_matrix((data, ind.astype(np.int32), ip.astype(np.int32)), shape=A.shape)
    indptr = F.indptr.astype(np.int32)
    indices = F.indices.astype(np.int32)
    vals = F.data.astype(np.float64).copy()
    diag = np.zeros(n, dtype=np.int32)
    st = _lib().oracle_ilu0_factor(n, _iptr(indptr), _iptr(indices), _dptr(vals), _iptr(diag))
    if st != 0:
        raise ZeroDivisionError("ILU(%d) pivot breakdown (status %d)" % (p, st))
    return sp.csr_matrix((vals, indices, indptr), shape=A.shape), diag


class RAS:
    """Schwarz preconditioner of Eq. invM with ILU(0), ILU(1), ILU(2) or exact LU
    subdomain solves (p.subdomain_solver, Sec. 4.2 Table 2).
    kind: 'left' = restricted extension  sum_k R_k^0T inv(A_k) R_k^delta,
          'as'   = classical              sum_k R_k^dT inv(A_k) R_k^delta,
          'right'= restricted restriction sum_k R_k^dT inv(A_k) R_k^0."""

    def __init__(self, p, J, kind="left"):
        self.kind = kind
        self.solver = getattr(p, "subdomain_solver", SUB_ILU0)
        self.subs = subdomains(p)
        for s in self.subs:
            s.idx = np.empty(2 * s.cells.size, dtype=np.int64)
            s.idx[0::2] = 2 * s.cells
            s.idx[1::2] = 2 * s.cells + 1
            A = J[s.idx][:, s.idx].tocsr()       # A_k = R_k J R_k^T
            A.sort_indices()
            if self.solver == SUB_LU:
                s.lu = scipy.linalg.lu_factor(A.toarray())
                continue
            F, s.diag = ilu_factor(A, self.solver)
            s.indptr, s.indices, s.data = F.indptr, F.indices, F.data

    def solve_local(self, s, b):
        if getattr(s, "lu", None) is not None:      # exact LU of this subdomain
            return scipy.linalg.lu_solve(s.lu, b)
        x = np.zeros_like(b)
        _lib().oracle_ilu0_solve(b.size, _iptr(s.indptr), _iptr(s.indices), _dptr(s.data),
                                 _iptr(s.diag), _dptr(b), _dptr(x))
        return x

    def apply(self, r):
        z = np.zeros_like(r)
        for s in self.subs:
            own2 = np.repeat(s.owned, 2)
            rk = np.ascontiguousarray(r[s.idx])
            if self.kind == "right":
                rk = np.where(own2, rk, 0.0)
            zk = self.solve_local(s, rk)
            if self.kind == "left":
                z[s.idx[own2]] += zk[own2]
            else:
                np.add.at(z, s.idx, zk)
        return z


# --------------------------------------------------------------------------- GMRES
@dataclass
class GmresResult:
    x: np.ndarray
    its: int
    converged: bool
    resid: float


def gmres(matvec, precond, b, rtol, atol, restart=30, maxit=500, cgs_refine=1):
    """Right-preconditioned restarted GMRES for A x = b, x0 = 0 (Sec. 3.1, Eq.
    hjacobi): builds an Arnoldi basis of A M^-1 with classical Gram–Schmidt
    (repeated once when cgs_refine), Givens rotations on the Hessenberg matrix,
    stops when the residual estimate |g_{j+1}| <= max(rtol ||b||, atol)."""
    n = b.size
    x = np.zeros(n)
    tol = max(rtol * float(np.linalg.norm(b)), atol)
    r = b.copy()
    beta = float(np.linalg.norm(r))
    its = 0
    if beta <= tol:
        return GmresResult(x, 0, True, beta)
    resid = beta
    while True:
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        gv = np.zeros(restart + 1)
        gv[0] = beta
        V[0] = r / beta
        k = 0
        done = False
        for j in range(restart):
            w = matvec(precond(V[j]))
            its += 1
            h = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h
            if cgs_refine:
                h2 = V[: j + 1] @ w
                w = w - V[: j + 1].T @ h2
                h = h + h2
            hn = float(np.linalg.norm(w))
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0.0:
                V[j + 1] = w / hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rho = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / rho
            sn[j] = H[j + 1, j] / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            gv[j + 1] = -sn[j] * gv[j]
            gv[j] = cs[j] * gv[j]
            resid = abs(gv[j + 1])
            k = j + 1
            if resid <= tol or its >= maxit or hn == 0.0:
                done = True
                break
        y = scipy.linalg.solve_triangular(H[:k, :k], gv[:k])
        x = x + precond(V[:k].T @ y)
        if done:
            return GmresResult(x, its, resid <= tol or hn == 0.0, resid)
        r = b - matvec(x)
        beta = float(np.linalg.norm(r))
        if beta <= tol:
            return GmresResult(x, its, True, beta)


# --------------------------------------------------------------------------- Newton
@dataclass
class NewtonInfo:
    status: int = OK
    newton_its: int = 0
    gmres_its: int = 0
    fnorm0: float = 0.0
    fnorm: float = 0.0
    reason: str = ""
    lambdas: list = field(default_factory=list)


def nks_solve(p, U0, dt, linear="nks", mode="midpoint"):
    """Inexact Newton with line search (Sec. 3.1, Eq. newton) for F(X) = 0 of scheme
    NSOA-1, started from X_0 = U^n.  linear = 'nks': GMRES with the Schwarz/ILU(0)
    preconditioner, factored at the first Newton iteration and reused within the
    step when p.ilu_reuse; 'dense': a dense direct solve of J S = -F.
    Stops when ||F(X_{m+1})|| <= max(rtol ||F(X_0)||, atol).  Returns (X, info)."""
    g = grid_for(p)
    shape = p.shape
    u0, v0 = U0
    info = NewtonInfo()
    if not admissible(u0, v0):
        info.status, info.reason = E_DOMAIN, "input outside admissible set"
        return None, info
    X = (u0.copy(), v0.copy())
    F = interleave(*residual(p, X, U0, dt, mode, g))
    fnorm = float(np.linalg.norm(F))
    info.fnorm0 = info.fnorm = fnorm
    stop = max(p.newton_rtol * fnorm, p.newton_atol)
    if fnorm <= stop:
        return X, info
    kind = {0: "left", 1: "as", 2: "right"}[p.ras_type]
    prec = None
    N = g.N
    while True:
        if info.newton_its >= p.newton_maxit:
            info.status, info.reason = E_DIVERGED, "newton maxit"
            return None, info
        J = jacobian(p, X, U0, dt, g)
        if linear == "dense":
            S = np.linalg.solve(J.toarray(), -F)
        else:
            if prec is None or not p.ilu_reuse:
                try:
                    prec = RAS(p, J, kind)
                except ZeroDivisionError:
                    info.status, info.reason = E_DIVERGED, "ilu pivot"
                    return None, info
            res = gmres(lambda w: J @ w, prec.apply, -F, p.gmres_rtol, p.gmres_atol,
                        p.gmres_restart, p.gmres_maxit, p.cgs_refine)
            info.gmres_its += res.its
            if not res.converged:
                info.status, info.reason = E_DIVERGED, "gmres maxit"
                return None, info
            S = res.x
        # mass: shift S_u so that sum(u + S_u) = sum(u^n), as the exact Newton step does
        Su = S[0::2]
        Su += (np.sum(u0) - np.sum(X[0]) - np.sum(Su)) / N
        Su_f, Sv_f = S[0::2].reshape(shape), S[1::2].reshape(shape)
        lam = 1.0
        f2 = fnorm * fnorm
        while True:
            Xt = (X[0] + lam * Su_f, X[1] + lam * Sv_f)
            if admissible(*Xt):
                Ft = interleave(*residual(p, Xt, U0, dt, mode, g))
                ft = float(np.linalg.norm(Ft))
                if np.isfinite(ft) and ft * ft <= (1.0 - 2e-4 * lam) * f2:
                    break
            lam *= 0.5
            if lam < 2.0 ** -10:
                info.status, info.reason = E_DIVERGED, "line search"
                return None, info
        info.lambdas.append(lam)
        X, F, fnorm = Xt, Ft, ft
        info.newton_its += 1
        info.fnorm = fnorm
        if fnorm <= stop:
            return X, info


# --------------------------------------------------------------------------- time stepping
@dataclass
class StepInfo:
    status: int = OK
    t: float = 0.0
    dt: float = 0.0
    eta: float = 0.0
    energy: float = 0.0
    mass: float = 0.0
    fnorm0: float = 0.0
    fnorm: float = 0.0
    newton_its: int = 0
    gmres_its: int = 0
    divergences: int = 0


class Stepper:
    """Adaptive time stepping of Sec. 3.2 (Eq. sencondt) around nks_solve.

    First step: dt0.  Later steps predict
        dt~ = max(dt_min, dt_max / sqrt(1 + eta X_d'^2)),  X_d' = ||X^n - X^{n-1}|| / dt_{n-1}
    (Euclidean norm over all 2N unknowns).  If the NKS solve diverges, dt~ <- dt~/sqrt(2)
    and eta <- 2 eta, and the step is retried; dt~ < dt_min is an error.  With
    dt_mode fixed every step uses dt0 and a divergence is an error."""

    def __init__(self, p, linear="nks", mode="midpoint"):
        self.p = p
        self.linear = linear
        self.mode = mode
        self.t = 0.0
        self.nstep = 0
        self.eta = p.eta0
        self.prev = None
        self.dt_prev = None

    def predict(self, u, v):
        p = self.p
        if p.dt_mode == 0 or self.prev is None:
            return p.dt0
        diff = np.sqrt(np.sum((u - self.prev[0]) ** 2) + np.sum((v - self.prev[1]) ** 2))
        xd = diff / self.dt_prev
        return max(p.dt_min, p.dt_max / math.sqrt(1.0 + self.eta * xd * xd))

    def step(self, u, v):
        p = self.p
        info = StepInfo()
        if not admissible(u, v):
            info.status = E_DOMAIN
            return None, info
        dt = self.predict(u, v)
        while True:
            X, ni = nks_solve(p, (u, v), dt, self.linear, self.mode)
            info.newton_its += ni.newton_its
            info.gmres_its += ni.gmres_its
            info.fnorm0, info.fnorm = ni.fnorm0, ni.fnorm
            if ni.status == OK:
                break
            if ni.status == E_DOMAIN:
                info.status = E_DOMAIN
                return None, info
            info.divergences += 1
            if p.dt_mode == 0:
                info.status = E_DIVERGED
                return None, info
            dt = dt / math.sqrt(2.0)
            self.eta *= 2.0
            if dt < p.dt_min:
                info.status = E_DT_UNDERFLOW
                return None, info
        self.prev = (u.copy(), v.copy())
        self.dt_prev = dt
        self.t += dt
        self.nstep += 1
        info.t, info.dt, info.eta = self.t, dt, self.eta
        info.energy = energy(p, *X)
        info.mass = mass(p, X[0])
        return X, info
