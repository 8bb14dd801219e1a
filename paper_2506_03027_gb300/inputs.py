"""Seeded synthetic inputs shared by the CUDA library's callers and the oracle.

This module holds the case descriptions (grid, decomposition, scheme, algorithm), the analytic
initial conditions of the paper's test problems and the seeded SAA delay tables.  It contains none
of the solver's arithmetic: no fluxes, derivatives, RK stages or AT weights.

Initial conditions:
  * Taylor-Green vortex, Sec. 5.2 (Eq. 17): u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
    p = 1/(gamma M^2) + (cos 2x + cos 2y)(cos 2z + 2)/16, isothermal T = 1 so rho = gamma M^2 p.
    The sign of v is the divergence-free one of the cited references (the printed v lacks it).
  * Isentropic vortex (Sec. 5.1 family): the exact translating Euler vortex of strength eps in the
    free-stream scaling u_inf = rho_inf = T_inf = 1, p_inf = 1/(gamma M^2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NV = 5


@dataclasses.dataclass
class Case:
    """One run description.  Lengths are the periodic box sizes; dx = L/n."""
    name: str = "case"
    nx: int = 32
    ny: int = 32
    nz: int = 1
    px: int = 1
    py: int = 1
    pz: int = 1
    lx: float = 2 * math.pi
    ly: float = 2 * math.pi
    lz: float = 2 * math.pi
    gamma: float = 1.4
    mach: float = 0.1
    re: float = 1600.0
    pr: float = 0.71
    viscous: bool = True
    visc_law: int = 0          # 0: mu = 1, 1: mu = T**visc_exp
    visc_exp: float = 0.76
    order: int = 4             # 4: LSERK4-CD4-AT4, 2: LSERK2-CD2-AT2 (Table 1)
    algo: str = "SA"           # SA | CAA | SAA (Alg. 1-3)
    at: bool = True            # True: AT schemes; False: AS (standard stencils on delayed data)
    caa_L: int = 4             # CAA maximum allowable delay L
    kmax: int = 0              # SAA: largest delay of the table
    filter: bool = False
    alpha_f: float = 0.499
    dt: float = 1e-3
    seed: int = 2506030
    curv: float = 0.0          # amplitude of the periodic curvilinear grid (0: uniform Cartesian)

    @property
    def dx(self) -> float:
        return self.lx / self.nx

    @property
    def dy(self) -> float:
        return self.ly / self.ny

    @property
    def dz(self) -> float:
        return self.lz / self.nz

    @property
    def nsub(self) -> int:
        return self.px * self.py * self.pz

    @property
    def npts(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def stages(self) -> int:
        return 5 if self.order == 4 else 2

    @property
    def levels(self) -> int:
        return 5 if self.order == 4 else 3

    def replace(self, **kw) -> "Case":
        return dataclasses.replace(self, **kw)


def grid(case: Case):
    """Cell-vertex coordinates x_i = x0 + i dx (periodic box starting at x0)."""
    if case.name.startswith("vortex"):
        x0 = -case.lx / 2
        y0 = -case.ly / 2
    else:
        x0 = y0 = 0.0
    x = x0 + case.dx * np.arange(case.nx)
    y = y0 + case.dy * np.arange(case.ny)
    z = case.dz * np.arange(case.nz)
    return x, y, z


def grid_xy(case: Case):
    """Point coordinates of the periodic curvilinear grid of amplitude A = case.curv:
    x = x0 + i dx + A sin(2 pi j / ny), y = y0 + j dy + A sin(2 pi i / nx), z = k dz (a smooth
    mapping of the index space (xi, eta) = (i, j), extruded in z).  Returns (xy [2][ny][nx],
    shift[4]) with shift = the (x, y) jump across the periodic wrap in i, then in j; or None
    for the uniform Cartesian grid."""
    if not case.curv:
        return None
    x, y, _ = grid(case)
    jj, ii = np.meshgrid(np.arange(case.ny), np.arange(case.nx), indexing="ij")
    X = x[ii] + case.curv * np.sin(2 * math.pi * jj / case.ny)
    Y = y[jj] + case.curv * np.sin(2 * math.pi * ii / case.nx)
    xy = np.ascontiguousarray(np.stack([X, Y]), dtype=np.float64)
    shift = np.array([case.lx, 0.0, 0.0, case.ly], dtype=np.float64)
    return xy, shift


def point_coords(case: Case):
    """X, Y, Z of every grid point, each [nz][ny][nx]."""
    x, y, z = grid(case)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    g = grid_xy(case)
    if g is not None:
        X = np.broadcast_to(g[0][0], X.shape).copy()
        Y = np.broadcast_to(g[0][1], Y.shape).copy()
    return X, Y, Z


def conserved(case: Case, rho, u, v, w, p) -> np.ndarray:
    """Pack primitive fields into U[5][nz][ny][nx] using p = rho T/(gamma M^2) and
    rho E_t = p/(gamma-1) + rho |u|^2 / 2 (App. A)."""
    U = np.empty((NV, case.nz, case.ny, case.nx), dtype=np.float64)
    U[0] = rho
    U[1] = rho * u
    U[2] = rho * v
    U[3] = rho * w
    U[4] = p / (case.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return U


def tgv_primitives(case: Case):
    X, Y, Z = point_coords(case)
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    gm2 = case.gamma * case.mach ** 2
    p = 1.0 / gm2 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    rho = gm2 * p  # T = 1
    return rho, u, v, w, p


def tgv_state(case: Case) -> np.ndarray:
    """Taylor-Green vortex initial condition (Sec. 5.2)."""
    return conserved(case, *tgv_primitives(case))


def vortex_primitives(case: Case, eps: float = 5.0, t: float = 0.0):
    """Isentropic vortex of strength eps centred at the origin at t = 0, translated by u_inf t = t
    (periodic wrap) at time t.  Exact for the Euler equations on the infinite plane."""
    X, Y, _ = point_coords(case)
    X, Y = X[0], Y[0]
    # position relative to the translated centre, wrapped into the periodic box
    xr = X - t
    xr = (xr + case.lx / 2) % case.lx - case.lx / 2
    yr = (Y + case.ly / 2) % case.ly - case.ly / 2
    r2 = xr * xr + yr * yr
    g = case.gamma
    f = np.exp(0.5 * (1.0 - r2))
    du = -(eps / (2 * math.pi)) * yr * f
    dv = (eps / (2 * math.pi)) * xr * f
    T = 1.0 - (g - 1.0) * eps * eps / (8.0 * g * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (g - 1.0))
    scale = 1.0 / (case.mach * math.sqrt(g))
    u = 1.0 + du * scale
    v = dv * scale
    p = rho * T / (g * case.mach ** 2)
    shape = (case.nz, case.ny, case.nx)
    return (rho.reshape(shape), u.reshape(shape), v.reshape(shape), np.zeros(shape), p.reshape(shape))


def vortex_state(case: Case, eps: float = 5.0, t: float = 0.0) -> np.ndarray:
    return conserved(case, *vortex_primitives(case, eps, t))


def cfl_dt(case: Case, U: np.ndarray, cfl: float = 0.5) -> float:
    """Fixed step from the initial condition: dt = CFL / max sum_d (|u_d| + c)/dx_d with
    c^2 = T/M^2 (nondimensional speed of sound)."""
    rho = U[0]
    u = U[1] / rho
    v = U[2] / rho
    w = U[3] / rho
    p = (case.gamma - 1.0) * (U[4] - 0.5 * rho * (u * u + v * v + w * w))
    c = np.sqrt(case.gamma * p / rho)
    s = (np.abs(u) + c) / case.dx + (np.abs(v) + c) / case.dy
    if case.nz > 1:
        s = s + (np.abs(w) + c) / case.dz
    return float(cfl / s.max())


def saa_delays(case: Case, nsteps: int, kmax: int | None = None, seed: int | None = None) -> np.ndarray:
    """Seeded SAA delay table int8[nsteps][nsub][6] (faces -x,+x,-y,+y,-z,+z), i.i.d. uniform on
    {0..kmax} per (step, sub-domain, face), drawn with numpy's PCG64 from ``seed``."""
    kmax = case.kmax if kmax is None else kmax
    seed = case.seed if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, kmax + 1, size=(nsteps, case.nsub, 6), dtype=np.int8)


# ---------------------------------------------------------------- the paper-shaped workloads

def vortex_case(n: int = 64, p: int = 2, **kw) -> Case:
    """2-D isentropic vortex, Euler, gamma 1.4, strength 5, Mach 0.5, periodic [-5,5]^2, n x n,
    p x p sub-domains, synchronous halos, LSERK4-CD4 (Table 1 case 4)."""
    c = Case(name="vortex", nx=n, ny=n, nz=1, px=p, py=p, pz=1, lx=10.0, ly=10.0, lz=1.0,
             mach=0.5, viscous=False, order=4, algo="SA", filter=False)
    c = c.replace(**kw)
    c.dt = cfl_dt(c, vortex_state(c), 0.5) if "dt" not in kw else kw["dt"]
    return c


def tgv_case(n: int = 128, p: int = 4, algo: str = "SA", **kw) -> Case:
    """3-D Taylor-Green vortex, Navier-Stokes, Re 1600, Mach 0.1, gamma 1.4, Pr 0.71, periodic
    [0, 2 pi]^3, n^3, p^3 sub-domains, LSERK4-CD4-AT4, tenth-order filter alpha_f = 0.499."""
    kmax = {"SA": 0, "CAA": 3, "SAA": 3}[algo]
    c = Case(name="tgv", nx=n, ny=n, nz=n, px=p, py=p, pz=p, mach=0.1, re=1600.0, pr=0.71,
             viscous=True, order=4, algo=algo, caa_L=4, kmax=kmax, filter=True, alpha_f=0.499)
    c = c.replace(**kw)
    if "dt" not in kw:
        c.dt = cfl_dt(c, tgv_state(c), 0.5)
    return c


def initial_state(case: Case) -> np.ndarray:
    if case.name.startswith("vortex"):
        return vortex_state(case)
    return tgv_state(case)
