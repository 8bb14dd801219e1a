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
    compact: int = 0           # 1: sixth-order compact derivatives (Eq. 2, alpha = 1/3) for the Euler fluxes

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

def saa_delays_arrival(case: Case, nsteps: int, L: int, p_late: float = 0.6, seed: int | None = None) -> np.ndarray:
    """SAA delays with the time structure of Alg. 3 (int8 [nsteps][nsub][6]): per (sub-domain,
    face) the newest visible level either stays one more step -- the delay grows by one, with
    probability p_late -- or a message arrives and the delay drops to 0; a delay that would reach
    L is reset by the local synchronization Alg. 3 forces.  The visible levels are therefore
    always consecutive, and the delays follow a geometric law truncated at L - 1 (mean about
    p_late / (1 - p_late) = 1.5 for p_late = 0.6: smaller delays more likely, a mean between 1 and
    2 levels, as the measured delay distributions of Sec. 5.3 show)."""
    rng = np.random.default_rng(case.seed if seed is None else seed)
    k = np.zeros((case.nsub, 6), dtype=np.int64)
    out = np.zeros((nsteps, case.nsub, 6), dtype=np.int8)
    for n in range(nsteps):
        late = rng.random((case.nsub, 6)) < p_late
        k = np.where(late & (k + 1 <= L - 1), k + 1, 0)
        out[n] = k
    return out


def vortex_case(n: int = 64, p: int = 2, **kw) -> Case:
    """2-D isentropic vortex, Euler, gamma 1.4, strength 5, Mach 0.5, periodic [-5,5]^2, n x n,
    p x p sub-domains, synchronous halos, LSERK4-CD4 (Table 1 case 4)."""
    c = Case(name="vortex", nx=n, ny=n, nz=1, px=p, py=p, pz=1, lx=10.0, ly=10.0, lz=1.0,
             mach=0.5, viscous=False, order=4, algo="SA", filter=False)
    c = c.replace(**kw)
    c.dt = cfl_dt(c, vortex_state(c), 0.5) if "dt" not in kw else kw["dt"]
    return c


def paper_vortex_case(n: int = 60, order: int = 4, algo: str = "SA", at: bool = True, L: int = 8, **kw) -> Case:
    """The paper's own vortex test (Sec. 5.1): Euler, M = 0.1, periodic [-8, 8]^2 on n x n points,
    three PEs along x, maximum allowable delay L (CAA: delays (n - C) mod L; SAA: 0..L-1), the
    time step 2e-3 (SA) or 1e-3 (CAA, SAA) at n = 60, scaled with the grid spacing."""
    dt = (2e-3 if algo == "SA" else 1e-3) * 60.0 / n
    c = Case(name="vortex_paper", nx=n, ny=n, nz=1, px=3, py=1, pz=1, lx=16.0, ly=16.0, lz=1.0, mach=0.1,
             viscous=False, order=order, algo=algo, at=at, caa_L=L, kmax=L - 1, filter=False, dt=dt)
    return c.replace(**kw)


def paper_vortex_state(case: Case, t: float = 0.0, beta: float = 0.02, R: float = 1.0) -> np.ndarray:
    """The Gaussian vortex of Sec. 5.1 at time t (centre translated by u_inf t = t, periodic):
    u = 1 - beta (y - y_c)/R^2 exp(-W^2/2), v = beta (x - x_c)/R^2 exp(-W^2/2),
    p = p_inf - rho beta^2/(2 R^2) exp(-W^2), W^2 = ((x - x_c)^2 + (y - y_c)^2)/R^2, with the strength
    beta/(u_inf R) = 0.02 of the paper, R = 1 (not printed) and constant density rho = 1 (the
    pressure of the paper's formula then balances the swirl exactly: a steady vortex carried by
    the free stream, an exact Euler solution)."""
    X, Y, _ = point_coords(case)
    xr = (X - t + case.lx / 2) % case.lx - case.lx / 2
    yr = (Y + case.ly / 2) % case.ly - case.ly / 2
    w2 = (xr * xr + yr * yr) / (R * R)
    g = np.exp(-0.5 * w2)
    rho = np.ones_like(X)
    u = 1.0 - beta * yr / (R * R) * g
    v = beta * xr / (R * R) * g
    p = 1.0 / (case.gamma * case.mach ** 2) - rho * beta ** 2 / (2 * R * R) * g * g
    return conserved(case, rho, u, v, np.zeros_like(X), p)


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


# ------------------------------------------------------------------ connected multi-block grids
#
# A multi-block grid: blocks (each a Case giving its size, split and spacing; the first block's
# Case also gives the physics and the scheme), optional point coordinates per block, and the six
# faces of every block.  Face types: periodic (the block wraps onto itself), interface (to face
# nf of block nb; node-disjoint; rev: the tangential in-plane index runs the other way on the
# neighbour), wall (no-slip adiabatic; the face's points are wall points), farfield (the given
# conserved state beyond the face) and outflow (the face values repeated beyond it).  Faces
# 0..5 = -x, +x, -y, +y, -z, +z; z faces are periodic.

FACE_TYPES = {"periodic": 0, "interface": 1, "wall": 2, "farfield": 3, "outflow": 4}


@dataclasses.dataclass
class Face:
    type: str = "periodic"
    nb: int = -1
    nf: int = -1
    rev: bool = False
    state: tuple = (0.0, 0.0, 0.0, 0.0, 0.0)
    shift: tuple = (0.0, 0.0)        # interface: (x, y) jump added to the neighbour's coordinates


@dataclasses.dataclass
class MultiBlock:
    blocks: list                     # Case per block
    faces: list                      # per block: six Face
    xy: list = None                  # per block: None or (xy [2][ny][nx], shift[4])
    name: str = "multiblock"

    def __post_init__(self):
        if self.xy is None:
            self.xy = [grid_xy(b) for b in self.blocks]

    @property
    def case(self) -> Case:
        return self.blocks[0]

    @property
    def npts(self) -> int:
        return sum(b.npts for b in self.blocks)

    @property
    def nsub(self) -> int:
        return sum(b.nsub for b in self.blocks)

    def replace_all(self, **kw) -> "MultiBlock":
        """The same grid with every block's Case updated (physics, scheme, algorithm, dt)."""
        return dataclasses.replace(self, blocks=[b.replace(**kw) for b in self.blocks])


def periodic_faces() -> list:
    return [Face() for _ in range(6)]


def split_states(mb: MultiBlock, U: np.ndarray) -> list:
    """A concatenated state (block after block, [5][nz][ny][nx] each) as a list of block states."""
    out, o = [], 0
    for b in mb.blocks:
        n = NV * b.npts
        out.append(U[o:o + n].reshape(NV, b.nz, b.ny, b.nx))
        o += n
    return out


def join_states(states) -> np.ndarray:
    return np.ascontiguousarray(np.concatenate([np.ascontiguousarray(s, dtype=np.float64).ravel() for s in states]))


def split_box_x(case: Case, n0: int, p0: int, p1: int) -> MultiBlock:
    """The periodic box of `case` cut at x index n0 into two blocks joined by two interfaces
    (y and z stay periodic); block 0 holds x indices [0, n0) split px = p0, block 1 the rest
    split px = p1."""
    b0 = case.replace(nx=n0, px=p0, lx=case.dx * n0)
    b1 = case.replace(nx=case.nx - n0, px=p1, lx=case.dx * (case.nx - n0))
    f0, f1 = periodic_faces(), periodic_faces()
    f0[1] = Face("interface", 1, 0)
    f0[0] = Face("interface", 1, 1)
    f1[0] = Face("interface", 0, 1)
    f1[1] = Face("interface", 0, 0)
    return MultiBlock([b0, b1], [f0, f1], xy=[None, None], name=case.name + "-split")


def rotated_pair(case: Case, n0: int, p0: int, p1: int) -> MultiBlock:
    """The curvilinear periodic grid of `case` (grid_xy) cut at x index n0 into two blocks, the
    second stored rotated by 180 degrees in the plane: its point (i', j') is the grid's point
    (nx - 1 - i', ny - 1 - j').  Both x faces of each block are interfaces with the tangential
    index reversed (-x to -x, +x to +x; the pair of -x faces closes the periodic x direction and
    carries its coordinate jump); y faces stay periodic (the rotated block's coordinate jump
    across its y wrap is -Ly)."""
    xy, shift = grid_xy(case)
    nx, ny = case.nx, case.ny
    n1 = nx - n0
    xy0 = np.ascontiguousarray(xy[:, :, :n0])
    # rotated block: columns n0..nx-1 reversed in both indices
    xy1 = np.ascontiguousarray(xy[:, ::-1, :][:, :, ::-1][:, :, :n1])
    b0 = case.replace(nx=n0, px=p0, lx=case.dx * n0)
    b1 = case.replace(nx=n1, px=p1, lx=case.dx * n1)
    f0, f1 = periodic_faces(), periodic_faces()
    f0[0] = Face("interface", 1, 0, True, shift=(-shift[0], -shift[1]))
    f0[1] = Face("interface", 1, 1, True)
    f1[0] = Face("interface", 0, 0, True, shift=(shift[0], shift[1]))
    f1[1] = Face("interface", 0, 1, True)
    s0 = np.array([0.0, 0.0, shift[2], shift[3]])
    s1 = np.array([0.0, 0.0, -shift[2], -shift[3]])
    return MultiBlock([b0, b1], [f0, f1], xy=[(xy0, s0), (xy1, s1)], name=case.name + "-rotated")


def rotate_state_pair(U: np.ndarray, n0: int):
    """Block states of rotated_pair from a state of the whole grid: block 1 is the columns
    n0.. of the 180-degree rotation (momentum components unchanged: they are Cartesian)."""
    nx = U.shape[-1]
    U0 = np.ascontiguousarray(U[..., :n0])
    U1 = np.ascontiguousarray(U[:, :, ::-1, ::-1][..., :nx - n0])
    return U0, U1


def span_pair(case: Case, n0: int, nz1: int, p0: int, p1: int) -> MultiBlock:
    """The periodic box of `case` cut at x index n0 into two blocks of different spanwise
    counts: block 0 keeps nz, block 1 has nz1 points over the same span."""
    m = split_box_x(case, n0, p0, p1)
    m.blocks[1] = m.blocks[1].replace(nz=nz1)
    m.name = case.name + "-span"
    return m


def wall_channel(case: Case) -> MultiBlock:
    """The box of `case` with no-slip adiabatic walls on both y faces (points j = 0 and
    j = ny - 1 are wall points); x and z periodic."""
    f = periodic_faces()
    f[2] = Face("wall")
    f[3] = Face("wall")
    return MultiBlock([case], [f], xy=[grid_xy(case)], name=case.name + "-channel")


def shear_wave_state(case: Case, eps: float) -> np.ndarray:
    """rho = 1, T = 1, u = eps sin(pi y / H) with y = j dy and H = (ny - 1) dy, v = w = 0."""
    H = (case.ny - 1) * case.dy
    y = case.dy * np.arange(case.ny)
    u = eps * np.sin(math.pi * y / H)
    shape = (case.nz, case.ny, case.nx)
    U = np.broadcast_to(u[None, :, None], shape)
    rho = np.ones(shape)
    p = np.full(shape, 1.0 / (case.gamma * case.mach ** 2))
    return conserved(case, rho, U, np.zeros(shape), np.zeros(shape), p)


# ------------------------------------------------------------------ NACA0012 C-grid (12 blocks)

def naca0012_half_thickness(x):
    """Four-digit NACA thickness distribution, t = 0.12, open trailing edge (y_t(1) = 0.00126)."""
    x = np.asarray(x, dtype=np.float64)
    return 5 * 0.12 * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2 + 0.2843 * x ** 3 - 0.1015 * x ** 4)


def _geometric_ratio(first: float, total: float, n: int) -> float:
    """Ratio r with first (r^n - 1)/(r - 1) = total (bisection)."""
    lo, hi = 1.0 + 1e-12, 4.0
    for _ in range(200):
        r = 0.5 * (lo + hi)
        if first * (r ** n - 1) / (r - 1) > total:
            hi = r
        else:
            lo = r
    return 0.5 * (lo + hi)


@dataclasses.dataclass
class CGridSpec:
    wake: int = 96           # points per side along the wake cut
    aft: int = 160           # points per side on the aft part of the airfoil
    fore: int = 512          # points per side on the fore part
    nj_in: int = 192         # wall-normal points of the inner layer
    nj_out: int = 64         # wall-normal points of the outer layer
    nz_in: int = 64          # spanwise points of the inner layer
    nz_out: int = 32         # spanwise points of the outer layer
    sub: tuple = (64, 64, 32)  # target sub-domain size (x, y, z)
    radius: float = 5.0      # far-field distance (chords)
    wake_len: float = 4.0    # wake length downstream of the trailing edge (chords)
    span: float = 0.25       # spanwise period (chords)
    alpha_deg: float = 2.0   # angle of attack
    mach: float = 0.3
    re: float = 5.0e4
    perturb: float = 1.0e-3  # amplitude of the seeded velocity perturbation (free-stream units)
    ramp: float = 0.05       # width of the initial wall-distance ramp of the velocity (chords)


def cgrid_reduced() -> CGridSpec:
    """A small C-grid with the same topology (43 k points, 80 sub-domains)."""
    return CGridSpec(wake=12, aft=20, fore=32, nj_in=24, nj_out=8, nz_in=12, nz_out=6, sub=(8, 12, 6))


def cgrid_plane(spec: CGridSpec):
    """Point coordinates of the whole C-grid plane, X, Y [nj][ni] with ni = 2 (wake + aft + fore)
    and nj = nj_in + nj_out.  Index i runs along the C from the lower end of the wake cut, under
    the airfoil to the leading edge, over it and back along the upper side of the cut; j runs
    outward.  Row j = 0: on the airfoil the surface points x = (1 - s)^2, y = -+ y_t(x) for
    s = (m + 1/2)/(aft + fore) (no point at the leading or trailing edge: blocks are
    node-disjoint); along the cut the lines y = -+ y_t(1), so that the cut spacing 2 y_t(1) equals
    the first wall-normal spacing.  Row nj - 1: the far field, a C of radius `radius` around
    (1/2, 0) closed by straight lines to the outflow.  Between them straight lines with a
    geometric wall-normal stretching."""
    ns = spec.aft + spec.fore
    nw = spec.wake
    s = (np.arange(ns) + 0.5) / ns
    xa = (1.0 - s) ** 2                           # trailing edge -> leading edge
    ya = naca0012_half_thickness(xa)
    te = float(naca0012_half_thickness(1.0))
    # wake: continues the surface spacing at the trailing edge, geometric growth to wake_len
    h0 = xa[0] - xa[1]
    q = _geometric_ratio(h0, spec.wake_len, nw)
    xw = 1.0 + (1.0 - xa[0]) + h0 * (q ** np.arange(nw) - 1.0) / (q - 1.0)  # nearest the trailing edge first
    # inner row, along i
    X0 = np.concatenate([xw[::-1], xa, xa[::-1], xw])
    Y0 = np.concatenate([np.full(nw, -te), -ya, ya[::-1], np.full(nw, te)])
    # outer row: straight lines y = -+R over the wake, around the airfoil a path from (1, -R)
    # along y = -R to (1/2, -R), a half circle of radius R around (1/2, 0), back to (1, R)
    R = spec.radius
    L1 = 0.5 + 0.5 * math.pi * R                  # one side's path length
    phi = s * L1
    def path(ph):
        if ph <= 0.5:
            return 1.0 - ph, -R
        th = (ph - 0.5) / R                       # angle swept from the bottom of the circle
        return 0.5 - R * math.sin(th), -R * math.cos(th)
    lower = np.array([path(ph) for ph in phi])
    X1 = np.concatenate([xw[::-1], lower[:, 0], lower[::-1, 0], xw])
    Y1 = np.concatenate([np.full(nw, -R), lower[:, 1], -lower[::-1, 1], np.full(nw, R)])
    nj = spec.nj_in + spec.nj_out
    r = _geometric_ratio(2 * te / (R - te), 1.0, nj - 1)
    sj = (r ** np.arange(nj) - 1.0) / (r ** (nj - 1) - 1.0)
    X = X0[None, :] + sj[:, None] * (X1 - X0)[None, :]
    Y = Y0[None, :] + sj[:, None] * (Y1 - Y0)[None, :]
    return X, Y


def naca_cgrid(spec: CGridSpec | None = None, algo: str = "SAA", kmax: int = 2) -> MultiBlock:
    """The 12-block C-grid around a NACA0012 airfoil: six segments along the C (lower wake,
    lower aft, lower fore, upper fore, upper aft, upper wake) times two layers (inner: nj_in x
    nz_in, outer: nj_out x nz_out, so the layers meet with different spanwise counts).  Faces:
    consecutive segments joined, the wake cut joins the two wake segments (tangential index
    reversed), the inner airfoil segments' j = 0 faces are no-slip adiabatic walls, the outer
    layer's far side is a far field at the free stream, the ends of the C are outflows; the span
    is periodic.  Navier-Stokes, Re_c, M, mu = T^0.76, CD4/AT4/LSERK4 with the filter."""
    spec = spec or CGridSpec()
    X, Y = cgrid_plane(spec)
    segs = [spec.wake, spec.aft, spec.fore, spec.fore, spec.aft, spec.wake]
    i0 = np.concatenate([[0], np.cumsum(segs)])
    al = math.radians(spec.alpha_deg)
    gam = 1.4
    p_inf = 1.0 / (gam * spec.mach ** 2)
    free = (1.0, math.cos(al), math.sin(al), 0.0, p_inf / (gam - 1.0) + 0.5)
    base = Case(name="naca0012", nx=8, ny=8, nz=8, mach=spec.mach, re=spec.re, pr=0.72, viscous=True,
                visc_law=1, visc_exp=0.76, order=4, algo=algo, at=True, caa_L=4, kmax=kmax, filter=True,
                lx=1.0, ly=1.0, lz=spec.span)
    blocks, faces, xy = [], [], []
    for layer in range(2):
        j0 = 0 if layer == 0 else spec.nj_in
        nj = spec.nj_in if layer == 0 else spec.nj_out
        nz = spec.nz_in if layer == 0 else spec.nz_out
        for sgi, ni in enumerate(segs):
            b = layer * 6 + sgi
            blocks.append(base.replace(nx=ni, ny=nj, nz=nz, px=max(1, ni // spec.sub[0]),
                                       py=max(1, nj // spec.sub[1]), pz=max(1, nz // spec.sub[2]),
                                       lx=float(ni), ly=float(nj), lz=spec.span))
            sl = (slice(j0, j0 + nj), slice(i0[sgi], i0[sgi + 1]))
            xy.append((np.ascontiguousarray(np.stack([X[sl], Y[sl]])), np.zeros(4)))
            f = periodic_faces()
            f[0] = Face("outflow") if sgi == 0 else Face("interface", b - 1, 1)
            f[1] = Face("outflow") if sgi == 5 else Face("interface", b + 1, 0)
            if layer == 0:
                if sgi == 0:
                    f[2] = Face("interface", 5, 2, True)
                elif sgi == 5:
                    f[2] = Face("interface", 0, 2, True)
                else:
                    f[2] = Face("wall")
                f[3] = Face("interface", b + 6, 2)
            else:
                f[2] = Face("interface", b - 6, 3)
                f[3] = Face("farfield", state=free)
            faces.append(f)
    return MultiBlock(blocks, faces, xy=xy, name="naca0012-cgrid")


def cgrid_state(mb: MultiBlock, spec: CGridSpec | None = None, seed: int = 2506030) -> list:
    """Initial state per block: rho = 1, T = 1, the free-stream velocity times the ramp
    1 - exp(-(d / ramp)^2) of the distance d to the airfoil (for a point of an airfoil segment the
    distance to the surface point at the foot of its grid line, for a wake point the distance to
    the trailing edge (1, 0)), plus seeded uniform perturbations of amplitude perturb times the
    ramp on all three velocity components (zero on the wall)."""
    spec = spec or CGridSpec()
    X, Y = cgrid_plane(spec)
    segs = [spec.wake, spec.aft, spec.fore, spec.fore, spec.aft, spec.wake]
    i0 = np.concatenate([[0], np.cumsum(segs)])
    al = math.radians(spec.alpha_deg)
    rng = np.random.default_rng(seed)
    out = []
    for b, c in enumerate(mb.blocks):
        layer, sgi = divmod(b, 6)
        j0 = 0 if layer == 0 else spec.nj_in
        sl = (slice(j0, j0 + c.ny), slice(i0[sgi], i0[sgi + 1]))
        x, y = X[sl], Y[sl]
        if sgi in (0, 5):
            dist = np.hypot(x - 1.0, y)
        else:
            dist = np.hypot(x - X[0, sl[1]][None, :], y - Y[0, sl[1]][None, :])
        g = 1.0 - np.exp(-(dist / spec.ramp) ** 2)
        shape = (c.nz, c.ny, c.nx)
        pert = spec.perturb * (2.0 * rng.random((3,) + shape) - 1.0) * g[None, None]
        u = math.cos(al) * g[None] + pert[0]
        v = math.sin(al) * g[None] + pert[1]
        w = pert[2]
        rho = np.ones(shape)
        p = np.full(shape, 1.0 / (c.gamma * c.mach ** 2))
        U = conserved(c, rho, np.broadcast_to(u, shape), np.broadcast_to(v, shape), w, p)
        out.append(U)
    return out


def cgrid_dt(mb: MultiBlock, cfl: float = 0.5) -> float:
    """CFL time step: cfl times the smallest in-plane point spacing (or the spanwise spacing)
    over the largest free-stream |u| + c = 1 + 1/M."""
    h = min(b.dz for b in mb.blocks)
    for (xy, _), b in zip(mb.xy, mb.blocks):
        X, Y = xy
        h = min(h, float(np.hypot(np.diff(X, axis=1), np.diff(Y, axis=1)).min()),
                float(np.hypot(np.diff(X, axis=0), np.diff(Y, axis=0)).min()))
    c = mb.case
    return cfl * h / (1.0 + 1.0 / c.mach)
