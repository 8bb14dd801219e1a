"""Pins of the oracle's connected multi-block path (no GPU).

Blocks meet at interfaces (node-disjoint, tangential index aligned or reversed, spanwise counts
equal or different) and end at physical boundaries (no-slip adiabatic walls, far fields,
outflows).  What fixes the results independently of the oracle:

  * a periodic box cut into two blocks joined by interfaces is the same PE decomposition as the
    uncut box, so the run is identical (delays, filter and all);
  * a cut box whose second block is stored rotated by 180 degrees (a curvilinear block with the
    index directions reversed, joined to the first across reversed interfaces, the topology of
    an airfoil C-grid's wake cut) is the same discrete problem: the run equals the unrotated one
    to rounding;
  * a flow that does not depend on z stays so, and the spanwise interpolation between blocks of
    different spanwise counts reproduces it; for a flow that does depend on z the interpolated
    halo values converge at fourth order;
  * between two no-slip walls the shear wave u = eps sin(pi y / H) is an exact discrete
    eigenmode: the mirrored halo continues the sine exactly, so each velocity sample decays by the
    LSERK4 stability polynomial of -dt kappa'^2 / Re, kappa' the CD4 modified wavenumber
    (App. B) of pi / H;
  * on the 12-block NACA0012 C-grid with the walls replaced by far fields at the free-stream
    state, the free stream is an exact solution: metric terms continued across interfaces and
    the wake cut keep it exact discretely (freestream preservation), with SAA delays too.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2506_03027_gb300 import inputs as I


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_state(U, ref):
    """Relative L2 per conserved variable; momentum components against the momentum norm."""
    mom = math.sqrt(sum(float(np.linalg.norm(ref[v])) ** 2 for v in (1, 2, 3)))
    return [float(np.linalg.norm(U[v] - ref[v]) / (mom if v in (1, 2, 3) else np.linalg.norm(ref[v])))
            for v in range(5)]


def test_split_box_equals_single_block():
    c = I.tgv_case(24, 2, "SAA", kmax=2, filter=True)
    c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), 0.1), px=3)
    U0 = I.tgv_state(c)
    n = 8
    d = I.saa_delays(c, n)
    Ur = orc.run(c, U0, n, delays=d)
    mb = I.split_box_x(c, 16, 2, 1)
    # the same PEs, numbered block after block: x index 0, 1 of each (y, z) in block 0, then 2
    idx0 = [ix + 3 * (iy + 2 * iz) for iz in range(2) for iy in range(2) for ix in range(2)]
    idx1 = [2 + 3 * (iy + 2 * iz) for iz in range(2) for iy in range(2)]
    dm = np.ascontiguousarray(d[:, idx0 + idx1, :])
    Um = orc.run(mb, [U0[..., :16], U0[..., 16:]], n, delays=dm)
    assert np.array_equal(Um[0], Ur[..., :16]) and np.array_equal(Um[1], Ur[..., 16:])


def test_rotated_block_equals_unrotated_grid():
    c = I.tgv_case(24, 2, "CAA", filter=True, curv=0.2)
    c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), 0.1), px=3)
    U0 = I.tgv_state(c)
    n = 10
    Ur = orc.run(c, U0, n)
    mb = I.rotated_pair(c, 16, 2, 1)
    Um = orc.run(mb, list(I.rotate_state_pair(U0, 16)), n)
    R0, R1 = I.rotate_state_pair(Ur, 16)
    assert max(rel_state(Um[0], R0)) < 1e-12 and max(rel_state(Um[1], R1)) < 1e-12
    # a reversed interface taken unreversed is a different (wrong) problem: the check has teeth
    bad = dataclasses.replace(mb, faces=[[dataclasses.replace(f, rev=False) if f.type == "interface" else f
                                           for f in fs] for fs in mb.faces])
    Ub = orc.run(bad, list(I.rotate_state_pair(U0, 16)), n)
    assert rel(Ub[1][1], R1[1]) > 1e-4


def _z_independent_state(c):
    """The 2-D isentropic vortex of `c`'s plane, extruded along z."""
    c2 = c.replace(nz=1, pz=1)
    U2 = I.vortex_state(c2)
    return np.ascontiguousarray(np.broadcast_to(U2, (5, c.nz, c.ny, c.nx)))


def test_spanwise_interface_keeps_z_independent_flow():
    c = I.vortex_case(24, 2).replace(nz=12, pz=1, lz=1.0, filter=True)
    c = c.replace(dt=I.cfl_dt(c.replace(nz=1, pz=1), I.vortex_state(c.replace(nz=1, pz=1)), 0.3))
    U0 = _z_independent_state(c)
    n = 12
    Ur = orc.run(c, U0, n)
    mb = I.span_pair(c, 12, 6, 1, 1)  # block 1: 6 spanwise points over the same span
    Um = orc.run(mb, [U0[..., :12], np.ascontiguousarray(U0[:, ::2, :, 12:])], n)
    assert max(rel_state(Um[0], Ur[:, :, :, :12])) < 1e-13
    assert max(rel_state(Um[1], Ur[:, ::2, :, 12:])) < 1e-13


def test_spanwise_interpolation_is_fourth_order():
    """RHS next to an interface with a coarser spanwise neighbour, against the RHS on the uniform
    fine grid, for a field with a z dependence: the difference comes from the interpolated halo
    values and falls by about 2^4 when the spanwise counts double."""
    errs = []
    for nz in (8, 16):
        c = I.vortex_case(24, 2).replace(nz=nz, pz=1, lz=1.0, viscous=False)
        U = _z_independent_state(c).copy()
        z = c.dz * np.arange(nz)
        U[1] = U[1] * (1.0 + 0.2 * np.sin(2 * math.pi * z)[:, None, None])
        Rf = orc.rhs(c, U)
        mb = I.span_pair(c, 12, nz // 2, 1, 1)
        Rm = orc.rhs(mb, [U[..., :12], np.ascontiguousarray(U[:, ::2, :, 12:])])
        errs.append(float(np.abs(Rm[0][1][:, :, -2:] - Rf[1][:, :, 10:12]).max()))
    assert errs[0] > 0 and 10.0 < errs[0] / errs[1] < 24.0, errs


def test_shear_wave_between_walls_decays_at_discrete_rate():
    c = I.tgv_case(16, 2, "SA").replace(ny=17, py=2, re=10.0, ly=1.0, filter=False)
    c = c.replace(dt=0.3 * c.dy * c.mach)  # acoustic CFL 0.3
    eps = 1e-6
    mb = I.wall_channel(c)
    U0 = I.shear_wave_state(c, eps)
    n = 30
    U = orc.run(mb, [U0], n)[0]
    # CD4 modified wavenumber (App. B: a = 4/3, b = -1/3) of k = pi / H
    H = (c.ny - 1) * c.dy
    k = math.pi / H
    kp = ((4.0 / 3.0) * math.sin(k * c.dy) + (-1.0 / 3.0) / 2.0 * math.sin(2 * k * c.dy)) / c.dy
    z = -c.dt * kp ** 2 / c.re
    A, B = orc.lserk(4)
    amp = 1.0
    for _ in range(n):
        u, q = amp, 0.0
        for m in range(len(A)):
            q = A[m] * q + z * u
            u = u + B[m] * q
        amp = u
    inner = np.abs(U0[1]) > 0.1 * eps
    ratio = U[1][inner] / U0[1][inner]
    assert np.allclose(ratio, amp, rtol=1e-9, atol=0), (ratio.min(), ratio.max(), amp)
    assert np.all(U[1][:, 0, :] == 0.0) and np.all(U[1][:, -1, :] == 0.0)
    assert np.abs(U[2]).max() < 1e-12 and amp < 0.99


@pytest.mark.parametrize("algo", ["SA", "SAA"])
def test_cgrid_freestream_preserved(algo):
    sp = I.cgrid_reduced()
    mb = I.naca_cgrid(sp, algo=algo)
    free = mb.faces[6][3].state
    faces = [[dataclasses.replace(f, type="farfield", state=free) if f.type == "wall" else f for f in fs]
             for fs in mb.faces]
    mb = dataclasses.replace(mb, faces=faces).replace_all(dt=I.cgrid_dt(mb, 0.05))
    U0 = [np.ascontiguousarray(np.broadcast_to(np.asarray(free)[:, None, None, None], (5, b.nz, b.ny, b.nx)))
          for b in mb.blocks]
    n = 12
    d = I.saa_delays(mb.case.replace(px=mb.nsub, py=1, pz=1), n) if algo == "SAA" else None
    U = orc.run(mb, U0, n, delays=d)
    assert max(float(np.abs(a - b).max()) for a, b in zip(U, U0)) < 1e-12 * max(free)
    # the same grid with a non-uniform state does move (the check has teeth)
    U1 = orc.run(mb, I.cgrid_state(mb, sp), 2, delays=d)
    assert max(float(np.abs(a - b).max()) for a, b in zip(U1, I.cgrid_state(mb, sp))) > 1e-6


def test_cgrid_topology():
    """The C-grid's faces pair up both ways with matching tangential counts, the wall points
    start at rest, and the grid cells all have positive area."""
    sp = I.cgrid_reduced()
    mb = I.naca_cgrid(sp)
    for b, fs in enumerate(mb.faces):
        for f, F in enumerate(fs):
            if F.type == "interface":
                G = mb.faces[F.nb][F.nf]
                assert G.type == "interface" and G.nb == b and G.nf == f and G.rev == F.rev
                t = (mb.blocks[b].ny, mb.blocks[b].nx)[f // 2]
                t2 = (mb.blocks[F.nb].ny, mb.blocks[F.nb].nx)[F.nf // 2]
                assert t == t2
    assert sum(F.type == "wall" for fs in mb.faces for F in fs) == 4
    U = I.cgrid_state(mb, sp)
    for b in range(1, 5):
        assert np.all(U[b][1:4, :, 0, :] == 0.0)
    X, Y = I.cgrid_plane(sp)
    area = (X[:-1, 1:] - X[:-1, :-1]) * (Y[1:, :-1] - Y[:-1, :-1]) - (Y[:-1, 1:] - Y[:-1, :-1]) * (X[1:, :-1] - X[:-1, :-1])
    assert area.min() > 0
    assert abs(mb.npts - 43008) == 0 and I.naca_cgrid().npts == 22020096


def test_conservation_across_reversed_interfaces():
    """The synchronous curvilinear scheme is conservative: the volume-weighted totals sum U J^-1
    of the rotated pair (two blocks joined by reversed interfaces, one stored rotated by 180
    degrees) stay constant to rounding -- they drift exactly as the uncut single block's do -- so
    the two blocks see one flux at their interfaces."""
    c = I.tgv_case(24, 2, "SA", curv=0.2).replace(px=3)
    c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), 0.25))
    mb = I.rotated_pair(c, 16, 2, 1)
    U0 = list(I.rotate_state_pair(I.tgv_state(c), 16))
    d0 = orc.diagnostics(mb, U0)
    U, dg = orc.run(mb, U0, 20, diag=True)
    # the single deformed block drifts by the rounding of J J^-1 != 1 times the pressure fluxes
    # (a few 1e-12 in 20 steps); the pair must drift exactly as much
    s0 = orc.diagnostics(c, I.tgv_state(c))
    _, ds = orc.run(c, I.tgv_state(c), 20, diag=True)
    scale = [abs(d0[2]), abs(d0[2]), abs(d0[2]), abs(d0[2]), abs(d0[6])]
    for v in range(5):
        pair = (dg[-1][2 + v] - d0[2 + v]) / scale[v]
        single = (ds[-1][2 + v] - s0[2 + v]) / scale[v]
        assert abs(pair) < 1e-10 and abs(pair - single) < 1e-14, (v, pair, single)
    # taking the interfaces unreversed breaks it (the run drifts or blows up)
    bad = dataclasses.replace(mb, faces=[[dataclasses.replace(f, rev=False) if f.type == "interface" else f
                                           for f in fs] for fs in mb.faces])
    Ub, db = orc.run(bad, U0, 20, diag=True)
    drift = abs(db[-1][6] - d0[6]) / scale[4]
    assert not np.isfinite(drift) or drift > 1e-9, drift


def test_cgrid_geometry_recipe():
    """The C-grid of config 3 as its recipe states it: airfoil rows on the NACA0012 surface
    (y = -+ y_t(x), no point at either edge), wake rows on y = -+ y_t(1) so that the cut spacing
    2 y_t(1) equals the first wall-normal spacing, the far field a C of radius 5 chords around
    (1/2, 0) closed by straight lines, the wake reaching 4
    chords downstream, the two sides of the cut mirror images, and the block sizes of the
    configuration (96 x 64 x 32 up to 512 x 192 x 64, 22.0 M points)."""
    for sp in (I.CGridSpec(), I.cgrid_reduced()):
        X, Y = I.cgrid_plane(sp)
        nw, ns = sp.wake, sp.aft + sp.fore
        te = float(I.naca0012_half_thickness(1.0))
        assert abs(te - 0.00126) < 1e-6
        air = slice(nw, nw + 2 * ns)
        xa, ya = X[0, air], Y[0, air]
        assert np.all((xa > 0) & (xa < 1))
        assert np.allclose(np.abs(ya), I.naca0012_half_thickness(xa), rtol=0, atol=1e-15)
        assert np.all(Y[0, :nw] == -te) and np.all(Y[0, -nw:] == te)
        # first wall-normal spacing in the wake equals the cut spacing 2 y_t(1)
        assert abs((Y[0, 0] - Y[1, 0]) - 2 * te) < 1e-9
        xf, yf = X[-1], Y[-1]  # far field: |y| = 5 downstream of x = 1/2, a half circle ahead of it
        assert np.allclose(np.abs(yf[xf >= 0.5]), 5.0, atol=1e-9)
        assert np.allclose(np.hypot(xf[xf < 0.5] - 0.5, yf[xf < 0.5]), 5.0, atol=1e-9)
        # the wake ends one geometric growth step short of x = 1 + 4 chords
        assert 3.0 < X[0, 0] < 5.0 and X[0, -1] == X[0, 0]
        h = np.diff(X[0, nw - 1::-1])  # wake spacings from the trailing edge downstream
        assert np.all(h > 0) and np.allclose(h[1:] / h[:-1], h[1] / h[0], rtol=1e-9)
        # the cut's two sides are mirror images
        assert np.allclose(X[:, :nw], X[:, ::-1][:, :nw], atol=1e-12)
        assert np.allclose(Y[:, :nw], -Y[:, ::-1][:, :nw], atol=1e-12)
    mb = I.naca_cgrid()
    sizes = sorted((b.nx * b.ny * b.nz, (b.nx, b.ny, b.nz)) for b in mb.blocks)
    assert sizes[0][1] == (96, 64, 32) and sizes[-1][1] == (512, 192, 64) and mb.npts == 22020096
