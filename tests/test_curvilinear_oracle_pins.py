"""Pins of the oracle's curvilinear path (App. A, Eq. A1-A4 on a periodic mapped grid; no GPU).

The mapped grid is x = x0 + i dx + A sin(2 pi j / ny), y = y0 + j dy + A sin(2 pi i / nx), extruded
in z.  What fixes the result independently of the oracle: a uniform flow is an exact solution of
the equations and the cofactor form of the metric terms keeps it exact discretely (freestream
preservation); with an undeformed grid given as coordinates the curvilinear form must reproduce
the Cartesian right-hand side; the translating vortex converges to the exact solution at the
scheme's order on the deformed grid; and the volume-weighted totals sum U J^-1 are conserved.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2506_03027_gb300 import inputs as I


def uniform_state(c, u=(0.7, -0.4, 0.3)):
    U = np.empty((5, c.nz, c.ny, c.nx))
    rho, p = 1.1, 1.0 / (c.gamma * c.mach ** 2)
    U[0] = rho
    for k in range(3):
        U[1 + k] = rho * (u[k] if (k < 2 or c.nz > 1) else 0.0)
    U[4] = p / (c.gamma - 1) + 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho
    return U


@pytest.mark.parametrize("three_d", [False, True])
def test_freestream_preserved_on_curvilinear_grid(three_d):
    if three_d:
        c = I.tgv_case(16, 2, "SA", curv=0.3)
    else:
        c = I.vortex_case(32, 2, curv=0.6)
    U = uniform_state(c)
    R = orc.rhs(c, U)
    scale = np.abs(U).max()
    assert np.abs(R).max() < 1e-12 * scale, np.abs(R).max()
    # and a deformed grid does change a non-uniform right-hand side (the path is active)
    V = I.tgv_state(c) if three_d else I.vortex_state(c)
    c0 = c.replace(curv=0.0)
    assert np.abs(orc.rhs(c, V) - orc.rhs(c0, V)).max() > 1e-3 * np.abs(orc.rhs(c0, V)).max()


@pytest.mark.parametrize("three_d", [False, True])
def test_undeformed_coordinates_reproduce_cartesian_rhs(three_d):
    """A grid of amplitude 1e-300 has exactly the Cartesian coordinates but takes the curvilinear
    code path (metric terms from the coordinates, fluxes with contravariant velocities)."""
    if three_d:
        c = I.tgv_case(16, 2, "SA")
        U = I.tgv_state(c)
    else:
        c = I.vortex_case(32, 2)
        U = I.vortex_state(c)
    Rc = orc.rhs(c, U)
    Rm = orc.rhs(c.replace(curv=1e-300), U)
    for v in range(5):
        ref = np.abs(Rc[v]).max() + 1e-300
        assert np.abs(Rm[v] - Rc[v]).max() < 1e-11 * max(ref, np.abs(Rc).max() * 1e-3), v


def test_curvilinear_vortex_order_of_accuracy():
    """The translating Euler vortex on the deformed grid converges at order 4 (CD4, LSERK4)."""
    e = []
    for n in (96, 192):
        c = I.vortex_case(n, 2, lx=16.0, ly=16.0, curv=0.8)
        dt0 = I.cfl_dt(c, I.vortex_state(c), 0.4)
        ns = int(math.ceil(0.5 / dt0))
        c = c.replace(dt=0.5 / ns)
        U = orc.run(c, I.vortex_state(c), ns)
        ex = I.vortex_state(c, t=0.5)
        e.append(math.sqrt(np.mean((U[0] - ex[0]) ** 2)))
    rate = math.log2(e[0] / e[1])
    assert abs(rate - 4) < 0.35, (e, rate)


def test_curvilinear_conservation():
    """sum U J^-1 is conserved to rounding on the deformed periodic grid (SA, filter off): the
    strong conservation form telescopes in index space."""
    c = I.tgv_case(16, 2, "SA", filter=False, curv=0.25)
    U0 = I.tgv_state(c)
    U = orc.run(c, U0, 8)
    d0 = orc.diagnostics(c, U0)
    d1 = orc.diagnostics(c, U)
    scale = np.abs(U0).reshape(5, -1).sum(axis=1) * c.dx * c.dy * c.dz
    scale = np.maximum(scale, scale[1])
    assert np.all(np.abs(d1[2:7] - d0[2:7]) < 1e-13 * scale), (d1[2:7] - d0[2:7]) / scale
    assert np.all(np.isfinite(U))
