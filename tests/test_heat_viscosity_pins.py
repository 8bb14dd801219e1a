"""Pins of the oracle's heat-flux and temperature-dependent viscosity terms (App. A, Eq. A3-A4),
which the isothermal, constant-viscosity Taylor-Green field cannot exercise (CPU only).

  * A fluid at rest with a temperature wave at uniform pressure: the inviscid fluxes and the
    stresses vanish, so the only right-hand side is the heat-flux divergence
    (1/Re) d/dx_i (mu / ((gamma-1) Pr M^2) dT/dx_i) in the energy equation.  With mu = 1 and the
    CD4 (or CD2) first derivative applied twice, R(rho E) of a sine wave is exactly
    -(kappa / Re) k'^2 eps sin(k x), k' the scheme's modified wavenumber (closed form).
  * With mu = T^a (the power law of the airfoil case) the same state converges to the calculus
    result (kappa/Re) d/dx (T^a dT/dx) at the scheme's order, and a shear wave at rest over a
    temperature wave converges to (1/Re) d/dy (T^a du/dy) in the momentum and
    (1/Re) d/dy (u T^a du/dy + kappa T^a dT/dy) in the energy equation.
  * The viscous part of R (R minus the same run without viscosity) of a non-isothermal
    three-dimensional field converges to the symbolically differentiated viscous operator with
    either law (sympy).
A factor or sign error in the heat flux, a double 1/Re, a wrong exponent or a viscosity that
misses the heat flux or the stresses fails one of them (checked by the tests' own variants in
the docstrings' derivations, not by editing the oracle).
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2506_03027_gb300 import inputs as I


def at_rest_case(n, axis, order, visc_law, gamma=1.3, mach=0.3, re=250.0, pr=0.8):
    """A periodic 3-D box of n points along `axis` (4 along the others), one sub-domain, at rest;
    physical constants chosen apart from the TGV's so that factors cannot compensate."""
    dims = [4, 4, 4]
    dims[axis] = n
    return I.Case(name="rest", nx=dims[0], ny=dims[1], nz=dims[2], px=1, py=1, pz=1, gamma=gamma, mach=mach,
                  re=re, pr=pr, viscous=True, visc_law=visc_law, visc_exp=0.76, order=order, filter=False)


def coords(case, axis):
    x, y, z = I.grid(case)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return (X, Y, Z)[axis]


def rest_state(case, T, u=None, u_axis=0):
    """U of a fluid at uniform pressure p0 = 1/(gamma M^2) with temperature T (rho = 1/T from
    p = rho T/(gamma M^2)), optionally moving with velocity u along u_axis."""
    p0 = 1.0 / (case.gamma * case.mach ** 2)
    rho = 1.0 / T
    vel = [np.zeros_like(T) for _ in range(3)]
    if u is not None:
        vel[u_axis] = u
    return I.conserved(case, rho, vel[0], vel[1], vel[2], np.full_like(T, p0))


def kappa(case):
    return 1.0 / ((case.gamma - 1.0) * case.pr * case.mach ** 2)


def modified_wavenumber(order, k, h):
    """k' of the central difference of Eq. 2 (alpha = 0): CD4 a = 4/3, b = -1/3; CD2 a = 1."""
    if order == 4:
        return ((4.0 / 3.0) * math.sin(k * h) - (1.0 / 6.0) * math.sin(2 * k * h)) / h
    return math.sin(k * h) / h


@pytest.mark.parametrize("curv", [0.0, 1e-300])
@pytest.mark.parametrize("order", [4, 2])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_temperature_wave_closed_form(order, axis, curv):
    """mu = 1: R = (0, 0, 0, 0, -(kappa/Re) k'^2 eps sin(k x)) exactly, on each axis; also through
    the curvilinear code path (an undeformed grid given as coordinates, curv = 1e-300)."""
    c = at_rest_case(24, axis, order, 0).replace(curv=curv)
    x = coords(c, axis)
    eps, k = 0.2, 3
    U = rest_state(c, 1.0 + eps * np.sin(k * x))
    R = orc.rhs(c, U)
    h = [c.dx, c.dy, c.dz][axis]
    kp = modified_wavenumber(order, k, h)
    exact = -(kappa(c) / c.re) * kp ** 2 * eps * np.sin(k * x)
    scale = np.abs(exact).max()
    assert np.abs(R[0]).max() < 1e-13 * scale
    assert np.abs(R[1:4]).max() < 1e-12 * scale
    np.testing.assert_allclose(R[4], exact, rtol=0, atol=1e-12 * scale)


def errors_and_rate(errs):
    return math.log2(errs[0] / errs[1])


@pytest.mark.parametrize("curv", [0.0, 1e-300])
@pytest.mark.parametrize("order", [4, 2])
def test_power_law_heat_flux_converges(order, curv):
    """mu = T^0.76, at rest: R(rho E) -> (kappa/Re) d/dx (T^a dT/dx) at the scheme's order;
    the viscosity does enter the heat flux (the mu = 1 operator differs by far more)."""
    a, eps, k = 0.76, 0.3, 1
    errs, diff_mu1 = [], None
    for n in (32, 64):
        c = at_rest_case(n, 0, order, 1).replace(curv=curv)
        x = coords(c, 0)
        T = 1.0 + eps * np.sin(k * x)
        Tx = eps * k * np.cos(k * x)
        Txx = -eps * k * k * np.sin(k * x)
        exact = (kappa(c) / c.re) * (a * T ** (a - 1) * Tx * Tx + T ** a * Txx)
        R = orc.rhs(c, rest_state(c, T))
        errs.append(np.abs(R[4] - exact).max())
        if diff_mu1 is None:
            diff_mu1 = np.abs(exact - (kappa(c) / c.re) * Txx).max()
        assert np.abs(R[:4]).max() < 1e-11 * np.abs(exact).max()
    assert abs(errors_and_rate(errs) - order) < 0.3, errs
    assert errs[1] < 0.05 * diff_mu1


@pytest.mark.parametrize("curv", [0.0, 1e-300])
@pytest.mark.parametrize("order", [4, 2])
def test_power_law_shear_wave_converges(order, curv):
    """mu = T^0.76: u = eps sin y over T = 1 + delta cos y at uniform pressure.  R(rho u) ->
    (1/Re) d/dy (T^a du/dy); R(rho E) -> (1/Re) d/dy (u T^a du/dy + kappa T^a dT/dy); rho, rho v,
    rho w unchanged."""
    a, eps, dl = 0.76, 0.05, 0.25
    errs_m, errs_e = [], []
    for n in (32, 64):
        c = at_rest_case(n, 1, order, 1).replace(curv=curv)
        y = coords(c, 1)
        u, uy, uyy = eps * np.sin(y), eps * np.cos(y), -eps * np.sin(y)
        T, Ty, Tyy = 1.0 + dl * np.cos(y), -dl * np.sin(y), -dl * np.cos(y)
        mu, muy = T ** a, a * T ** (a - 1) * Ty
        rm = (muy * uy + mu * uyy) / c.re
        re_ = (uy * mu * uy + u * muy * uy + u * mu * uyy + kappa(c) * (muy * Ty + mu * Tyy)) / c.re
        R = orc.rhs(c, rest_state(c, T, u=u, u_axis=0))
        errs_m.append(np.abs(R[1] - rm).max())
        errs_e.append(np.abs(R[4] - re_).max())
        assert np.abs(R[0]).max() < 1e-12 * np.abs(re_).max()
        assert np.abs(R[2:4]).max() < 1e-11 * np.abs(re_).max()
    assert abs(errors_and_rate(errs_m) - order) < 0.3, errs_m
    assert abs(errors_and_rate(errs_e) - order) < 0.3, errs_e


def continuous_viscous_operator(case, visc_law):
    """The viscous part of Eq. 1 for a non-isothermal field (textbook tensor form, sympy):
    (1/Re) div of (0, tau_i1, tau_i2, tau_i3, u_j tau_ij + mu/((gamma-1) Pr M^2) dT/dx_i) with
    tau_ij = mu (du_i/dx_j + du_j/dx_i) - 2/3 mu div u delta_ij and mu = 1 or T^a."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    X = [x, y, z]
    g, M, Re, Pr = case.gamma, case.mach, case.re, case.pr
    vel = [sp.sin(x) * sp.cos(y) * sp.cos(z), -sp.cos(x) * sp.sin(y) * sp.cos(z),
           sp.Rational(1, 4) * sp.sin(2 * z) * sp.cos(x)]
    T = 1 + sp.Rational(1, 5) * sp.sin(x + 2 * y) * sp.cos(z) + sp.Rational(1, 10) * sp.cos(2 * x)
    p = 1 / (g * M ** 2) + (sp.cos(2 * x) + sp.cos(2 * y)) * (sp.cos(2 * z) + 2) / 16
    rho = g * M ** 2 * p / T
    mu = T ** sp.Float(case.visc_exp) if visc_law == 1 else sp.Integer(1)
    grad = [[sp.diff(vel[i], X[j]) for j in range(3)] for i in range(3)]
    div = sum(grad[i][i] for i in range(3))
    tau = [[mu * (grad[i][j] + grad[j][i]) - sp.Rational(2, 3) * mu * div * (1 if i == j else 0)
            for j in range(3)] for i in range(3)]
    heat = [mu / ((g - 1) * Pr * M ** 2) * sp.diff(T, X[i]) for i in range(3)]
    flux = [[0, 0, 0]] + [[tau[a][c] for a in range(3)] for c in range(3)]
    flux.append([sum(vel[j] * tau[a][j] for j in range(3)) + heat[a] for a in range(3)])
    ops = [sp.lambdify((x, y, z), sum(sp.diff(flux[v][a], X[a]) for a in range(3)) / Re, "numpy")
           for v in range(5)]
    prims = [sp.lambdify((x, y, z), e, "numpy") for e in (rho, vel[0], vel[1], vel[2], p)]
    return ops, prims


@pytest.mark.parametrize("curv", [0.0, 0.2])
@pytest.mark.parametrize("visc_law", [0, 1])
@pytest.mark.parametrize("order", [4, 2])
def test_viscous_part_converges_non_isothermal(order, visc_law, curv):
    """R(viscous) - R(Euler) of the oracle converges to the continuous viscous operator at the
    scheme's order for a field whose temperature varies in all three directions; on the uniform
    grid and on a deformed curvilinear grid (App. A metric terms, the field sampled at the mapped
    points)."""
    base = I.tgv_case(16, 2, "SA", order=order, filter=False, visc_law=visc_law, re=100.0, curv=curv)
    ops, prims = continuous_viscous_operator(base, visc_law)
    errs, mags = [], []
    for n in (16, 32):
        c = base.replace(nx=n, ny=n, nz=n)
        X, Y, Z = I.point_coords(c)
        f = [np.broadcast_to(np.asarray(fn(X, Y, Z), dtype=np.float64), X.shape) for fn in prims]
        U = I.conserved(c, f[0], f[1], f[2], f[3], f[4])
        Rv = orc.rhs(c, U) - orc.rhs(c.replace(viscous=False), U)
        e = 0.0
        for v in range(1, 5):
            ex = np.broadcast_to(np.asarray(ops[v](X, Y, Z), dtype=np.float64), X.shape)
            e = max(e, np.abs(Rv[v] - ex).max() / np.abs(ex).max())
        assert np.abs(Rv[0]).max() == 0.0
        errs.append(e)
    assert abs(errors_and_rate(errs) - order) < 0.4, errs
