"""Parameter studies of the asynchronous schemes run through the library.

async_error_vs_delay: the error the asynchrony adds on the translating isentropic vortex under
CAA-AT with the second-order schemes (LSERK2, CD2, AT2: Table 1, case 3) as a function of the
maximum allowable delay L and of the number of sub-domains P (the study of Sec. 5.1 behind its
Fig. 4).  The added error of a run is the RMS difference of its u-velocity from the synchronous
run with the same grid, decomposition and time step, after the same number of steps; the
synchronous run's error against the exact translated vortex is returned beside it.
"""
from __future__ import annotations

import math

import numpy as np

from . import cfs
from . import inputs as I


def _u(U):
    return U[1] / U[0]


def async_error_vs_delay(n: int, p: int, Ls, t_end: float = 1.0, cfl: float = 0.2, order: int = 2) -> dict:
    """Vortex on n x n points, p x p sub-domains; one synchronous run and one CAA-AT run per L in
    ``Ls`` (delays k(n) = (n - C) mod L), all with the time step of CFL ``cfl`` and t_end."""
    base = I.vortex_case(n, p, order=order)
    dt = I.cfl_dt(base, I.vortex_state(base), cfl)
    nsteps = int(math.ceil(t_end / dt))
    base = base.replace(dt=t_end / nsteps)
    U0 = I.vortex_state(base)

    def run(case):
        s = cfs.Solver(case, max_delay=max(0, case.caa_L - 1) if case.algo == "CAA" else None)
        try:
            s.set_schedule()
            s.set_state(U0)
            s.step(nsteps)
            return s.get_state()
        finally:
            s.close()

    Usa = run(base)
    exact = I.vortex_state(base, t=t_end)
    out = {"n": n, "P": p * p, "steps": nsteps, "dt": base.dt,
           "sa_error": float(math.sqrt(np.mean((_u(Usa) - _u(exact)) ** 2))), "L": [], "async_error": []}
    for L in Ls:
        U = run(base.replace(algo="CAA", at=True, caa_L=int(L), kmax=max(0, int(L) - 1)))
        out["L"].append(int(L))
        out["async_error"].append(float(math.sqrt(np.mean((_u(U) - _u(Usa)) ** 2))))
    return out


def cubic_fit(L, E):
    """Least-squares fit E ~ g1 L + g2 L^2 + g3 L^3 (the moments of the delay in the error
    estimate of the AT schemes); returns (g1, g2, g3) and the relative RMS residual."""
    L = np.asarray(L, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    A = np.stack([L, L ** 2, L ** 3], axis=1)
    g, *_ = np.linalg.lstsq(A, E, rcond=None)
    res = float(np.sqrt(np.mean((A @ g - E) ** 2)) / np.sqrt(np.mean(E ** 2)))
    return g, res
