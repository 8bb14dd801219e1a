"""Parameter studies of the asynchronous schemes run through the library.

async_error_vs_delay: the error the asynchrony adds on the translating isentropic vortex under
CAA-AT with the second-order schemes (LSERK2, CD2, AT2: Table 1, case 3) as a function of the
maximum allowable delay L and of the number of sub-domains P (the study of Sec. 5.1 behind its
Fig. 4).  The added error of a run is the RMS difference of its u-velocity from the synchronous
run with the same grid, decomposition and time step, after the same number of steps; the
synchronous run's error against the exact translated vortex is returned beside it.

paper_vortex_errors: the paper's own vortex setup (Sec. 5.1, Table 1, Fig. 2(a)) -- convergence
of the density error over one advection cycle for the six scheme cases, on the GPU.
stability_sweep: the first non-finite step of the Taylor-Green configuration per schedule and CFL.
Command line: python -m paper_2506_03027_gb300.studies paper-vortex [n ...] | stability [n p nsteps]
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


# Table 1 of the paper: scheme cases (kind, LSERK/CD order, AT, expected overall order)
TABLE1 = {1: ("SA", 2, True, 2), 2: ("AS", 2, False, 1), 3: ("AT", 2, True, 2),
          4: ("SA", 4, True, 4), 5: ("AS", 4, False, 1), 6: ("AT", 4, True, 4)}

# (case, algorithm, maximum allowable delay L) of the study: the paper's L = 8 throughout, and
# SAA-AT with the fourth-order schemes also at L = 4 (at L = 8 it goes unstable, see below)
PAPER_VORTEX_RUNS = ((1, "SA", 8), (2, "CAA", 8), (2, "SAA", 8), (3, "CAA", 8), (3, "SAA", 8),
                     (4, "SA", 8), (5, "CAA", 8), (5, "SAA", 8), (6, "CAA", 8), (6, "SAA", 8), (6, "SAA", 4))


def paper_vortex_errors(ns=(60, 120, 240), runs=PAPER_VORTEX_RUNS, seeds=(1, 2, 3), t_end: float = 16.0,
                        p_late: float = 0.6) -> dict:
    """The paper's vortex test (Sec. 5.1, Fig. 2(a)): one advection cycle (t = 16) of the Gaussian
    vortex on [-8, 8]^2 with three PEs along x, for the scheme cases of Table 1 -- SA (cases 1,
    4), CAA-AS and SAA-AS (2, 5), CAA-AT and SAA-AT (3, 6) -- at the resolutions `ns` and the
    paper's time steps.  SAA delays follow the arrival model of Alg. 3 (inputs.saa_delays_arrival:
    consecutive visible levels, mean delay about 1.5).  The error of a run is the RMS density
    error over all points against the exact solution (the vortex back at its initial position);
    SAA errors are means over independent delay sequences (`seeds`).  A run that goes
    non-finite reports NaN.  Returns the errors and the orders between consecutive resolutions."""
    import torch
    rows = []
    for case_no, algo, L in runs:
        kind, order, at, expected = TABLE1[case_no]
        errs = []
        for n in ns:
            c = I.paper_vortex_case(n, order=order, algo=algo, at=at, L=L)
            nsteps = int(round(t_end / c.dt))
            c = c.replace(dt=t_end / nsteps)
            U0 = I.paper_vortex_state(c)
            exact = I.paper_vortex_state(c, t=t_end)
            e = []
            for sd in (seeds if algo == "SAA" else (None,)):
                d = I.saa_delays_arrival(c, nsteps, L, p_late=p_late, seed=sd) if algo == "SAA" else None
                st = torch.cuda.Stream()
                with torch.cuda.stream(st):
                    s = cfs.Solver(c, max_delay=0 if algo == "SA" else L - 1, graph=True, stream=st)
                    try:
                        s.set_schedule(delays=d)
                        s.set_state(U0)
                        s.step(nsteps)
                        U = s.get_state()
                    finally:
                        s.close()
                e.append(float(np.sqrt(np.mean((U[0] - exact[0]) ** 2))))
            errs.append(float(np.mean(e)))
        orders = [math.log(errs[i] / errs[i + 1]) / math.log(ns[i + 1] / ns[i]) for i in range(len(ns) - 1)]
        label = algo if kind == "SA" else f"{algo}-{kind}"
        rows.append({"case": case_no, "algorithm": label, "L": L, "time_stepping": f"LSERK{order}",
                     "expected_order": expected, "errors": errs, "orders": orders})
    return {"n": list(ns), "t_end": t_end, "p_late": p_late, "rows": rows}


def stability_sweep(n: int = 128, p: int = 4, algos=("SAA", "CAA", "SA"), cfls=(0.5, 0.25, 0.1, 0.05),
                    nsteps: int = 600, every: int = 25, kmax: int = 3) -> list:
    """Asynchronous stability of the Taylor-Green configuration (Navier-Stokes, filter, n^3 on p^3
    sub-domains, FP64): per schedule (SA, CAA with L = 4, SAA with delays 0..kmax) and CFL number,
    the first multiple of `every` steps at which the state holds a non-finite value (None when it
    stays finite for nsteps steps) and the kinetic energy at the last finite check."""
    rows = []
    for algo in algos:
        for cfl in cfls:
            c = I.tgv_case(n, p, algo, kmax=kmax)
            c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), cfl))
            d = I.saa_delays(c, nsteps) if algo == "SAA" else None
            s = cfs.Solver(c)
            first, k_last = None, None
            try:
                s.set_schedule(delays=d)
                s.set_state(I.tgv_state(c))
                for done in range(every, nsteps + 1, every):
                    s.step(every)
                    dg = s.diagnostics(check_finite=False)
                    if dg[7] != 0.0:
                        first = done
                        break
                    k_last = float(dg[0])
            finally:
                s.close()
            rows.append({"algo": algo, "cfl": cfl, "dt": c.dt, "first_nonfinite_by_step": first, "K_last": k_last})
    return rows


def _main(argv):
    import json
    if argv and argv[0] == "paper-vortex":
        ns = tuple(int(v) for v in argv[1:]) or (60, 120, 240)
        out = paper_vortex_errors(ns)
        print(json.dumps(out))
        print("case  algorithm   L  expected  errors (n = " + ", ".join(str(n) for n in ns) + ")  orders")
        for r in out["rows"]:
            print(f"{r['case']:4d}  {r['algorithm']:10s} {r['L']:2d} {r['expected_order']:5d}     "
                  + "  ".join(f"{e:.3e}" for e in r["errors"]) + "   " + "  ".join(f"{o:.2f}" for o in r["orders"]))
    elif argv and argv[0] == "stability":
        n = int(argv[1]) if len(argv) > 1 else 128
        p = int(argv[2]) if len(argv) > 2 else 4
        nsteps = int(argv[3]) if len(argv) > 3 else 600
        for r in stability_sweep(n, p, nsteps=nsteps):
            print(f"{r['algo']} cfl={r['cfl']} dt={r['dt']:.3e} first_nonfinite_by_step={r['first_nonfinite_by_step']} "
                  f"K_last={r['K_last']}")
    else:
        print("usage: python -m paper_2506_03027_gb300.studies paper-vortex [n ...] | stability [n p nsteps]")


if __name__ == "__main__":
    import sys
    _main(sys.argv[1:])
