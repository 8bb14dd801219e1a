"""Parameter studies of the asynchronous schemes run through the library.

async_error_vs_delay: the error the asynchrony adds on the translating isentropic vortex under
CAA-AT with the second-order schemes (LSERK2, CD2, AT2: Table 1, case 3) as a function of the
maximum allowable delay L and of the number of sub-domains P (the study of Sec. 5.1 behind its
Fig. 4).  The added error of a run is the RMS difference of its u-velocity from the synchronous
run with the same grid, decomposition and time step, after the same number of steps; the
synchronous run's error against the exact translated vortex is returned beside it.

paper_vortex_errors: the paper's own vortex setup (Sec. 5.1, Table 1, Fig. 2(a)) -- convergence
of the density error over one advection cycle for the six scheme cases, on the GPU.
paper_delay_study: the study of Fig. 4 at the paper's size -- the asynchrony error of CAA-AT
(case 3) on the paper's vortex on 2048^2 points against L at P = 1024 PEs and against P at L = 4.
stability_sweep: the first non-finite step of the Taylor-Green configuration per schedule and CFL.
Command line: python -m paper_2506_03027_gb300.studies paper-vortex [n ...] | stability [n p nsteps] |
delay-study [paper|c1 n t_end cfl]
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


def cubic_fit_full(L, E):
    """Least-squares fit E ~ g0 + g1 L + g2 L^2 + g3 L^3 (a constant for the error the AT buffer
    updates add even at zero delay); returns (g0 .. g3) and the relative RMS residual."""
    L = np.asarray(L, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    A = np.stack([np.ones_like(L), L, L ** 2, L ** 3], axis=1)
    g, *_ = np.linalg.lstsq(A, E, rcond=None)
    return g, float(np.sqrt(np.mean((A @ g - E) ** 2)) / np.sqrt(np.mean(E ** 2)))


def paper_delay_study(n: int = 2048, Ls=(1, 2, 3, 4, 5, 6, 7, 8), Ps=(16, 64, 256, 1024, 4096), P_fixed: int = 1024,
                      L_fixed: int = 4, t_end: float = 4.0, cfl: float = 0.1, vortex: str = "paper") -> dict:
    """Fig. 4 of the paper: the u-velocity error the asynchrony adds under CAA-AT with the
    second-order schemes (LSERK2, CD2, AT2: Table 1 case 3) on an advected vortex with a
    two-dimensional decomposition into P = p x p PEs, after t_end -- (a) against the maximum
    allowable delay L at P = P_fixed, (b) against P at L = L_fixed.  vortex "paper": the Gaussian
    vortex of Sec. 5.1 (beta 0.02, M 0.1, periodic [-8, 8]^2); "c1": the isentropic vortex of
    strength 5 at M 0.5 on [-5, 5]^2.  The added error of a run is the RMS difference of its
    u-velocity from the synchronous run (one run: SA with P sub-domains equals the single-domain
    run to rounding for every P); the synchronous run's error against the exact solution is
    returned beside it.  The time step is that of CFL `cfl` (the paper's own steps, CFL about 0.04,
    would take 136 k steps per run at 2048^2); a run that goes non-finite reports NaN and stays
    out of the fits; CUDA-graph mode."""
    import torch
    paper = vortex == "paper"
    state = I.paper_vortex_state if paper else I.vortex_state

    def case(P, algo, L):
        p = int(round(math.sqrt(P)))
        assert p * p == P, P
        if paper:
            c = I.paper_vortex_case(n, order=2, algo=algo, at=True, L=L).replace(px=p, py=p)
        else:
            c = I.vortex_case(n, p, order=2, algo=algo, at=True, caa_L=L, kmax=max(0, L - 1))
        dt = I.cfl_dt(c, state(c), cfl)
        nsteps = int(math.ceil(t_end / dt))
        return c.replace(dt=t_end / nsteps), nsteps

    def run(c, nsteps):
        U0 = state(c)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            s = cfs.Solver(c, max_delay=0 if c.algo == "SA" else c.caa_L - 1, graph=True, stream=st)
            try:
                s.set_schedule()
                s.set_state(U0)
                s.step(nsteps)
                return s.get_state()
            finally:
                s.close()

    c_sa, nsteps = case(P_fixed, "SA", 8)
    Usa = run(c_sa, nsteps)
    exact = state(c_sa, t=t_end)
    out = {"vortex": vortex, "n": n, "t_end": t_end, "steps": nsteps, "dt": c_sa.dt, "cfl": cfl,
           "sa_error": float(math.sqrt(np.mean((_u(Usa) - _u(exact)) ** 2))),
           "P_fixed": P_fixed, "L": [], "error_vs_L": [], "L_fixed": L_fixed, "P": [], "error_vs_P": []}

    def added(P, L):
        c, ns = case(P, "CAA", L)
        assert ns == nsteps
        U = run(c, ns)
        return float(math.sqrt(np.mean((_u(U) - _u(Usa)) ** 2)))

    for L in Ls:
        out["L"].append(int(L))
        out["error_vs_L"].append(added(P_fixed, int(L)))
    for P in Ps:
        out["P"].append(int(P))
        out["error_vs_P"].append(out["error_vs_L"][out["L"].index(L_fixed)] if P == P_fixed and L_fixed in out["L"]
                                 else added(int(P), L_fixed))
    okL = [i for i, e in enumerate(out["error_vs_L"]) if math.isfinite(e)]
    g, res = cubic_fit_full([out["L"][i] for i in okL], [out["error_vs_L"][i] for i in okL])
    out["cubic_fit_L"] = {"g0_g1_g2_g3": [float(v) for v in g], "relative_rms_residual": res,
                          "points": len(okL)}
    okP = [i for i, e in enumerate(out["error_vs_P"]) if math.isfinite(e)]
    Pv = np.array([out["P"][i] for i in okP], dtype=np.float64)
    Ev = np.array([out["error_vs_P"][i] for i in okP])
    A = np.stack([Pv, np.ones_like(Pv)], axis=1)
    ab, *_ = np.linalg.lstsq(A, Ev, rcond=None)
    out["linear_fit_P"] = {"slope": float(ab[0]), "intercept": float(ab[1]),
                           "relative_rms_residual": float(np.sqrt(np.mean((A @ ab - Ev) ** 2)) / np.sqrt(np.mean(Ev ** 2)))}
    out["loglog_slope_P"] = float(np.polyfit(np.log(Pv), np.log(Ev), 1)[0])
    return out


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
    elif argv and argv[0] == "delay-study":
        vortex = argv[1] if len(argv) > 1 else "paper"
        n = int(argv[2]) if len(argv) > 2 else 2048
        t_end = float(argv[3]) if len(argv) > 3 else 4.0
        cfl = float(argv[4]) if len(argv) > 4 else 0.1
        out = paper_delay_study(n, t_end=t_end, cfl=cfl, vortex=vortex)
        print(json.dumps(out))
        print(f"{vortex} vortex, n = {n}, t = {t_end}, {out['steps']} steps of dt = {out['dt']:.3e} (CFL {cfl}); "
              f"SA error against the exact solution {out['sa_error']:.3e}")
        print(f"(a) P = {out['P_fixed']}:  L  added error")
        for L, e in zip(out["L"], out["error_vs_L"]):
            print(f"    {L:2d}  {e:.4e}")
        cf = out["cubic_fit_L"]
        print(f"    cubic fit g0 + g1 L + g2 L^2 + g3 L^3 over {cf['points']} finite points: g = "
              + ", ".join(f"{v:.3e}" for v in cf["g0_g1_g2_g3"]) + f"; relative residual {cf['relative_rms_residual']:.3f}")
        print(f"(b) L = {out['L_fixed']}:  P  added error")
        for P, e in zip(out["P"], out["error_vs_P"]):
            print(f"    {P:5d}  {e:.4e}")
        lf = out["linear_fit_P"]
        print(f"    linear fit a P + b: a = {lf['slope']:.4e}, b = {lf['intercept']:.4e}, relative residual "
              f"{lf['relative_rms_residual']:.3f}; log-log slope {out['loglog_slope_P']:.3f}")
    else:
        print("usage: python -m paper_2506_03027_gb300.studies paper-vortex [n ...] | stability [n p nsteps] | "
              "delay-study [paper|c1 n t_end cfl]")


if __name__ == "__main__":
    import sys
    _main(sys.argv[1:])
