"""The asynchrony error of CAA-AT (LSERK2-CD2-AT2, Table 1 case 3) on the translating vortex
grows with the maximum allowable delay L faster than linearly, as the error estimate of the AT
schemes (a polynomial in the moments of the delay) predicts -- the study behind Fig. 4."""
import numpy as np
import pytest

from gpu_util import ensure_built

pytestmark = pytest.mark.gpu


def test_async_error_grows_with_the_delay():
    ensure_built()
    from paper_2506_03027_gb300 import studies
    r = studies.async_error_vs_delay(256, 8, (1, 2, 3, 4, 6), t_end=0.5)
    E = np.array(r["async_error"])
    print(r)
    assert np.all(np.isfinite(E)) and np.all(E > 0)
    assert np.all(np.diff(E) > 0), E                  # monotone in L
    assert E[4] / E[2] >= 4.0, E                      # L 3 -> 6: at least quadratic
    assert E[-1] < 0.1 * r["sa_error"], r             # asynchrony error stays below the scheme's own
    g, res = studies.cubic_fit(r["L"], E)
    assert res < 0.1, (g, res)                        # a cubic in L describes it


def test_paper_vortex_orders_of_table1():
    """The paper's own vortex test (Sec. 5.1): one advection cycle of the Gaussian vortex with
    three PEs at the paper's time steps, SAA delays from the arrival model of Alg. 3.  Between
    n = 120 and 240 the density error falls at the orders Table 1 states -- 2 for SA, CAA-AT and
    SAA-AT with LSERK2/CD2/AT2 (L = 8), 4 for SA and CAA-AT (L = 8) and SAA-AT (L = 4) with
    LSERK4/CD4/AT4 -- and the standard schemes on delayed data (AS, L = 8) leave a larger error
    than AT."""
    ensure_built()
    from paper_2506_03027_gb300 import studies
    runs = ((1, "SA", 8), (2, "CAA", 8), (2, "SAA", 8), (3, "CAA", 8), (3, "SAA", 8), (4, "SA", 8),
            (6, "CAA", 8), (6, "SAA", 4))
    r = studies.paper_vortex_errors(ns=(120, 240), runs=runs, seeds=(1, 2))
    print(r)
    by = {(row["case"], row["algorithm"]): row for row in r["rows"]}
    for (case, algo), row in by.items():
        assert np.all(np.isfinite(row["errors"])), row
        if row["expected_order"] > 1:
            assert row["orders"][0] >= row["expected_order"] - 0.4, row
    for algo in ("CAA", "SAA"):
        assert by[(2, f"{algo}-AS")]["errors"][-1] > 3.0 * by[(3, f"{algo}-AT")]["errors"][-1], algo


def test_async_error_grows_with_the_number_of_pes():
    """The paper's vortex under CAA-AT (case 3) split into P = p x p PEs: the added error grows with
    P at fixed L and with L at fixed P (Fig. 4 (b) and (a), at a small size)."""
    ensure_built()
    from paper_2506_03027_gb300 import studies
    r = studies.paper_delay_study(n=256, Ls=(2, 4), Ps=(4, 16, 64), P_fixed=16, L_fixed=4, t_end=0.5)
    print(r)
    EL, EP = np.array(r["error_vs_L"]), np.array(r["error_vs_P"])
    assert np.all(np.isfinite(EL)) and np.all(EL > 0) and np.all(np.isfinite(EP)) and np.all(EP > 0)
    assert np.all(np.diff(EL) > 0), EL
    assert np.all(np.diff(EP) > 0), EP


# ------------------------------------------------------------------ parity at the study configurations

def _check(Ug, Uo):
    from gpu_util import PARITY_TOL, rel_l2, rel_l2_per_component
    e = rel_l2(Ug, Uo)
    assert np.all(np.isfinite(Ug))
    assert np.all(e <= PARITY_TOL), (e, rel_l2_per_component(Ug, Uo))


@pytest.mark.parametrize("L", [4, 8])
def test_study_vortex_caa_parity(L):
    """The configuration of the delay study (Sec. 5.1, Fig. 4) against the oracle, whole fields:
    the translating vortex with LSERK2-CD2-AT2 (Table 1 case 3) under CAA-AT with maximum
    allowable delay L, 64^2 on 4 x 4 sub-domains of 16^2, CFL 0.2, 60 steps (the first 3
    synchronous)."""
    ensure_built()
    from gpu_util import gpu_run
    from oracle import oracle as orc
    from paper_2506_03027_gb300 import inputs as I
    base = I.vortex_case(64, 4, order=2)
    c = base.replace(dt=I.cfl_dt(base, I.vortex_state(base), 0.2), algo="CAA", at=True, caa_L=L, kmax=L - 1)
    U0 = I.vortex_state(c)
    Ug, _ = gpu_run(c, U0, 60)
    Uo = orc.run(c, U0, 60)
    _check(Ug, Uo)


@pytest.mark.parametrize("order,algo,at,L,nsteps", [(2, "SAA", True, 8, 60), (2, "CAA", False, 8, 60),
                                                    (4, "SAA", True, 4, 60), (4, "CAA", True, 8, 20),
                                                    (2, "SAA", False, 8, 60)])
def test_paper_vortex_parity(order, algo, at, L, nsteps):
    """The paper's own vortex test (Sec. 5.1) against the oracle, whole fields: the Gaussian
    vortex on [-8, 8]^2, 60^2 points on the three PEs of the paper, its time steps, Table 1 cases
    2, 3 and 6 under CAA with L = 8 and SAA with delays from the arrival model of Alg. 3
    (consecutive visible levels, reset at L); 60 steps.  LSERK4-AT4 under CAA with L = 8 (delays up
    to 7, whose five-level extrapolation weights amplify rounding) runs 20 steps -- every delay
    0..7 occurs from step 5 on: the oracle alone spreads a one-ulp change of the initial state to
    8e-14 after 20 steps but to 1.2e-12 after 60, so no two FP64 evaluation orders agree to 1e-12
    over the longer window."""
    ensure_built()
    from gpu_util import gpu_run
    from oracle import oracle as orc
    from paper_2506_03027_gb300 import inputs as I
    c = I.paper_vortex_case(60, order=order, algo=algo, at=at, L=L)
    d = I.saa_delays_arrival(c, nsteps, L, seed=1) if algo == "SAA" else None
    U0 = I.paper_vortex_state(c)
    Ug, _ = gpu_run(c, U0, nsteps, delays=d, max_delay=L - 1)
    Uo = orc.run(c, U0, nsteps, delays=d)
    _check(Ug, Uo)
