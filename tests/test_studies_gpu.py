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
