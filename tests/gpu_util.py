"""Helpers shared by the GPU tests: run the CUDA library through its C ABI binding, compare with
the oracle."""
import numpy as np

from paper_2506_03027_gb300 import build as B
from paper_2506_03027_gb300 import cfs

PARITY_TOL = 1e-12  # relative L2 per conserved variable, FP64 path vs FP64 oracle


def ensure_built():
    B.build()
    cfs.load()


def gpu_run(case, U0, nsteps, delays=None, precision=0, max_delay=None):
    s = cfs.Solver(case, precision=precision, max_delay=max_delay)
    try:
        s.set_schedule(delays=delays)
        s.set_state(U0)
        s.step(nsteps)
        U = s.get_state()
        d = s.diagnostics(check_finite=False)
    finally:
        s.close()
    return U, d


def rel_l2(a, ref):
    """Relative L2 error per conserved variable.  A variable whose reference norm is tiny compared
    with the momentum scale (rho w of a 2-D run) is measured against 1e-6 of that scale."""
    mom = max(np.linalg.norm(ref[v]) for v in (1, 2, 3))
    out = []
    for v in range(5):
        den = max(np.linalg.norm(ref[v]), 1e-6 * mom if v in (1, 2, 3) else 0.0)
        num = np.linalg.norm(a[v] - ref[v])
        out.append(num / den if den > 0 else num)
    return np.array(out)
