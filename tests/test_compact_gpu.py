"""The sixth-order compact scheme (Eq. 2 with alpha = 1/3, explicit sixth-order closure at the first
halo point of every sub-domain line) on the GPU against the FP64 oracle, whole fields at 1e-12:
the 2-D vortex and a ragged 3-D Euler Taylor-Green field under SA, CAA-AT and SAA-AT, with and
without the filter, and the CUDA-graph replay against the step-by-step launches."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2506_03027_gb300 import cfs
from paper_2506_03027_gb300 import inputs as I

from gpu_util import PARITY_TOL, ensure_built, gpu_run, rel_l2, rel_l2_per_component

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()


def check(U, ref, tol=PARITY_TOL):
    e = rel_l2(U, ref)
    assert np.all(np.isfinite(U))
    assert np.all(e <= tol), (e, rel_l2_per_component(U, ref))


def test_compact_vortex_parity():
    """2-D translating vortex, Euler, 64^2 on 2 x 2 sub-domains, SA, CFL 0.4, 100 steps."""
    c = I.vortex_case(64, 2, compact=1)
    c = c.replace(dt=I.cfl_dt(c, I.vortex_state(c), 0.4))
    U0 = I.vortex_state(c)
    Ug, _ = gpu_run(c, U0, 100)
    check(Ug, orc.run(c, U0, 100))


@pytest.mark.parametrize("algo,kmax,cfl,filt", [("SA", 0, 0.25, True), ("CAA", 0, 0.25, True),
                                                ("SAA", 1, 0.1, False), ("SAA", 2, 0.1, True)])
def test_compact_tgv_euler_ragged_parity(algo, kmax, cfl, filt):
    """3-D Euler Taylor-Green field on 34^3 points over 4^3 ragged sub-domains (9, 9, 8, 8), 20
    steps (5 synchronous, then the schedule; CAA with L = 4)."""
    c = I.tgv_case(34, 4, algo, viscous=False, filter=filt, compact=1, kmax=kmax)
    c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), cfl))
    d = I.saa_delays(c, 20) if algo == "SAA" else None
    U0 = I.tgv_state(c)
    Ug, _ = gpu_run(c, U0, 20, delays=d)
    check(Ug, orc.run(c, U0, 20, delays=d))


def test_compact_graph_replay_is_identical():
    import torch
    c = I.tgv_case(32, 2, "SAA", viscous=False, filter=True, compact=1, kmax=2)
    c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), 0.1))
    d = I.saa_delays(c, 12)
    out = []
    for graph in (False, True):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            s = cfs.Solver(c, graph=graph, stream=st)
            try:
                s.set_schedule(delays=d)
                s.set_state(I.tgv_state(c))
                s.step(12)
                out.append(s.get_state())
            finally:
                s.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_compact_rejects_unsupported_configurations():
    c = I.tgv_case(16, 2, "SA", filter=False, compact=1)            # viscous
    with pytest.raises(cfs.CfsError):
        cfs.Solver(c)
