"""Failure reporting of bounded device waits, on the GPU without a fault: a kernel waits on an
mbarrier that nothing arrives at, gives up after a poll limit, records it in the context's
status word; the next synchronising call reports CFS_ETIMEOUT once and the context stays usable
(the same path the tensor-core halo network takes when its MMA wait gives up)."""
import numpy as np
import pytest

from paper_2506_03027_gb300 import cfs
from paper_2506_03027_gb300 import inputs as I

from gpu_util import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()


def _run(case, nsteps, check=None):
    s = cfs.Solver(case)
    try:
        s.set_schedule()
        s.set_state(I.tgv_state(case))
        if check is not None:
            check(s)
        s.step(nsteps)
        return s.get_state()
    finally:
        s.close()


def test_wait_that_gives_up_reports_timeout_once():
    c = I.tgv_case(24, 2, "SA")

    def check(s):
        cfs.cfs_wait_check(s.ctx, 1000)
        with pytest.raises(cfs.CfsError) as e:
            s.diagnostics()
        assert e.value.status == cfs.CFS_ETIMEOUT
        d = s.diagnostics()                       # reported once, then cleared
        assert d[7] == 0.0
        cfs.cfs_wait_check(s.ctx, 10)
        with pytest.raises(cfs.CfsError) as e:
            s.get_state()
        assert e.value.status == cfs.CFS_ETIMEOUT

    U = _run(c, 3, check)
    ref = _run(c, 3)
    np.testing.assert_array_equal(U, ref)          # the context stayed usable: same results
