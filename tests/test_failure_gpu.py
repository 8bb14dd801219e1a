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


# ------------------------------------------------------------------ partitioned contexts
# Failures made on the host: a transport that raises, a peer process that is gone.  No kernel
# waits on another process, so nothing waits on the GPU.

def _part_case():
    c = I.tgv_case(16, 2, "SA")                       # 8 sub-domains, synchronous: an exchange per stage
    return c.replace(dt=I.cfl_dt(c, I.tgv_state(c), 0.25))


def test_failing_transport_reports_exchange_and_keeps_the_context():
    case = _part_case()

    def broken(nranks, send, scnt, recv, rcnt, stream):
        raise RuntimeError("the link to the peer is down")

    s = cfs.Solver(case, partition=(2, [0, 4, 8], 0), exchange=broken)
    try:
        s.set_schedule()
        s.set_state(I.tgv_state(case))
        with pytest.raises(cfs.CfsError) as e:
            s.step(1)
        assert e.value.status == cfs.CFS_EXCHANGE
        U = s.get_state()                              # the context still answers
        assert np.all(np.isfinite(U))
    finally:
        s.close()


def test_step_without_a_transport_is_refused():
    case = _part_case()
    s = cfs.Solver(case, partition=(2, [0, 4, 8], 0))
    try:
        s.set_schedule()
        s.set_state(I.tgv_state(case))
        with pytest.raises(cfs.CfsError) as e:
            s.step(1)
        assert e.value.status == cfs.CFS_ESTATE
    finally:
        s.close()


def _gone_peer_rank(rank, port, out):
    import datetime
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from paper_2506_03027_gb300 import build as B
    from paper_2506_03027_gb300 import cfs as C
    from paper_2506_03027_gb300 import inputs as J
    B.build()
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2,
                            timeout=datetime.timedelta(seconds=15))
    if rank == 1:
        os._exit(0)                                    # leaves before its first step, nothing in flight
    c = J.tgv_case(16, 2, "SA")
    c = c.replace(dt=J.cfl_dt(c, J.tgv_state(c), 0.25))
    s = C.Solver(c, partition=(2, [0, 4, 8], 0), exchange=C.torch_exchange())
    try:
        s.set_schedule()
        s.set_state(J.tgv_state(c))
        try:
            s.step(1)
            out[0] = "stepped"
        except C.CfsError as e:
            out[0] = e.status
        out[1] = bool(np.all(np.isfinite(s.get_state())))
    finally:
        s.close()
    os._exit(0)


def test_peer_that_is_gone_ends_the_exchange_with_an_error():
    """Rank 1 joins the process group and leaves before its first step; rank 0's first exchange
    (gloo, 15 s timeout) fails on the host, cfs_step reports CFS_EXCHANGE, the context stays usable."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mctx = mp.get_context("spawn")
    with mctx.Manager() as mgr:
        out = mgr.dict()
        procs = [mctx.Process(target=_gone_peer_rank, args=(r, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
        for p in procs:
            if p.is_alive():
                p.terminate()
                p.join(timeout=30)
        res = dict(out)
    assert res.get(0) == cfs.CFS_EXCHANGE, res
    assert res.get(1) is True, res
