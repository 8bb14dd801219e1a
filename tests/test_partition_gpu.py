"""A grid split over two processes (the paper's PEs spread over processes, Sec. 3, Alg. 1-3), both on
the one GPU, exchanging boundary strips through the library's exchange callback over a gloo
process group (cfs.torch_exchange: device -> host -> gloo -> host -> device).  No kernel waits on
another process: every exchange happens on the host between launches.  Every point each process computes must equal, bit
for bit, the run of one context computing every sub-domain; the diagnostics of the two processes
must add up to the whole grid's."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(name):
    from paper_2506_03027_gb300 import inputs as I
    algo, kmax, cfl = {"SA": ("SA", 0, 0.25), "CAA": ("CAA", 0, 0.25), "SAA": ("SAA", 3, 0.1)}[name]
    c = I.tgv_case(34, 4, algo)                       # 64 ragged sub-domains (widths 9, 9, 8, 8)
    return c.replace(dt=I.cfl_dt(c, I.tgv_state(c), cfl), kmax=kmax)


def _rank(rank, world, port, name, starts, nsteps, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    from paper_2506_03027_gb300 import build as B
    from paper_2506_03027_gb300 import cfs
    from paper_2506_03027_gb300 import inputs as I
    B.build()
    torch.cuda.set_device(0)
    import datetime
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=180))
    try:
        case = _case(name)
        d = I.saa_delays(case, nsteps) if case.algo == "SAA" else None
        U0 = I.tgv_state(case)
        part = cfs.Solver(case, partition=(world, starts, rank), exchange=cfs.torch_exchange())
        part.set_schedule(delays=d)
        part.set_state(U0)
        part.step(nsteps)
        Up = part.get_state()
        xc = cfs.cfs_exchange_count(part.ctx)
        dp = part.diagnostics()
        part.close()

        full = cfs.Solver(case)
        full.set_schedule(delays=d)
        full.set_state(U0)
        full.step(nsteps)
        Uf = full.get_state()
        df = full.diagnostics()
        full.close()

        # the points of this rank's sub-domains
        mask = np.zeros((case.nz, case.ny, case.nx), dtype=bool)
        for sid in range(starts[rank], starts[rank + 1]):
            ix, iy, iz = sid % case.px, (sid // case.px) % case.py, sid // (case.px * case.py)
            sl = []
            for n, p, i in ((case.nz, case.pz, iz), (case.ny, case.py, iy), (case.nx, case.px, ix)):
                q, rem = divmod(n, p)
                o = i * q + min(i, rem)
                sl.append(slice(o, o + q + (1 if i < rem else 0)))
            mask[tuple(sl)] = True
        same = bool(np.array_equal(Up[:, mask], Uf[:, mask]))
        ndiff = int(np.count_nonzero(Up[:, mask] != Uf[:, mask]))
        out[rank] = (same, ndiff, int(mask.sum()), xc, dp.tolist(), df.tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,starts", [("SA", [0, 32, 64]), ("CAA", [0, 27, 64]), ("SAA", [0, 40, 64])])
def test_two_processes_match_one_context_bit_for_bit(name, starts):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03027_gb300 import build as B
    B.build()                                          # once, before the processes start
    import torch.multiprocessing as mp
    world, nsteps = 2, 10                              # 5 synchronous warm-up steps, then the schedule
    mctx = mp.get_context("spawn")
    with mctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [mctx.Process(target=_rank, args=(r, world, port, name, starts, nsteps, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=600)
        for p in procs:
            if p.is_alive():                           # a rank that failed leaves its peer waiting
                p.terminate()
                p.join(timeout=30)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    npts = 34 ** 3
    assert res[0][2] + res[1][2] == npts
    for r in range(world):
        same, ndiff, _, xc, _, _ = res[r]
        assert same, (r, ndiff)
        # SA steps: one exchange before each of stages 2..5 and each of the 3 filter passes, and
        # the publish at the end of the step; asynchronous steps publish only
        sync_steps = nsteps if name == "SA" else 5
        assert xc == sync_steps * 8 + (nsteps - sync_steps) * 1, xc
    dp0, dp1, df = np.array(res[0][4]), np.array(res[1][4]), np.array(res[0][5])
    np.testing.assert_allclose(dp0[0] + dp1[0], df[0], rtol=1e-12)          # K
    scale = np.abs(df[2:7]).max()
    np.testing.assert_allclose(dp0[2:7] + dp1[2:7], df[2:7], rtol=1e-12, atol=1e-12 * scale)  # totals
    assert dp0[7] == dp1[7] == df[7] == 0.0


def _rank_cgrid(rank, world, port, algo, starts, nsteps, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    from paper_2506_03027_gb300 import build as B
    from paper_2506_03027_gb300 import cfs
    from paper_2506_03027_gb300 import inputs as I
    B.build()
    torch.cuda.set_device(0)
    import datetime
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=180))
    try:
        sp = I.cgrid_reduced()
        mb = I.naca_cgrid(sp, algo=algo, kmax=2)
        mb = mb.replace_all(dt=I.cgrid_dt(mb, 0.2))
        d = I.saa_delays(mb.case.replace(px=mb.nsub, py=1, pz=1), nsteps) if algo == "SAA" else None
        U0 = I.cgrid_state(mb, sp)
        part = cfs.Solver(mb, partition=(world, starts, rank), exchange=cfs.torch_exchange())
        part.set_schedule(delays=d)
        part.set_states(U0)
        part.step(nsteps)
        Up = part.get_states()
        xc = cfs.cfs_exchange_count(part.ctx)
        part.close()
        full = cfs.Solver(mb)
        full.set_schedule(delays=d)
        full.set_states(U0)
        full.step(nsteps)
        Uf = full.get_states()
        full.close()
        same, ndiff, npts, sid0 = True, 0, 0, 0
        for b, up, uf in zip(mb.blocks, Up, Uf):
            mask = np.zeros((b.nz, b.ny, b.nx), dtype=bool)
            for sid in range(sid0, sid0 + b.px * b.py * b.pz):
                if not starts[rank] <= sid < starts[rank + 1]:
                    continue
                loc = sid - sid0
                ix, iy, iz = loc % b.px, (loc // b.px) % b.py, loc // (b.px * b.py)
                sl = []
                for n, p, i in ((b.nz, b.pz, iz), (b.ny, b.py, iy), (b.nx, b.px, ix)):
                    q, rem = divmod(n, p)
                    o = i * q + min(i, rem)
                    sl.append(slice(o, o + q + (1 if i < rem else 0)))
                mask[tuple(sl)] = True
            sid0 += b.px * b.py * b.pz
            same = same and bool(np.array_equal(up[:, mask], uf[:, mask]))
            ndiff += int(np.count_nonzero(up[:, mask] != uf[:, mask]))
            npts += int(mask.sum())
        out[rank] = (same, ndiff, npts, xc, bool(all(np.isfinite(u).all() for u in Uf)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("algo,cut", [("SA", 0.5), ("CAA", 0.6), ("SAA", 0.3)])
def test_connected_grid_two_processes_match_one_context(algo, cut):
    """The 12-block NACA0012 C-grid (reduced size) split between two processes -- interfaces, the
    wake cut, walls and the spanwise interpolation between the layers all crossing the split --
    gives every point bit for bit as one context."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03027_gb300 import build as B
    from paper_2506_03027_gb300 import inputs as I
    B.build()
    nsub = I.naca_cgrid(I.cgrid_reduced()).nsub
    starts = [0, int(round(cut * nsub)), nsub]
    import torch.multiprocessing as mp
    world, nsteps = 2, 10                              # 5 synchronous warm-up steps, then the schedule
    mctx = mp.get_context("spawn")
    with mctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [mctx.Process(target=_rank_cgrid, args=(r, world, port, algo, starts, nsteps, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=600)
        for p in procs:
            if p.is_alive():
                p.terminate()
                p.join(timeout=30)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    mb = I.naca_cgrid(I.cgrid_reduced())
    assert res[0][2] + res[1][2] == sum(b.nx * b.ny * b.nz for b in mb.blocks)
    for r in range(world):
        same, ndiff, _, xc, finite = res[r]
        assert finite
        assert same, (r, ndiff)
        assert xc > 0
