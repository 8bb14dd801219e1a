"""No value the library did not write reaches a result: every configuration runs twice, with
every device allocation of the context filled with 0xff bytes (NaN in FP32 and FP64) and with
zeros, and the two states agree bit for bit.  (Device memory from PyTorch's caching allocator
keeps whatever a previous user left, so a read before a write shows up only with some histories.)"""
import numpy as np
import pytest

from paper_2506_03027_gb300 import cfs
from paper_2506_03027_gb300 import inputs as I

from gpu_util import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    return torch


def _tgv(n, p, algo, **kw):
    c = I.tgv_case(n, p, algo, **kw)
    return c.replace(dt=I.cfl_dt(c, I.tgv_state(c), 0.1))


def _cgrid(algo):
    mb = I.naca_cgrid(I.cgrid_reduced(), algo=algo)
    mb = mb.replace_all(dt=I.cgrid_dt(mb, 0.05))
    return mb.replace_all(caa_L=3, kmax=2) if algo == "CAA" else mb


CONFIGS = {
    "tgv_fp64_saa": dict(case=lambda: _tgv(34, 4, "SAA")),
    "tgv_fp64_saa_graph": dict(case=lambda: _tgv(34, 4, "SAA"), graph=True),
    "tgv_fp32_caa_fused_subdomain_filter": dict(case=lambda: _tgv(32, 2, "CAA"), precision=1),
    "tgv_fp32_saa_ragged_graph": dict(case=lambda: _tgv(34, 4, "SAA"), precision=1, graph=True),
    "euler_compact_caa": dict(case=lambda: _tgv(32, 2, "CAA", viscous=False, compact=1)),
    "curvilinear_fp32_caa": dict(case=lambda: _tgv(26, 2, "CAA", curv=0.25), precision=1),
    "learned_saa": dict(case=lambda: _tgv(64, 2, "SAA", kmax=4), learned=True),
    "cgrid_fp64_saa": dict(mb=lambda: _cgrid("SAA")),
    "cgrid_fp32_caa": dict(mb=lambda: _cgrid("CAA"), precision=1),
    "cgrid_fp32_saa_graph": dict(mb=lambda: _cgrid("SAA"), precision=1, graph=True),
}


def _run(torch, case=None, mb=None, precision=0, graph=False, learned=False, nst=10):
    from paper_2506_03027_gb300 import learned as L
    if mb is not None:
        m = mb()
        U0 = I.cgrid_state(m, I.cgrid_reduced())
        d = I.saa_delays(m.case.replace(px=m.nsub, py=1, pz=1), nst) if m.case.algo == "SAA" else None
    else:
        c = case()
        U0 = I.tgv_state(c)
        d = I.saa_delays(c, nst) if c.algo == "SAA" else None
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        if mb is not None:
            s = cfs.Solver(m, precision=precision, graph=graph, stream=st)
        else:
            s = cfs.Solver(c, precision=precision, graph=graph, stream=st, max_delay=4 if learned else None)
        try:
            s.set_schedule(delays=d)
            if learned:
                scales = np.array([3e3, 2e3, 2e3, 2e3, 1e3, 4e2, 3e2, 3e2, 3e2, 2e2, 1e7, 1e6, 1e6, 1e6, 5e5])
                cfs.cfs_set_halo_model(s.ctx, L.init_params(1), scales)
            if mb is not None:
                s.set_states(U0)
            else:
                s.set_state(U0)
            s.step(nst)
            out = s.get_states() if mb is not None else [s.get_state()]
        finally:
            s.close()
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_no_read_of_unwritten_device_memory(torch, monkeypatch, name):
    orig = cfs.TorchAllocator._alloc
    fill = {"v": 0}

    def filled(self, nbytes, user):
        ptr = orig(self, nbytes, user)
        if ptr:
            self.live[ptr].fill_(fill["v"])
        return ptr

    monkeypatch.setattr(cfs.TorchAllocator, "_alloc", filled)
    res = {}
    for v in (0, 255):
        fill["v"] = v
        res[v] = _run(torch, **CONFIGS[name])
    for a, b in zip(res[0], res[255]):
        assert np.all(np.isfinite(b))
        np.testing.assert_array_equal(a, b)


def test_contexts_alive_together_give_their_own_bits(torch):
    """Three contexts of different kinds -- the FP64 TGV path, the FP32 fused stage with the
    sub-domain filter, the FP32 C-grid -- created together and stepped alternately, each on its own
    stream, give the bits each gives alone (no state shared between contexts)."""
    cases = [dict(case=lambda: _tgv(34, 4, "SAA")),
             dict(case=lambda: _tgv(32, 2, "CAA"), precision=1),
             dict(mb=lambda: _cgrid("SAA"), precision=1)]
    nst = 8
    alone = [_run(torch, nst=nst, **kw) for kw in cases]
    solvers, streams = [], []
    try:
        for kw in cases:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                if "mb" in kw:
                    m = kw["mb"]()
                    s = cfs.Solver(m, precision=kw.get("precision", 0), stream=st)
                    s.set_schedule(delays=I.saa_delays(m.case.replace(px=m.nsub, py=1, pz=1), nst))
                    s.set_states(I.cgrid_state(m, I.cgrid_reduced()))
                else:
                    c = kw["case"]()
                    s = cfs.Solver(c, precision=kw.get("precision", 0), stream=st)
                    s.set_schedule(delays=I.saa_delays(c, nst) if c.algo == "SAA" else None)
                    s.set_state(I.tgv_state(c))
            solvers.append(s)
            streams.append(st)
        for _ in range(nst):
            for s, st in zip(solvers, streams):
                with torch.cuda.stream(st):
                    s.step(1)
        together = []
        for s, st, kw in zip(solvers, streams, cases):
            with torch.cuda.stream(st):
                together.append(s.get_states() if "mb" in kw else [s.get_state()])
    finally:
        for s in solvers:
            s.close()
    for a_list, b_list in zip(alone, together):
        for a, b in zip(a_list, b_list):
            np.testing.assert_array_equal(a, b)


def test_repeated_contexts_leave_no_device_memory(torch):
    """Contexts created, stepped as CUDA graphs and destroyed over and over return their memory:
    PyTorch's count of allocated bytes comes back to its start, and the device's free memory stays
    level after the first round (graph executables, events, tables)."""
    c = _tgv(32, 2, "CAA")
    U0 = I.tgv_state(c)
    torch.cuda.synchronize()
    base_alloc = torch.cuda.memory_allocated()
    free = []
    for it in range(12):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            s = cfs.Solver(c, precision=it % 2, graph=True, stream=st)
            try:
                s.set_schedule()
                s.set_state(U0)
                s.step(3)
                s.diagnostics()
            finally:
                s.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base_alloc
        torch.cuda.empty_cache()  # the caching allocator keeps freed blocks per stream
        free.append(torch.cuda.mem_get_info()[0])
    assert max(free[2:]) - min(free[2:]) < (64 << 20), [f - free[2] for f in free]
