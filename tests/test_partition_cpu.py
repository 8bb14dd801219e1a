"""Host logic of partitioned contexts (the paper's PEs spread over processes, Sec. 3 and Alg. 1-3),
without a GPU: the exchange plans the library derives, checked against a brute-force enumeration of
what each sub-domain's stencils read, and an exchange of strips between two gloo ranks on CPU that
leaves every value the own sub-domains read equal to the whole grid's."""
import os
import socket

import numpy as np
import pytest

from paper_2506_03027_gb300 import build as B
from paper_2506_03027_gb300 import cfs
from paper_2506_03027_gb300 import inputs as I


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    return cfs.load()


def split(n, p, i):
    """Origin and length of part i of n points split into p parts, the first n mod p one longer."""
    q, rem = divmod(n, p)
    return i * q + min(i, rem), q + (1 if i < rem else 0)


def context(case, starts, rank):
    ctx = cfs.cfs_create(cfs.params_from_case(case), None)
    cfs.describe_blocks(ctx, [case])
    cfs.cfs_set_partition(ctx, len(starts) - 1, starts, rank)
    return ctx


def read_set(case, sid):
    """Every point sub-domain sid reads from beyond its faces, by brute force: the view halo
    (faces to the halo depth G = 2r viscous / r Euler, viscous edges to r x r) and the filter
    lines (faces to depth 5) -- as global offsets (wrapped periodically)."""
    r = 2 if case.order == 4 else 1
    G = 2 * r if case.viscous else r
    D = max(G, 5) if case.filter else G
    px, py, pz = case.px, case.py, case.pz
    ix, iy, iz = sid % px, (sid // px) % py, sid // (px * py)
    o, s = zip(split(case.nx, px, ix), split(case.ny, py, iy), split(case.nz, pz, iz))
    n = (case.nx, case.ny, case.nz)
    three_d = case.nz > 1
    dep = (D, D, D if three_d else 0)
    out = set()
    for k in range(-dep[2], s[2] + dep[2]):
        for j in range(-dep[1], s[1] + dep[1]):
            for i in range(-dep[0], s[0] + dep[0]):
                c = (i, j, k)
                d = [(-c[a] if c[a] < 0 else (c[a] - s[a] + 1 if c[a] >= s[a] else 0)) for a in range(3)]
                nout = sum(x > 0 for x in d)
                if nout == 0 or nout == 3:
                    continue
                if nout == 2 and not (case.viscous and max(d) <= r):
                    continue
                g = [(o[a] + c[a]) % n[a] for a in range(3)]
                out.add(g[0] + n[0] * (g[1] + n[1] * g[2]))
    return out


def owner_of(case):
    """Sub-domain of every global point."""
    own = np.empty((case.nz, case.ny, case.nx), dtype=np.int64)
    for iz in range(case.pz):
        oz, sz = split(case.nz, case.pz, iz)
        for iy in range(case.py):
            oy, sy = split(case.ny, case.py, iy)
            for ix in range(case.px):
                ox, sx = split(case.nx, case.px, ix)
                own[oz:oz + sz, oy:oy + sy, ox:ox + sx] = ix + case.px * (iy + case.py * iz)
    return own.reshape(-1)


CASES = {
    "ns_filter_3d": I.tgv_case(24, 2, "SAA", filter=True).replace(nx=26, ny=20, nz=16, px=3, py=2, pz=2),
    "euler_cd2_3d": I.tgv_case(20, 2, "CAA", viscous=False, order=2, filter=False).replace(px=3),
    "vortex_2d": I.vortex_case(48, 3, filter=True, algo="SAA", kmax=2),
    "ns_filter_3d_wide": I.tgv_case(24, 2, "SAA", filter=True).replace(nx=40, ny=32, nz=24, px=2, py=2, pz=1),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("nranks", [2, 3])
def test_plan_matches_brute_force_read_sets(name, nranks):
    case = CASES[name]
    nsub = case.nsub
    starts = [round(q * nsub / nranks) for q in range(nranks + 1)]
    own = owner_of(case)
    rank_of = np.searchsorted(np.array(starts[1:]), np.arange(nsub), side="right")
    reads = [read_set(case, s) for s in range(nsub)]
    plans = {}
    for p in range(nranks):
        ctx = context(case, starts, p)
        try:
            for q in range(nranks):
                plans[p, q, 0] = cfs.cfs_exchange_plan(ctx, q, 0)
                plans[p, q, 1] = cfs.cfs_exchange_plan(ctx, q, 1)
        finally:
            cfs.cfs_destroy(ctx)
    for p in range(nranks):
        mine = set().union(*[reads[s] for s in range(nsub) if rank_of[s] == p])
        for q in range(nranks):
            expect = sorted(x for x in mine if rank_of[own[x]] == q) if q != p else []
            assert list(plans[p, q, 1]) == expect, (p, q)
            # what p sends to q is what q receives from p, in the same order
            np.testing.assert_array_equal(plans[p, q, 0], plans[q, p, 1])
    assert any(len(plans[0, q, 1]) for q in range(1, nranks))


def cgrid_read_sets(mb, ctx):
    """Read sets of every sub-domain of a connected grid, in sub-domain order: as read_set, with
    every point beyond a non-periodic block face replaced by the sources of its gather entry
    (cfs_halo_sources: interface neighbours, wall mirror points, outflow face points; a far field
    has none) -- as state offsets (5 x the points of the blocks before, plus the point index)."""
    c0 = mb.case
    r = 2 if c0.order == 4 else 1
    G = 2 * r if c0.viscous else r
    D = max(G, 5) if c0.filter else G
    base = 5 * np.concatenate([[0], np.cumsum([b.nx * b.ny * b.nz for b in mb.blocks])])
    sets = []
    for bi, b in enumerate(mb.blocks):
        n = (b.nx, b.ny, b.nz)
        per = [(mb.faces[bi][2 * a].type == "periodic", mb.faces[bi][2 * a + 1].type == "periodic") for a in range(3)]
        dep = (D, D, D if b.nz > 1 else 0)
        for iz in range(b.pz):
            for iy in range(b.py):
                for ix in range(b.px):
                    o, s = zip(split(b.nx, b.px, ix), split(b.ny, b.py, iy), split(b.nz, b.pz, iz))
                    out = set()
                    for k in range(-dep[2], s[2] + dep[2]):
                        for j in range(-dep[1], s[1] + dep[1]):
                            for i in range(-dep[0], s[0] + dep[0]):
                                c = (i, j, k)
                                d = [(-c[a] if c[a] < 0 else (c[a] - s[a] + 1 if c[a] >= s[a] else 0)) for a in range(3)]
                                nout = sum(x > 0 for x in d)
                                if nout == 0 or nout == 3:
                                    continue
                                if nout == 2 and not (c0.viscous and max(d) <= r):
                                    continue
                                g = [o[a] + c[a] for a in range(3)]
                                if any((g[a] < 0 and not per[a][0]) or (g[a] >= n[a] and not per[a][1]) for a in range(3)):
                                    for sb, si, sj, sk, _, _, _ in cfs.cfs_halo_sources(ctx, bi, *g)[1]:
                                        B2 = mb.blocks[sb]
                                        out.add(int(base[sb]) + si + B2.nx * (sj + B2.ny * sk))
                                else:
                                    g = [g[a] % n[a] for a in range(3)]
                                    out.add(int(base[bi]) + g[0] + n[0] * (g[1] + n[1] * g[2]))
                    sets.append(out)
    return sets


@pytest.mark.parametrize("nranks", [2, 3])
def test_plan_on_a_connected_grid(nranks):
    """The 12-block C-grid (reduced size: interfaces with reversed and non-matching spanwise
    neighbours, walls, far field, outflows): the plan equals the brute-force read sets with the
    gather sources of the points beyond the block faces, and both sides of a pair agree."""
    mb = I.naca_cgrid(I.cgrid_reduced())
    nsub = sum(b.px * b.py * b.pz for b in mb.blocks)
    starts = [round(q * nsub / nranks) for q in range(nranks + 1)]
    # sub-domain of every state offset of variable 0 (a block's points follow its 5 x points base)
    own = np.full(5 * sum(b.nx * b.ny * b.nz for b in mb.blocks), -1, dtype=np.int64)
    base, sid0 = 0, 0
    for b in mb.blocks:
        npb = b.nx * b.ny * b.nz
        own[base:base + npb] = owner_of(b) + sid0
        base += 5 * npb
        sid0 += b.px * b.py * b.pz
    rank_of = np.searchsorted(np.array(starts[1:]), np.arange(nsub), side="right")
    plans = {}
    reads = None
    for p in range(nranks):
        ctx = cfs.cfs_create(cfs.params_from_case(mb.case), None)
        try:
            cfs.describe_blocks(ctx, mb.blocks, mb)
            cfs.cfs_set_partition(ctx, nranks, starts, p)
            if reads is None:
                reads = cgrid_read_sets(mb, ctx)
            for q in range(nranks):
                plans[p, q, 0] = cfs.cfs_exchange_plan(ctx, q, 0)
                plans[p, q, 1] = cfs.cfs_exchange_plan(ctx, q, 1)
        finally:
            cfs.cfs_destroy(ctx)
    assert len(reads) == nsub
    crossing = 0
    for p in range(nranks):
        mine = set().union(*[reads[s] for s in range(nsub) if rank_of[s] == p])
        for q in range(nranks):
            expect = sorted(x for x in mine if rank_of[own[x]] == q) if q != p else []
            assert list(plans[p, q, 1]) == expect, (p, q)
            np.testing.assert_array_equal(plans[p, q, 0], plans[q, p, 1])
            crossing += len(expect)
    assert crossing > 0


def test_plan_with_a_process_that_computes_nothing():
    """starts = [0, 5, 5, 12]: the middle process owns no sub-domain, so it reads nothing and
    nobody reads from it; the two others exchange as in a two-process split."""
    case = CASES["ns_filter_3d"]
    starts = [0, 5, 5, 12]
    plans = {}
    for p in range(3):
        ctx = context(case, starts, p)
        try:
            for q in range(3):
                plans[p, q, 0] = cfs.cfs_exchange_plan(ctx, q, 0)
                plans[p, q, 1] = cfs.cfs_exchange_plan(ctx, q, 1)
        finally:
            cfs.cfs_destroy(ctx)
    for q in range(3):
        assert len(plans[1, q, 0]) == 0 and len(plans[1, q, 1]) == 0
        assert len(plans[q, 1, 0]) == 0 and len(plans[q, 1, 1]) == 0
    two = {}
    for p, r in ((0, 0), (2, 1)):
        ctx = context(case, [0, 5, 12], r)
        try:
            two[p] = (cfs.cfs_exchange_plan(ctx, 1 - r, 0), cfs.cfs_exchange_plan(ctx, 1 - r, 1))
        finally:
            cfs.cfs_destroy(ctx)
    np.testing.assert_array_equal(plans[0, 2, 0], two[0][0])
    np.testing.assert_array_equal(plans[0, 2, 1], two[0][1])
    np.testing.assert_array_equal(plans[2, 0, 0], two[2][0])
    assert len(plans[0, 2, 1]) > 0


def test_plan_rejects_bad_partitions():
    case = CASES["ns_filter_3d"]
    ctx = cfs.cfs_create(cfs.params_from_case(case), None)
    try:
        cfs.describe_blocks(ctx, [case])
        with pytest.raises(cfs.CfsError):
            cfs.cfs_set_partition(ctx, 2, [0, 7, 5], 0)          # decreasing
        with pytest.raises(cfs.CfsError):
            cfs.cfs_set_partition(ctx, 2, [1, 5, 12], 0)         # does not start at 0
        with pytest.raises(cfs.CfsError):
            cfs.cfs_set_partition(ctx, 2, [0, 5, 12], 2)         # rank out of range
        cfs.cfs_set_partition(ctx, 2, [0, 5, 11], 0)             # does not cover the 12 sub-domains
        with pytest.raises(cfs.CfsError):
            cfs.cfs_exchange_plan(ctx, 1, 0)
    finally:
        cfs.cfs_destroy(ctx)


# ------------------------------------------------------------------ two gloo ranks on CPU

def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, name, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    from paper_2506_03027_gb300 import cfs as C
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        case = CASES[name]
        nsub = case.nsub
        starts = [round(q * nsub / world) for q in range(world + 1)]
        ctx = context(case, starts, rank)
        send = [C.cfs_exchange_plan(ctx, q, 0) for q in range(world)]
        recv = [C.cfs_exchange_plan(ctx, q, 1) for q in range(world)]
        C.cfs_destroy(ctx)
        # the whole grid's state, known here only at the own sub-domains' points
        rng = np.random.default_rng(11)
        Uall = rng.standard_normal((5, case.npts))
        own = owner_of(case)
        rank_of = np.searchsorted(np.array(starts[1:]), np.arange(nsub), side="right")
        mine = rank_of[own] == rank
        U = np.full_like(Uall, np.nan)
        U[:, mine] = Uall[:, mine]
        # pack 5 values per point in plan order, send / receive with the peer, unpack
        for q in range(world):
            if q == rank:
                continue
            sbuf = torch.from_numpy(np.ascontiguousarray(U[:, send[q]].T).reshape(-1))
            rbuf = torch.empty(5 * len(recv[q]), dtype=torch.float64)
            if rank < q:
                dist.send(sbuf, q)
                dist.recv(rbuf, q)
            else:
                dist.recv(rbuf, q)
                dist.send(sbuf, q)
            U[:, recv[q]] = rbuf.numpy().reshape(-1, 5).T
        reads = set().union(*[read_set(case, s) for s in range(nsub) if rank_of[s] == rank])
        idx = np.array(sorted(reads))
        out[rank] = (bool(np.array_equal(U[:, idx], Uall[:, idx])), int(np.count_nonzero(~mine)),
                     int(sum(len(r) for r in recv)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["ns_filter_3d_wide", "vortex_2d"])
def test_two_gloo_ranks_exchange_strips(name):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mctx = mp.get_context("spawn")
    with mctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [mctx.Process(target=_rank, args=(r, world, port, name, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    for r in range(world):
        ok, foreign, received = res[r]
        assert ok, r
        assert 0 < received < foreign   # strips only, not the other rank's whole sub-domains
