"""Library checks that need no GPU: build, exported symbols, host-side coefficient generation
and argument validation of the C ABI."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2506_03027_gb300 import build as B
from paper_2506_03027_gb300 import cfs


@pytest.fixture(scope="module")
def lib():
    B.build()
    return cfs.load()


def test_header_declares_the_boundary():
    names = cfs.header_symbols()
    for must in ("cfs_create", "cfs_add_block", "cfs_split_block", "cfs_finalize", "cfs_set_schedule",
                 "cfs_set_state", "cfs_get_state", "cfs_step", "cfs_diagnostics", "cfs_get_ring",
                 "cfs_set_ring", "cfs_last_error", "cfs_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in cfs.header_symbols():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


@pytest.mark.parametrize("order", [2, 4])
def test_at_weights_match_oracle_tables(lib, order):
    """The library solves the constraint systems of Eq. 6 and Eq. 13 itself; its collapsed halo
    weights must equal the oracle's printed polynomials (Eq. 14-15, Table 5) run through the
    buffer recursion of Eq. 8."""
    kmax = 6
    W = cfs.cfs_at_weights(order, kmax)
    A, Bc = orc.lserk(order)
    s = len(A)
    for k in range(kmax + 1):
        w = orc.extrap_weights(order, k).copy()
        v = np.zeros_like(w)
        np.testing.assert_allclose(W[k, 0], w, rtol=1e-13, atol=1e-13 * np.abs(w).max())
        for m in range(1, s):
            v = A[m - 1] * v + orc.buffer_dudt(order, m - 1, k)
            w = w + Bc[m - 1] * v
            np.testing.assert_allclose(W[k, m], w, rtol=1e-12, atol=1e-12 * np.abs(w).max())


def test_zero_delay_stage0_weights_are_exact_identity(lib):
    for order in (2, 4):
        W = cfs.cfs_at_weights(order, 0)
        assert W[0, 0, 0] == 1.0 and np.all(W[0, 0, 1:] == 0.0)


def test_at_weights_reject_bad_arguments(lib):
    out = np.zeros(1000)
    p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.cfs_at_weights(3, 2, p) == -1
    assert lib.cfs_at_weights(4, -1, p) == -1
    assert lib.cfs_at_weights(4, 99, p) == -1


def test_create_validates_parameters(lib):
    good = dict(order=4, viscous=1, visc_law=0, visc_exp=0.76, gamma=1.4, mach=0.1, re=1600.0, pr=0.71,
                filter=1, alpha_f=0.499, precision=0)
    ctx = cfs.cfs_create(cfs.CfsParams(**good))
    cfs.cfs_destroy(ctx)
    for bad in (dict(order=3), dict(precision=2), dict(alpha_f=0.5), dict(gamma=1.0), dict(re=0.0)):
        with pytest.raises(cfs.CfsError) as e:
            cfs.cfs_create(cfs.CfsParams(**{**good, **bad}))
        assert e.value.status == cfs.CFS_EINVAL


def test_call_order_and_block_validation(lib):
    p = cfs.CfsParams(order=4, viscous=0, gamma=1.4, mach=0.5, re=1.0, pr=1.0, filter=0, alpha_f=0.0)
    ctx = cfs.cfs_create(p)
    try:
        with pytest.raises(cfs.CfsError) as e:
            cfs.cfs_step(ctx, 1)
        assert e.value.status == cfs.CFS_ESTATE
        with pytest.raises(cfs.CfsError) as e:
            cfs.cfs_finalize(ctx, 0)
        assert e.value.status == cfs.CFS_ESTATE  # no block yet
        with pytest.raises(cfs.CfsError) as e:
            cfs.cfs_add_block(ctx, 0, 4, 4, (1.0, 1.0, 1.0))
        assert e.value.status == cfs.CFS_EINVAL
        assert cfs.cfs_add_block(ctx, 16, 16, 1, (0.1, 0.1, 1.0)) == 0
        assert cfs.cfs_add_block(ctx, 12, 20, 1, (0.1, 0.1, 1.0)) == 1  # batches of blocks
        with pytest.raises(cfs.CfsError):
            cfs.cfs_add_block(ctx, 16, 16, 8, (0.1, 0.1, 0.1))  # 2-D and 3-D blocks do not mix
        with pytest.raises(cfs.CfsError):
            cfs.cfs_split_block(ctx, 2, 1, 1, 1)  # unknown block
        with pytest.raises(cfs.CfsError):
            cfs.cfs_split_block(ctx, 0, 17, 1, 1)
        for bad in [(0, 6, 1, 0, 0), (0, 0, 1, 1, 2), (0, 4, 1, 0, 0), (0, 1, 0, 1, 0), (0, 0, 3, 1, 0)]:
            with pytest.raises(cfs.CfsError) as e:
                cfs.cfs_connect(ctx, *bad)  # bad face, orientation, z face, face to itself, block
            assert e.value.status == cfs.CFS_EINVAL
        cfs.cfs_connect(ctx, 0, 0, 0, 1)  # the periodic default
        for bad in [(0, 0, 7), (0, 4, cfs.BC_WALL), (0, 0, cfs.BC_FARFIELD), (5, 0, cfs.BC_WALL)]:
            with pytest.raises(cfs.CfsError) as e:
                cfs.cfs_set_bc(ctx, *bad)  # unknown type, z face, far field without a state, block
            assert e.value.status == cfs.CFS_EINVAL
        with pytest.raises(cfs.CfsError):
            cfs.cfs_set_face_shift(ctx, 0, 0, (1.0, 0.0))  # not an interface
        with pytest.raises(cfs.CfsError) as e:
            cfs.cfs_set_schedule(ctx, 1, 1, 4, None)
        assert e.value.status == cfs.CFS_ESTATE
        with pytest.raises(cfs.CfsError):
            cfs.cfs_set_dt(ctx, -1.0)
        assert "dt" in cfs.cfs_last_error(ctx)
    finally:
        cfs.cfs_destroy(ctx)


def test_set_block_grid_validation(lib):
    p = cfs.CfsParams(order=4, viscous=0, gamma=1.4, mach=0.5, re=1.0, pr=1.0, filter=0, alpha_f=0.0)
    ctx = cfs.cfs_create(p)
    try:
        assert cfs.cfs_add_block(ctx, 16, 12, 1, (0.1, 0.1, 1.0)) == 0
        xy = np.zeros((2, 12, 16))
        with pytest.raises(cfs.CfsError) as e:
            cfs.cfs_set_block_grid(ctx, 1, xy, (1.6, 0, 0, 1.2))
        assert e.value.status == cfs.CFS_EINVAL
        bad = xy.copy()
        bad[0, 3, 4] = np.nan
        with pytest.raises(cfs.CfsError):
            cfs.cfs_set_block_grid(ctx, 0, bad, (1.6, 0, 0, 1.2))
        with pytest.raises(cfs.CfsError):
            cfs.cfs_set_block_grid(ctx, 0, xy, (1.6, np.inf, 0, 1.2))
        cfs.cfs_set_block_grid(ctx, 0, xy, (1.6, 0, 0, 1.2))
    finally:
        cfs.cfs_destroy(ctx)


def test_topology_validation_at_finalize(lib):
    """Face descriptions are checked when the context is finalized, before any device memory is
    touched: an interface between faces of different tangential point counts, a Cartesian
    interface joining non-opposite faces, and a curvilinear block joined to a Cartesian one are
    rejected with EINVAL."""
    p = cfs.CfsParams(order=4, viscous=0, gamma=1.4, mach=0.5, re=1.0, pr=1.0, filter=0, alpha_f=0.0)

    def attempt(setup):
        ctx = cfs.cfs_create(p)
        try:
            cfs.cfs_add_block(ctx, 16, 16, 1, (0.1, 0.1, 1.0))
            cfs.cfs_add_block(ctx, 12, 20, 1, (0.1, 0.1, 1.0))
            cfs.cfs_add_block(ctx, 12, 16, 1, (0.1, 0.1, 1.0))
            setup(ctx)
            with pytest.raises(cfs.CfsError) as e:
                cfs.cfs_finalize(ctx, 0)
            return e.value.status, cfs.cfs_last_error(ctx)
        finally:
            cfs.cfs_destroy(ctx)

    st, msg = attempt(lambda ctx: cfs.cfs_connect(ctx, 0, 1, 1, 0))  # 16 vs 20 points along y
    assert st == cfs.CFS_EINVAL and "tangential" in msg
    st, msg = attempt(lambda ctx: cfs.cfs_connect(ctx, 0, 3, 2, 1))  # Cartesian +y to +x
    assert st == cfs.CFS_EINVAL and "Cartesian" in msg

    def curv_to_cart(ctx):
        xy = np.stack(np.meshgrid(np.arange(16) * 0.1, np.arange(16) * 0.1)).astype(np.float64)
        cfs.cfs_set_block_grid(ctx, 0, xy, (1.6, 0.0, 0.0, 1.6))
        cfs.cfs_connect(ctx, 0, 1, 2, 0)
    st, msg = attempt(curv_to_cart)
    assert st == cfs.CFS_EINVAL and "curvilinear" in msg



def _ctx_for(mb):
    c = mb.case
    p = cfs.CfsParams(order=c.order, viscous=int(c.viscous), visc_law=c.visc_law, visc_exp=c.visc_exp,
                      gamma=c.gamma, mach=c.mach, re=c.re, pr=c.pr, filter=int(c.filter), alpha_f=c.alpha_f)
    ctx = cfs.cfs_create(p)
    cfs.describe_blocks(ctx, mb.blocks, mb)
    return ctx


@pytest.mark.parametrize("topology", ["cgrid", "rotated", "span", "channel"])
def test_halo_sources_match_the_oracle(lib, topology):
    """The library's host resolution of the points beyond non-periodic block faces (the gather
    entries its kernels read: sources, weights, mirror and crossing flags, far-field constants)
    agrees, point by point, with the oracle's independent resolution -- on the reduced C-grid
    (wake cut, walls, far field, outflows, spanwise interpolation), a 180-degree rotated block, a
    spanwise-interpolated pair and a wall channel; faces to the filter's depth 5, corners to r x r.
    No device is touched: the faces are validated and resolved on the host."""
    from paper_2506_03027_gb300 import inputs as I
    if topology == "cgrid":
        mb = I.naca_cgrid(I.cgrid_reduced())
    elif topology == "rotated":
        c = I.tgv_case(24, 2, "CAA", filter=True, curv=0.2).replace(px=3)
        mb = I.rotated_pair(c, 16, 2, 1)
    elif topology == "span":
        mb = I.span_pair(I.tgv_case(24, 2, "SAA", kmax=2, filter=True).replace(px=3), 16, 12, 2, 1)
    else:
        mb = I.wall_channel(I.tgv_case(20, 2, "SAA", kmax=2, filter=True).replace(ny=21, py=3, ly=2.0))
    ctx = _ctx_for(mb)
    try:
        n = 0
        for bi, b in enumerate(mb.blocks):
            nonper = [F.type != "periodic" for F in mb.faces[bi]]
            pts = []
            for k in range(b.nz):
                for j in range(-5, b.ny + 5):
                    for i in range(-5, b.nx + 5):
                        di = -i if i < 0 else (i - b.nx + 1 if i >= b.nx else 0)
                        dj = -j if j < 0 else (j - b.ny + 1 if j >= b.ny else 0)
                        if (di == 0 and dj == 0) or (di and dj and (di > 2 or dj > 2)):
                            continue
                        if (di and nonper[0 if i < 0 else 1]) or (dj and nonper[2 if j < 0 else 3]):
                            pts.append((i, j, k))
            if not pts:
                continue
            ref = orc.halo_sources(mb, bi, pts)
            for (i, j, k), (co, to) in zip(pts, ref):
                cl, tl = cfs.cfs_halo_sources(ctx, bi, i, j, k)
                assert np.array_equal(cl, co), (bi, i, j, k, cl, co)
                key = lambda t: t[:4] + t[5:]
                tl, to = sorted(tl, key=key), sorted(to, key=key)
                assert [key(t) for t in tl] == [key(t) for t in to], (bi, i, j, k, tl, to)
                assert np.allclose([t[4] for t in tl], [t[4] for t in to], rtol=0, atol=1e-15), (tl, to)
                n += 1
        assert n > 0
    finally:
        cfs.cfs_destroy(ctx)


@pytest.mark.parametrize("topology", ["cgrid", "rotated"])
def test_metric_terms_match_the_oracle(lib, topology):
    """The library's metric terms (App. A) of curvilinear blocks, continued across interfaces, the
    wake cut and physical faces, agree with the oracle's own computation at every point of the
    block planes and their halos to the stencil radius (1e-12 relative to the largest term of
    each kind; beyond it both give NaN).  No device is touched."""
    from paper_2506_03027_gb300 import inputs as I
    if topology == "cgrid":
        mb = I.naca_cgrid(I.cgrid_reduced())
    else:
        c = I.tgv_case(24, 2, "CAA", filter=True, curv=0.2).replace(px=3)
        mb = I.rotated_pair(c, 16, 2, 1)
    ctx = _ctx_for(mb)
    try:
        G = 4
        for bi, b in enumerate(mb.blocks):
            pts = [(i, j) for j in range(-G, b.ny + G) for i in range(-G, b.nx + G)]
            ref = orc.metric_terms(mb, bi, pts)
            got = np.array([cfs.cfs_metric_terms(ctx, bi, i, j)[:6] for i, j in pts])
            fin = np.isfinite(ref)
            assert np.array_equal(fin, np.isfinite(got)), bi
            scale = np.nanmax(np.abs(ref), axis=0)
            err = np.where(fin, np.abs(got - ref), 0.0) / scale
            assert err.max() < 1e-12, (bi, err.max(axis=0))
            assert fin[:, 5].sum() > b.nx * b.ny  # the halo carries finite terms too
    finally:
        cfs.cfs_destroy(ctx)


def test_compact_scheme_accepted_only_where_built(lib):
    """The compact scheme (cfs_params.compact = 1) is accepted for the Euler equations with the
    fourth-order time / AT schemes in FP64, and rejected with EINVAL otherwise."""
    from paper_2506_03027_gb300 import inputs as I
    ok = I.tgv_case(16, 2, "SA", viscous=False, filter=False, compact=1)
    ctx = cfs.cfs_create(cfs.params_from_case(ok), None)
    cfs.cfs_destroy(ctx)
    for bad in (ok.replace(viscous=True), ok.replace(order=2)):
        with pytest.raises(cfs.CfsError):
            cfs.cfs_create(cfs.params_from_case(bad), None)
    with pytest.raises(cfs.CfsError):
        cfs.cfs_create(cfs.params_from_case(ok, precision=1), None)
