"""Parity of the connected multi-block path (interfaces, the wake cut's reversed orientation,
spanwise interpolation, no-slip walls, far fields, outflows) through the C ABI with the FP64
oracle: relative L2 per conserved variable at most 1e-12 per block for the FP64 path."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2506_03027_gb300 import cfs
from paper_2506_03027_gb300 import inputs as I

from gpu_util import PARITY_TOL, ensure_built, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()


def run_mb(mb, U0, nsteps, delays=None, precision=0, graph=False, diag=False):
    import torch
    st = torch.cuda.Stream() if graph else None
    ctx = torch.cuda.stream(st) if graph else torch.cuda.stream(torch.cuda.current_stream())
    with ctx:
        s = cfs.Solver(mb, precision=precision, graph=graph, stream=st)
        try:
            s.set_schedule(delays=delays)
            s.set_states(U0)
            s.step(nsteps)
            U = s.get_states()
            d = s.diagnostics(check_finite=False) if diag else None
        finally:
            s.close()
    return (U, d) if diag else U


def check_blocks(Ug, Uo, tol=PARITY_TOL):
    for b, (a, r) in enumerate(zip(Ug, Uo)):
        e = rel_l2(a, r)
        assert np.all(np.isfinite(a)) and np.all(e <= tol), (b, e)


def cgrid(algo, cfl=0.05):
    sp = I.cgrid_reduced()
    mb = I.naca_cgrid(sp, algo=algo)
    mb = mb.replace_all(dt=I.cgrid_dt(mb, cfl))
    return mb, I.cgrid_state(mb, sp)


def sub_delays(mb, n):
    return I.saa_delays(mb.case.replace(px=mb.nsub, py=1, pz=1), n)


@pytest.mark.parametrize("algo", ["SA", "CAA", "SAA"])
def test_cgrid_parity(algo):
    """The reduced 12-block NACA0012 C-grid (walls, wake cut, far field, outflows, inner/outer
    layers of different spanwise counts), 50 steps; each block against the oracle, and the
    diagnostics (volume-weighted K, enstrophy away from non-periodic faces, totals)."""
    mb, U0 = cgrid(algo)
    if algo == "CAA":
        mb = mb.replace_all(caa_L=3, kmax=2)
    n = 50
    d = sub_delays(mb, n) if algo == "SAA" else None
    Ug, dg = run_mb(mb, U0, n, delays=d, diag=True)
    Uo, do = orc.run(mb, U0, n, delays=d, diag=True)
    check_blocks(Ug, Uo)
    for b in range(1, 5):  # wall points at rest
        assert np.all(Ug[b][1:4, :, 0, :] == 0.0)
    np.testing.assert_allclose(dg[:2], do[-1][:2], rtol=1e-11)
    np.testing.assert_allclose(dg[2], do[-1][2], rtol=1e-12)
    np.testing.assert_allclose(dg[6], do[-1][6], rtol=1e-12)


def test_cgrid_graph_mode_is_bitwise_identical():
    mb, U0 = cgrid("SAA")
    n = 12
    d = sub_delays(mb, n)
    Ua = run_mb(mb, U0, n, delays=d)
    Ub = run_mb(mb, U0, n, delays=d, graph=True)
    for a, b in zip(Ua, Ub):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("algo", ["SA", "CAA", "SAA"])
def test_cgrid_fp32_form(algo):
    """FP32 intermediates on the C-grid through the fused stage (one launch per RK stage): halo
    points beyond interfaces and far fields from the per-step halo store (AT/AS steps) or an inline
    gather of the live values (synchronous steps), wall mirrors and outflow copies from the own
    points of the same plane, wall points' momentum held at zero; within the FP32-form error bound
    of the oracle, walls at rest."""
    mb, U0 = cgrid(algo)
    if algo == "CAA":
        mb = mb.replace_all(caa_L=3, kmax=2)
    n = 20
    d = sub_delays(mb, n) if algo == "SAA" else None
    Ug = run_mb(mb, U0, n, delays=d, precision=1)
    Uo = orc.run(mb, U0, n, delays=d)
    for b, (a, r) in enumerate(zip(Ug, Uo)):
        e = rel_l2(a, r)
        assert np.all(np.isfinite(a)) and np.all(e < 1e-6), (b, e)
    for b in range(1, 5):  # the airfoil blocks' wall rows
        assert np.all(Ug[b][1:4, :, 0, :] == 0.0)


@pytest.mark.parametrize("algo", ["CAA", "SAA"])
def test_cgrid_fp32_form_on_reused_memory(algo):
    """Every entry of the per-step halo store the fused stage reads is written first: the run gets
    device memory that PyTorch's caching allocator hands back after it held 0xff bytes (NaN in
    FP32 and FP64).  The C-grid's outer layer has one sub-domain along z, so its wall mirrors and
    outflow copies beyond the z faces reach their own points across the periodic wrap (foreign,
    from the store); the result matches the oracle as on fresh memory."""
    import torch
    junk = torch.full((256 << 20,), 255, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    del junk
    mb, U0 = cgrid(algo)
    if algo == "CAA":
        mb = mb.replace_all(caa_L=3, kmax=2)
    n = 12
    d = sub_delays(mb, n) if algo == "SAA" else None
    Ug = run_mb(mb, U0, n, delays=d, precision=1)
    Uo = orc.run(mb, U0, n, delays=d)
    for b, (a, r) in enumerate(zip(Ug, Uo)):
        e = rel_l2(a, r)
        assert np.all(np.isfinite(a)) and np.all(e < 1e-6), (b, e)


def test_cgrid_fp32_fused_graph_and_tiles_identical():
    """The C-grid's fused FP32 stage gives the same bits step by step, as CUDA-graph replays and
    for another tile shape."""
    import torch
    mb, U0 = cgrid("SAA")
    n = 9
    d = sub_delays(mb, n)
    Ua = run_mb(mb, U0, n, delays=d, precision=1)
    Ub = run_mb(mb, U0, n, delays=d, precision=1, graph=True)
    s = cfs.Solver(mb, precision=1, tiles=(4, 8, 256))
    try:
        s.set_schedule(delays=d)
        s.set_states(U0)
        s.step(n)
        Uc = s.get_states()
    finally:
        s.close()
    for a, b, c in zip(Ua, Ub, Uc):
        assert np.array_equal(a, b) and np.array_equal(a, c)


def test_cgrid_freestream_preserved_on_gpu():
    mb, _ = cgrid("SAA")
    free = mb.faces[6][3].state
    faces = [[dataclasses.replace(f, type="farfield", state=free) if f.type == "wall" else f for f in fs]
             for fs in mb.faces]
    mb = dataclasses.replace(mb, faces=faces)
    U0 = [np.ascontiguousarray(np.broadcast_to(np.asarray(free)[:, None, None, None], (5, b.nz, b.ny, b.nx)))
          for b in mb.blocks]
    n = 12
    Ug = run_mb(mb, U0, n, delays=sub_delays(mb, n))
    assert max(float(np.abs(a - b).max()) for a, b in zip(Ug, U0)) < 1e-12 * max(free)


def test_rotated_block_parity():
    c = I.tgv_case(24, 2, "SAA", kmax=2, filter=True, curv=0.2)
    c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), 0.1), px=3)
    mb = I.rotated_pair(c, 16, 2, 1)
    U0 = list(I.rotate_state_pair(I.tgv_state(c), 16))
    n = 12
    d = sub_delays(mb, n)
    check_blocks(run_mb(mb, U0, n, delays=d), orc.run(mb, U0, n, delays=d))


def test_split_and_span_pairs_parity():
    c = I.tgv_case(24, 2, "SAA", kmax=2, filter=True)
    c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), 0.1), px=3)
    U = I.tgv_state(c)
    n = 10
    mb = I.split_box_x(c, 16, 2, 1)
    U0 = [U[..., :16], U[..., 16:]]
    d = sub_delays(mb, n)
    check_blocks(run_mb(mb, U0, n, delays=d), orc.run(mb, U0, n, delays=d))
    mb = I.span_pair(c, 16, 12, 2, 1)
    U0 = [U[..., :16], np.ascontiguousarray(U[:, ::2, :, 16:])]
    check_blocks(run_mb(mb, U0, n, delays=d), orc.run(mb, U0, n, delays=d))


@pytest.mark.parametrize("precision", [0, 1])
def test_wall_channel_parity(precision):
    """No-slip walls on both y faces of a Cartesian box, SAA delays on the sub-domain faces inside
    the block, TGV-like initial field with zero wall momentum."""
    c = I.tgv_case(20, 2, "SAA", kmax=2, filter=True).replace(ny=21, py=3, ly=2.0)
    U = I.tgv_state(c)
    U[1:4, :, 0, :] = 0.0
    U[1:4, :, -1, :] = 0.0
    c = c.replace(dt=I.cfl_dt(c, U, 0.1))
    mb = I.wall_channel(c)
    n = 16
    d = I.saa_delays(c, n)
    Ug = run_mb(mb, [U], n, delays=d, precision=precision)
    Uo = orc.run(mb, [U], n, delays=d)
    if precision == 0:
        check_blocks(Ug, Uo)
    else:
        assert np.all(rel_l2(Ug[0], Uo[0]) < 1e-6)
    assert np.all(Ug[0][1:4, :, 0, :] == 0.0) and np.all(Ug[0][1:4, :, -1, :] == 0.0)


_FULL = {}


def _full_cgrid():
    """The full C-grid, its initial state, delays and the oracle's 7 steps (computed once)."""
    if not _FULL:
        spec = I.CGridSpec()
        mb = I.naca_cgrid(spec, algo="SAA", kmax=2)
        mb = mb.replace_all(dt=I.cgrid_dt(mb, 0.05))
        U0 = I.cgrid_state(mb, spec)
        n = 7
        d = sub_delays(mb, n)
        _FULL.update(mb=mb, U0=U0, n=n, d=d, Uo=orc.run(mb, U0, n, delays=d))
    return _FULL


def test_cgrid_full_size_parity():
    """The full 12-block C-grid of the benchmark (22.0 M points, 154 sub-domains, CUDA graph) for 7
    steps -- five synchronous warm-up steps, then two with SAA delays -- against the oracle over
    the whole field (the oracle takes about a minute on the host cores)."""
    f = _full_cgrid()
    Ug = run_mb(f["mb"], f["U0"], f["n"], delays=f["d"], graph=True)
    check_blocks(Ug, f["Uo"])


def test_cgrid_full_size_fp32_form():
    """The same run through the FP32 form as the benchmark times it (one fused launch per RK stage,
    CUDA graph): every block within the FP32-form bound of the oracle, the wall points at rest."""
    f = _full_cgrid()
    Ug = run_mb(f["mb"], f["U0"], f["n"], delays=f["d"], precision=1, graph=True)
    for b, (a, r) in enumerate(zip(Ug, f["Uo"])):
        e = rel_l2(a, r)
        assert np.all(np.isfinite(a)) and np.all(e < 1e-6), (b, e)
    for b in range(1, 5):  # the airfoil blocks' wall rows
        assert np.all(Ug[b][1:4, :, 0, :] == 0.0)


def test_fp64_power_within_a_few_ulp():
    """The FP64 path's own power (the viscosity law mu = T^0.76 of the C-grid) against numpy's
    and CUDA's pow: exp(a ln x) carries the rounding of a ln x into the result, so the relative
    error is bounded by 6e-16 (1 + |a ln x|) -- 1.2e-15 near T = 1 -- over positive normal x;
    equal special cases."""
    import torch
    rng = np.random.default_rng(7)
    x = np.concatenate([np.exp(rng.uniform(np.log(1e-300), np.log(1e300), 100000)), rng.uniform(0.5, 2.0, 100000),
                        [1.0, 2.0, 0.5, 2.2250738585072014e-308, 5e-324, 0.0, np.inf]])
    xt = torch.tensor(x, device="cuda", dtype=torch.float64)
    for a in (0.76, 0.5, 1.0, -1.3, 0.0):
        yt = torch.empty_like(xt)
        cfs.cfs_eval_power(xt, a, yt)
        torch.cuda.synchronize()
        y = yt.cpu().numpy()
        ref = np.power(x, a)
        cuda_ref = torch.pow(xt, a).cpu().numpy()
        normal = (x >= 2.2250738585072014e-308) & np.isfinite(x)
        ok = normal & np.isfinite(ref) & (ref >= 2.3e-308) & (ref < 1e300)  # normal results
        bound = 6e-16 * (1.0 + np.abs(a * np.log(x[ok])))
        assert np.all(np.abs(y[ok] / ref[ok] - 1.0) <= bound), a
        assert np.all(np.abs(y[ok] / cuda_ref[ok] - 1.0) <= bound + 2.3e-16), a
        near = ok & (np.abs(x - 1.0) < 0.5)
        assert np.max(np.abs(y[near] / ref[near] - 1.0)) < 1.2e-15, a
        # zero, subnormal and infinite x go to CUDA's pow
        assert np.array_equal(np.isinf(y), np.isinf(ref)) and np.array_equal(y[~normal], cuda_ref[~normal])


def test_connected_grid_rejects_the_learned_halo():
    """The learned halo model is built on periodic face columns: a context with non-periodic
    block faces refuses it (EINVAL) and keeps running the plain AT halo."""
    mb, U0 = cgrid("SAA")
    s = cfs.Solver(mb)
    try:
        params = np.zeros(9684, dtype=np.float32)
        scales = np.ones(15)
        with pytest.raises(cfs.CfsError) as e:
            cfs.cfs_set_halo_model(s.ctx, params, scales, True)
        assert e.value.status == cfs.CFS_EINVAL and "periodic" in cfs.cfs_last_error(s.ctx)
        s.set_schedule(delays=sub_delays(mb, 6))
        s.set_states(U0)
        s.step(6)
        assert all(np.all(np.isfinite(u)) for u in s.get_states())
    finally:
        s.close()
