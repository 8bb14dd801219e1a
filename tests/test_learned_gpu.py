"""The learned halo predictor on the GPU: forward and gradient kernels against the FP64 numpy
oracle, training samples against the C oracle's features, the solver with the network against the
oracle with the same network, and what training gains over the extrapolation it corrects."""
import ctypes

import numpy as np
import pytest

from oracle import mlp as omlp
from oracle import oracle as orc
from paper_2506_03027_gb300 import cfs
from paper_2506_03027_gb300 import inputs as I
from paper_2506_03027_gb300 import learned as L

from gpu_util import ensure_built, gpu_run, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    return torch


def bf16_features(rng, n):
    """Random features that are exact BF16 values, and their bit patterns."""
    x = rng.standard_normal((n, omlp.NIN)).astype(np.float32)
    bits = (x.view(np.uint32) + 0x7FFF + ((x.view(np.uint32) >> 16) & 1)) >> 16
    xb = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return xb, bits.astype(np.uint16).view(np.int16)


def test_forward_matches_fp64_oracle(torch):
    rng = np.random.default_rng(0)
    p = L.init_params(3)
    xb, bits = bf16_features(rng, 777)
    y = L.predict(p, torch.from_numpy(bits).cuda()).cpu().numpy().astype(np.float64)
    ref = omlp.forward(p.astype(np.float64), xb)[0]
    assert np.abs(y - ref).max() <= 2e-5 * max(1.0, np.abs(ref).max())


def test_gradient_matches_fp64_oracle(torch):
    rng = np.random.default_rng(1)
    p = L.init_params(4)
    n = 1000
    xb, bits = bf16_features(rng, n)
    T = rng.standard_normal((n, omlp.NOUT)).astype(np.float32)
    pt = torch.from_numpy(p).cuda()
    xt = torch.from_numpy(bits).cuda()
    tt = torch.from_numpy(T).cuda()
    g = torch.zeros_like(pt)
    loss = torch.zeros(1, device="cuda")
    ws = torch.empty(cfs.cfs_mlp_workspace_bytes(n) // 4 + 1, device="cuda")
    cfs.cfs_mlp_grad(pt.data_ptr(), xt.data_ptr(), tt.data_ptr(), n, ws.data_ptr(), g.data_ptr(), loss.data_ptr())
    torch.cuda.synchronize()
    lref, gref = omlp.loss_and_grad(p.astype(np.float64), xb, T.astype(np.float64))
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - lref) <= 1e-5 * lref
    assert np.linalg.norm(gg - gref) <= 1e-5 * np.linalg.norm(gref), np.linalg.norm(gg - gref) / np.linalg.norm(gref)
    # determinism: the same call gives the same bits
    g2 = torch.zeros_like(pt)
    cfs.cfs_mlp_grad(pt.data_ptr(), xt.data_ptr(), tt.data_ptr(), n, ws.data_ptr(), g2.data_ptr(), 0)
    torch.cuda.synchronize()
    assert torch.equal(g, g2)


def halo_index(case, sid, f, t1, t2, j):
    """Flat index of halo point j of a face column (grid geometry only)."""
    def split(n, p, i):
        b, r = divmod(n, p)
        return i * b + min(i, r), b + (1 if i < r else 0)
    ix, iy, iz = sid % case.px, (sid // case.px) % case.py, sid // (case.px * case.py)
    o, sz = zip(split(case.nx, case.px, ix), split(case.ny, case.py, iy), split(case.nz, case.pz, iz))
    a, side = f // 2, f % 2
    c = [0, 0, 0]
    c[(a + 1) % 3] = t1
    c[(a + 2) % 3] = t2
    c[a] = -j if side == 0 else sz[a] - 1 + j
    n = (case.nx, case.ny, case.nz)
    gx, gy, gz = [(o[q] + c[q]) % n[q] for q in range(3)]
    return gx + case.nx * (gy + case.ny * gz)


def oracle_levels(case, nsteps):
    """U^0..U^nsteps of a synchronous run, computed by the oracle one step at a time."""
    levels = [I.initial_state(case)]
    for n in range(nsteps):
        levels.append(orc.run(case, levels[-1], 1, n0=n))
    return levels


def test_samples_match_oracle_features(torch):
    c = I.tgv_case(24, 2, "SA", filter=False)
    c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), 0.05))
    nst = 8
    scales = np.array([3e3, 2e3, 2e3, 2e3, 1e3, 4e2, 3e2, 3e2, 3e2, 2e2, 1e7, 1e6, 1e6, 1e6, 5e5])
    s = cfs.Solver(c, max_delay=4)
    s.set_schedule()
    s.set_state(I.tgv_state(c))
    s.step(nst)
    specs = L.sample_specs(c, 300, np.random.default_rng(5))
    spec_t = torch.from_numpy(specs).cuda()
    x = torch.empty((300, 65), dtype=torch.int16, device="cuda")
    t = torch.empty((300, 20), dtype=torch.float32, device="cuda")
    cfs.cfs_halo_samples(s.ctx, spec_t.data_ptr(), 300, scales, x.data_ptr(), t.data_ptr())
    torch.cuda.synchronize()
    s.close()
    xg = ((x.cpu().numpy().view(np.uint16).astype(np.uint32)) << 16).view(np.float32).astype(np.float64)
    tg = t.cpu().numpy().astype(np.float64)
    lev = oracle_levels(c, nst)
    p = orc.params(c)
    p.mlp_scales = np.ascontiguousarray(scales).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    lib = orc._load()
    fn = lib.or_column_features
    Dp = ctypes.POINTER(ctypes.c_double)
    fn.argtypes = [ctypes.POINTER(orc.OrParams), ctypes.POINTER(Dp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_int, ctypes.c_int, Dp, Dp]
    mism = 0
    for i, (sid, f, t1, t2, k) in enumerate(specs):
        arrs = [lev[nst], lev[nst - k], lev[nst - k - 1], lev[nst - k - 2]]
        ptrs = (Dp * 4)(*[a.ctypes.data_as(Dp) for a in arrs])
        xo = np.zeros(65)
        at3 = np.zeros(20)
        fn(ctypes.byref(p), ptrs, int(sid), int(f), int(t1), int(t2), int(k), xo.ctypes.data_as(Dp), at3.ctypes.data_as(Dp))
        # features: identical BF16 values unless a rounding boundary separates the two FP64 runs;
        # level differences that vanish by symmetry (rho w) carry the runs' roundoff (~1e-12 after
        # scaling), hence the absolute floor
        d = np.abs(xg[i] - xo)
        mism += int(np.sum(d > 1e-9))
        assert np.all(d <= 2.0 ** -7 * np.abs(xo) + 1e-9), (i, np.max(d))
        # targets: (U^n at the halo points - extrapolation) * out_scale
        truth = np.array([[lev[nst][v].ravel()[halo_index(c, sid, f, t1, t2, j)] for v in range(5)]
                          for j in range(1, 5)]).ravel()
        tref = (truth - at3) * np.tile(scales[10:15], 4)
        assert np.all(np.abs(tg[i] - tref) <= 1e-6 * np.abs(tref) + 1e-3), (i, tg[i] - tref)
    assert mism <= 0.01 * specs.shape[0] * 65


def test_learned_solver_matches_oracle(torch):
    """The solver with a (seeded, untrained) network in the stage-0 face halos against the oracle
    with the same network: same step, same delays."""
    c = I.tgv_case(24, 2, "SAA", kmax=4, filter=True)
    c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), 0.05))
    nst = 12
    d = I.saa_delays(c, nst)
    params = L.init_params(7)
    scales = np.array([3e3, 2e3, 2e3, 2e3, 1e3, 4e2, 3e2, 3e2, 3e2, 2e2, 1e7, 1e6, 1e6, 1e6, 5e5])
    s = cfs.Solver(c, max_delay=4)
    s.set_schedule(delays=d)
    cfs.cfs_set_halo_model(s.ctx, params, scales)
    s.set_state(I.tgv_state(c))
    s.step(nst)
    Ug = s.get_state()
    s.close()
    Uo = orc.run(c, I.tgv_state(c), nst, delays=d, model=(params, scales))
    Uplain = orc.run(c, I.tgv_state(c), nst, delays=d)
    e = rel_l2(Ug, Uo)
    assert np.all(e <= 1e-11), e
    assert rel_l2(Uo, Uplain).max() > 100 * e.max()  # the network really changed the run


def test_training_beats_its_extrapolation(torch):
    """Trained on synchronous-run halos, the network's current-level prediction on held-out steps
    has a smaller error than the three-level extrapolation it corrects."""
    c = I.tgv_case(64, 2, "SA")
    c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), 0.05))
    scales = L.fit_scales(c, seed=1, first_step=6, nsteps=4, per_step=20000)
    X, T = L.generate(c, 6, 40, 20000, seed=2, scales=scales)
    Xh, Th = L.generate(c, 60, 70, 20000, seed=3, scales=scales)
    params, hist = L.train(X, T, steps=1500, batch=4096, lr=2e-3, seed=0)
    assert hist[-1][1] < hist[0][1]
    ev = L.halo_errors(params, Xh, Th)
    print("held-out halo MSE (target units):", ev, "training loss:", hist[0], hist[-1])
    assert ev["ratio"] < 0.5, ev


def test_learned_halo_against_at4(torch):
    """What the trained network changes against the method it replaces (AT4, Eq. 15), on a TGV
    64^3 grid of 2^3 sub-domains of 32^3 with SAA delays 0..4 at CFL 0.05 (trained on synchronous
    halos at the same time step):
      * sample by sample the AT4 extrapolation predicts the held-out current-level halo values far
        better than the network does (smaller mean squared error);
      * in the solver the plain AT4 halos amplify the asynchrony error (the high-order
        extrapolation over delays up to 4 has weights summing in magnitude to about 100), while the
        network, built on the 3-level extrapolation, keeps the run closer to the synchronous one
        after 200 steps.  The 3-level extrapolation alone is reported beside it."""
    c = I.tgv_case(64, 2, "SA")
    c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), 0.05))
    scales = L.fit_scales(c, seed=1, first_step=9, nsteps=4, per_step=20000)
    X, T = L.generate(c, 9, 40, 20000, seed=2, scales=scales)
    params, hist = L.train(X, T, steps=1500, batch=4096, lr=2e-3, seed=0)
    Xh, Th, A4 = L.generate(c, 60, 66, 20000, seed=3, scales=scales, with_at4=True)
    halo = L.halo_errors(params, Xh, Th, A4)
    cmp = L.solver_comparison(c, I.tgv_state(c), params, scales, 200)
    print("halo:", halo, "solver:", cmp)
    assert halo["at4_mse"] < halo["learned_mse"] < halo["extrapolation3_mse"], halo
    e = cmp["rel_l2_vs_sa"]
    assert cmp["finite"]["learned"]
    worst_learned = max(e["learned"])
    worst_at = max(e["AT"]) if cmp["finite"]["AT"] else float("inf")
    assert worst_learned < worst_at, (e, cmp["finite"])
