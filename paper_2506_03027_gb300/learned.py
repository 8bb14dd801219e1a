"""Learned halo predictor: training data from synchronous runs, training on the GPU with the
library's own kernels (cfs_mlp_grad / cfs_mlp_adamw), and evaluation.

The network (see include/cfs.h) predicts, per face column of a sub-domain's 4-deep halo, the
residual of the current-level values over the three-level extrapolation of Eq. 14 from the
delayed levels n-k, n-k-1, n-k-2 and the change of the sub-domain's own boundary values since
level n-k.  In a synchronous run every halo value at level n is known exactly, so any step of such
a run yields training samples for every delay k <= 4 at once.
"""
from __future__ import annotations

import math

import numpy as np

from . import cfs
from .inputs import Case, initial_state

KMAX = 4
NIN, NOUT, NPARAM = cfs.MLP_NIN, cfs.MLP_NOUT, cfs.MLP_NPARAM


def _axis_split(n: int, p: int):
    base, rem = divmod(n, p)
    lens = [base + (1 if i < rem else 0) for i in range(p)]
    return lens


def sample_specs(case: Case, n: int, rng: np.random.Generator) -> np.ndarray:
    """Random (sub-domain, face, t1, t2, k) with k uniform on 0..4 and (t1, t2) uniform over the face."""
    lx, ly, lz = (_axis_split(case.nx, case.px), _axis_split(case.ny, case.py), _axis_split(case.nz, case.pz))
    sid = rng.integers(0, case.nsub, size=n)
    ix = sid % case.px
    iy = (sid // case.px) % case.py
    iz = sid // (case.px * case.py)
    nfaces = 6 if case.nz > 1 else 4
    face = rng.integers(0, nfaces, size=n)
    sz = np.stack([np.array(lx)[ix], np.array(ly)[iy], np.array(lz)[iz]], axis=1)
    a = face // 2
    n1 = sz[np.arange(n), (a + 1) % 3]
    n2 = sz[np.arange(n), (a + 2) % 3]
    t1 = (rng.random(n) * n1).astype(np.int64)
    t2 = (rng.random(n) * n2).astype(np.int64)
    k = rng.integers(0, KMAX + 1, size=n)
    return np.stack([sid, face, t1, t2, k], axis=1).astype(np.int32)


def generate(case: Case, first_step: int, last_step: int, per_step: int, seed: int, scales: np.ndarray,
             start=None, with_at4: bool = False):
    """Run the case synchronously (from `start`, default its initial state) and draw `per_step`
    samples at every step in [first_step, last_step).  Returns device tensors (x BF16 bit patterns
    as int16 [n][65], target FP32 [n][20]) and, with with_at4, the AT4 stage-0 residuals of Eq. 15
    in target units (FP32 [n][20]) as a third."""
    import torch
    assert first_step >= KMAX + (5 if with_at4 else 2)
    rng = np.random.default_rng(seed)
    sa = case.replace(algo="SA")
    s = cfs.Solver(sa, max_delay=KMAX)
    s.set_schedule()
    s.set_state(initial_state(sa) if start is None else start)
    s.step(first_step)
    xs, ts, a4 = [], [], []
    for _ in range(first_step, last_step):
        spec = torch.from_numpy(sample_specs(sa, per_step, rng)).cuda()
        x = torch.empty((per_step, NIN), dtype=torch.int16, device="cuda")
        t = torch.empty((per_step, NOUT), dtype=torch.float32, device="cuda")
        a = torch.empty((per_step, NOUT), dtype=torch.float32, device="cuda") if with_at4 else None
        cfs.cfs_halo_samples(s.ctx, spec.data_ptr(), per_step, scales, x.data_ptr(), t.data_ptr(),
                             a.data_ptr() if with_at4 else 0)
        xs.append(x)
        ts.append(t)
        if with_at4:
            a4.append(a)
        s.step(1)
    torch.cuda.synchronize()
    s.close()
    if with_at4:
        return torch.cat(xs), torch.cat(ts), torch.cat(a4)
    return torch.cat(xs), torch.cat(ts)


def bf16_to_float(x):
    """int16 BF16 bit patterns (torch) to float32."""
    import torch
    return (x.to(torch.int32) << 16).view(torch.float32) if x.dtype == torch.int32 else \
        ((x.to(torch.int32) & 0xFFFF) << 16).view(torch.float32)


def fit_scales(case: Case, seed: int = 1, first_step: int = 6, nsteps: int = 6, per_step: int = 20000,
               start=None) -> np.ndarray:
    """Per-variable scales from unscaled samples: 1 / RMS of each feature group and of the target."""
    unit = np.ones(15)
    X, T = generate(case, first_step, first_step + nsteps, per_step, seed, unit, start=start)
    Xf = bf16_to_float(X).double().cpu().numpy()
    Tf = T.double().cpu().numpy()
    sc = np.ones(15)
    for v in range(5):
        d1 = Xf[:, [j * 5 + v for j in range(4)]]
        own = Xf[:, [40 + j * 5 + v for j in range(4)]]
        tv = Tf[:, [j * 5 + v for j in range(4)]]
        sc[v] = 1.0 / max(math.sqrt(np.mean(d1 ** 2)), 1e-30)
        sc[5 + v] = 1.0 / max(math.sqrt(np.mean(own ** 2)), 1e-30)
        sc[10 + v] = 1.0 / max(math.sqrt(np.mean(tv ** 2)), 1e-30)
    return sc


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters: uniform +-1/sqrt(fan_in) weights, zero biases (FP32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, shape in ((NIN, (64, NIN)), (None, (64,)), (64, (64, 64)), (None, (64,)), (64, (NOUT, 64)),
                          (None, (NOUT,))):
        parts.append(np.zeros(shape) if fan_in is None else rng.uniform(-1, 1, size=shape) / math.sqrt(fan_in))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def train(X, T, steps: int = 3000, batch: int = 4096, lr: float = 2e-3, seed: int = 0, log_every: int = 500):
    """AdamW on the mean squared error with the library's gradient and update kernels; cosine
    learning-rate decay.  Returns (params as numpy float32, list of (step, loss))."""
    import torch
    n = X.shape[0]
    params = torch.from_numpy(init_params(seed)).cuda()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ws = torch.empty(cfs.cfs_mlp_workspace_bytes(batch) // 4 + 1, dtype=torch.float32, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    stream = torch.cuda.current_stream().cuda_stream
    hist = []
    for it in range(1, steps + 1):
        idx = torch.randint(0, n, (batch,), device="cuda", generator=g)
        xb = X[idx].contiguous()
        tb = T[idx].contiguous()
        cfs.cfs_mlp_grad(params.data_ptr(), xb.data_ptr(), tb.data_ptr(), batch, ws.data_ptr(), grad.data_ptr(),
                         loss.data_ptr(), stream)
        rate = lr * 0.5 * (1.0 + math.cos(math.pi * (it - 1) / steps))
        cfs.cfs_mlp_adamw(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), it, rate, 0.9, 0.999, 1e-8,
                          1e-5, stream)
        if it % log_every == 0 or it == 1 or it == steps:
            hist.append((it, float(loss.item())))
    return params.cpu().numpy(), hist


def predict(params: np.ndarray, X):
    """Network outputs for device features X (int16 BF16 patterns) with the library's forward."""
    import torch
    p = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).cuda()
    y = torch.empty((X.shape[0], NOUT), dtype=torch.float32, device="cuda")
    cfs.cfs_mlp_forward(p.data_ptr(), X.data_ptr(), y.data_ptr(), X.shape[0], torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return y


def halo_errors(params: np.ndarray, X, T, A4=None) -> dict:
    """Mean squared error of the current-level halo values, in target units, of the three-level
    extrapolation alone (target itself), with the network's residual added, and (A4 given) of the
    AT4 stage-0 value of Eq. 15 that the network replaces in the solver."""
    y = predict(params, X)
    base = float((T.double() ** 2).mean())
    net = float(((T - y).double() ** 2).mean())
    out = {"extrapolation3_mse": base, "learned_mse": net, "ratio": net / base if base > 0 else float("nan")}
    if A4 is not None:
        at4 = float((A4.double() ** 2).mean())
        out["at4_mse"] = at4
        out["learned_over_at4"] = net / at4 if at4 > 0 else float("nan")
    return out


def developed_state(case: Case, t_end: float, cfl: float = 0.5):
    """The synchronous run of the case's initial field to time t_end at CFL `cfl` (no delays):
    a flow with the smaller scales of later times, from which the comparisons start."""
    from .inputs import cfl_dt
    U0 = initial_state(case)
    dt = cfl_dt(case, U0, cfl)
    n = int(math.ceil(t_end / dt))
    c = case.replace(algo="SA", dt=t_end / n)
    s = cfs.Solver(c)
    try:
        s.set_schedule()
        s.set_state(U0)
        s.step(n)
        return s.get_state(), n
    finally:
        s.close()


def solver_comparison(case: Case, start, params, scales, nsteps: int, seed: int = None) -> dict:
    """SA, plain AT, the 3-level extrapolation of Eq. 14 alone in the stage-0 face halos (the
    network's base: a network whose parameters are all zero) and the trained network, on the same
    SAA schedule (delays 0..4), all from `start`, for nsteps steps: each asynchronous run's
    relative L2 difference from the synchronous run per conserved variable (rho, rho E against
    their own norms, momentum against the momentum vector's), whether it stayed finite, and the ms
    per step of each."""
    import torch
    from .inputs import saa_delays
    saa = case.replace(algo="SAA", kmax=KMAX)
    d = saa_delays(saa, nsteps, seed=seed)
    res = {}
    for name in ("SA", "AT", "extrap3", "learned"):
        cc = case.replace(algo="SA") if name == "SA" else saa
        s = cfs.Solver(cc, max_delay=KMAX)
        try:
            s.set_schedule(delays=d if name != "SA" else None)
            if name == "learned":
                cfs.cfs_set_halo_model(s.ctx, params, scales)
            elif name == "extrap3":
                cfs.cfs_set_halo_model(s.ctx, np.zeros(NPARAM, dtype=np.float32), scales)
            s.set_state(start)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            s.step(nsteps)
            e1.record()
            torch.cuda.synchronize()
            res[name] = (s.get_state(), e0.elapsed_time(e1) / nsteps)
        finally:
            s.close()
    ref = res["SA"][0]
    mom = math.sqrt(sum(float(np.linalg.norm(ref[v])) ** 2 for v in (1, 2, 3)))

    def err(U):
        return [float(np.linalg.norm(U[v] - ref[v]) / (mom if v in (1, 2, 3) else np.linalg.norm(ref[v])))
                for v in range(5)]
    return {"rel_l2_vs_sa": {k: err(res[k][0]) for k in ("AT", "extrap3", "learned")},
            "ms_per_step": {k: v[1] for k, v in res.items()}, "steps": nsteps, "dt": case.dt,
            "finite": {k: bool(np.all(np.isfinite(v[0]))) for k, v in res.items()}}


def solver_run(n: int = 160, p: int = 5, steps: int = 12, seed: int = 1) -> dict:
    """A Taylor-Green run (n^3, p^3 sub-domains, SAA delays 0..4, CFL 0.05) with a seeded untrained
    network in the stage-0 face halos; returns the per-kernel-kind times (ms per launch) of the
    last four steps.  Used to time and profile the network's solver kernel."""
    import torch
    from .inputs import cfl_dt, saa_delays, tgv_case, tgv_state
    c = tgv_case(n, p, "SAA", kmax=4)
    c = c.replace(dt=cfl_dt(c, tgv_state(c), 0.05))
    s = cfs.Solver(c, max_delay=4)
    try:
        s.set_schedule(delays=saa_delays(c, steps))
        scales = np.array([3e3, 2e3, 2e3, 2e3, 1e3, 4e2, 3e2, 3e2, 3e2, 2e2, 1e7, 1e6, 1e6, 1e6, 5e5])
        cfs.cfs_set_halo_model(s.ctx, init_params(seed), scales)
        s.set_state(tgv_state(c))
        s.step(steps - 4)
        torch.cuda.synchronize()
        cfs.cfs_set_timing(s.ctx, True)
        s.step(4)
        torch.cuda.synchronize()
        return {k: v[0] / max(v[1], 1) for k, v in cfs.cfs_get_timing(s.ctx).items() if v[1]}
    finally:
        s.close()


if __name__ == "__main__":
    import sys
    print(solver_run(int(sys.argv[1]) if len(sys.argv) > 1 else 160, int(sys.argv[2]) if len(sys.argv) > 2 else 5))
