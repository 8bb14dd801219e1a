"""Autotuner of the launch shapes (cfs_set_tiles): times a few steps of a workload for every
candidate and keeps the fastest, persisted per device, precision and decomposition in a JSON
file (default: ~/.cache/cfs_autotune.json, or $CFS_AUTOTUNE_CACHE)."""
from __future__ import annotations

import json
import os

import numpy as np

from . import cfs
from .inputs import MultiBlock, initial_state, saa_delays

FUSED = [(fy, zc, 256) for fy in (4, 8, 16) for zc in (8, 16, 32)]
PLAIN = [(8, 16, t) for t in (128, 256, 512)]


def cache_path() -> str:
    return os.environ.get("CFS_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "cfs_autotune.json"))


def key(case, precision: int, nblocks: int = 1) -> str:
    import torch
    name = torch.cuda.get_device_name()
    return (f"{name}|p{precision}|o{case.order}|v{int(case.viscous)}|f{int(case.filter)}|"
            f"{case.nx}x{case.ny}x{case.nz}/{case.px}x{case.py}x{case.pz}|b{nblocks}|c{int(bool(case.curv))}")


def load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def store(k: str, tiles, ms: dict) -> None:
    d = load_cache()
    d[k] = {"tiles": list(tiles), "ms_per_step": ms}
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, path)


def time_candidate(case, tiles, precision: int, blocks=None, steps: int = 4, warmup: int = 6, states=None) -> float:
    """Milliseconds per step of `case` (a Case, or an inputs.MultiBlock with its block `states`)."""
    import torch
    mb = case if isinstance(case, MultiBlock) else None
    c0 = mb.case if mb is not None else case
    blocks = mb.blocks if mb is not None else (blocks or [case])
    nsub = sum(b.nsub for b in blocks)
    s = cfs.Solver(case, precision=precision, blocks=None if mb is not None else blocks, tiles=tiles)
    try:
        d = saa_delays(c0.replace(px=nsub, py=1, pz=1), warmup + steps) if c0.algo == "SAA" else None
        s.set_schedule(delays=d)
        for i, b in enumerate(blocks):
            s.set_state(states[i] if states is not None else initial_state(b), block=i)
        s.step(warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        s.step(steps)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps
    finally:
        s.close()


def tune(case, precision: int = 0, blocks=None, use_cache: bool = True, states=None):
    """Fastest launch shapes for the workload (from the cache when present).  `case` may be an
    inputs.MultiBlock (connected blocks; `states` its initial block states)."""
    mb = case if isinstance(case, MultiBlock) else None
    c0 = mb.case if mb is not None else case
    k = key(c0, precision, len(mb.blocks) if mb is not None else len(blocks or [case]))
    if mb is not None:
        k += f"|{mb.name}|{mb.npts}"
    if use_cache:
        hit = load_cache().get(k)
        if hit:
            return tuple(hit["tiles"])
    # the fused FP32 stage: 3-D Navier-Stokes CD4 blocks, Cartesian or curvilinear, periodic or
    # connected
    fused = precision == 1 and c0.nz > 1 and c0.viscous and c0.order == 4
    cands = FUSED if fused else PLAIN
    ms = {}
    for t in cands:
        ms[str(t)] = time_candidate(case, t, precision, blocks, states=states)
    best = min(cands, key=lambda t: ms[str(t)])
    store(k, best, ms)
    return best
