"""Thin Python binding of libcfs (the C ABI in include/cfs.h).

Argument marshalling only: every step of the hot path runs in the library's CUDA kernels.  The
functions ``cfs_*`` mirror the C entry points one to one and raise ``CfsError`` on a non-OK
status.  ``Solver`` strings them together for one block and lets PyTorch own the device memory
(through the allocator callback) and the stream.

There is no fallback: if ``libcfs.so`` has not been built, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from .inputs import grid_xy

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcfs.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "cfs.h")

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESTATE", 5: "ENAN", 6: "ETIMEOUT", 7: "EXCHANGE"}
CFS_OK, CFS_EINVAL, CFS_ENOMEM, CFS_ECUDA, CFS_ESTATE, CFS_ENAN, CFS_ETIMEOUT, CFS_EXCHANGE = range(8)
ALGO = {"SA": 0, "CAA": 1, "SAA": 2}
HOST, DEVICE = 0, 1


class CfsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class CfsParams(ctypes.Structure):
    _fields_ = [
        ("order", ctypes.c_int), ("viscous", ctypes.c_int), ("visc_law", ctypes.c_int),
        ("visc_exp", ctypes.c_double), ("gamma", ctypes.c_double), ("mach", ctypes.c_double),
        ("re", ctypes.c_double), ("pr", ctypes.c_double), ("filter", ctypes.c_int),
        ("alpha_f", ctypes.c_double), ("precision", ctypes.c_int), ("compact", ctypes.c_int),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
# exchange transport of a partitioned context: (user, nranks, send, send_counts, recv, recv_counts, stream)
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                               ctypes.POINTER(ctypes.c_longlong), ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                               ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_lock = threading.Lock()


def header_symbols() -> list[str]:
    """Entry points declared in include/cfs.h."""
    with open(HEADER) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:cfs_status|int|void|size_t|const char\*)\s+(cfs_\w+)\s*\(", src, re.M)))


def load() -> ctypes.CDLL:
    """Open libcfs.so (built by ``paper_2506_03027_gb300.build``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcfs.so not found at {LIB_PATH}: run paper_2506_03027_gb300/build.py "
                               "(the solver has no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
        ll = ctypes.c_longlong
        sig = {
            "cfs_create": ([ctypes.POINTER(CfsParams), vp, ctypes.POINTER(vp)], ip),
            "cfs_set_allocator": ([vp, ALLOC_FN, FREE_FN, vp], ip),
            "cfs_add_block": ([vp, ip, ip, ip, dp, ctypes.POINTER(ip)], ip),
            "cfs_split_block": ([vp, ip, ip, ip, ip], ip),
            "cfs_set_block_grid": ([vp, ip, dp, dp], ip),
            "cfs_connect": ([vp, ip, ip, ip, ip, ip], ip),
            "cfs_set_bc": ([vp, ip, ip, ip, dp], ip),
            "cfs_set_face_shift": ([vp, ip, ip, dp], ip),
            "cfs_eval_power": ([vp, ctypes.c_double, vp, ll, vp], ip),
            "cfs_fp64_probe": ([vp, ip, ip, vp], ip),
            "cfs_wait_check": ([vp, ctypes.c_uint], ip),
            "cfs_halo_sources": ([vp, ip, ip, ip, ip, dp], ip),
            "cfs_metric_terms": ([vp, ip, ip, ip, dp], ip),
            "cfs_finalize": ([vp, ip], ip),
            "cfs_set_schedule": ([vp, ip, ip, ip, ll, ctypes.POINTER(ctypes.c_int8)], ip),
            "cfs_set_state": ([vp, ip, vp, ip], ip),
            "cfs_get_state": ([vp, ip, vp, ip], ip),
            "cfs_set_dt": ([vp, ctypes.c_double], ip),
            "cfs_get_step": ([vp, ctypes.POINTER(ll)], ip),
            "cfs_set_step": ([vp, ll], ip),
            "cfs_step": ([vp, ll], ip),
            "cfs_diagnostics": ([vp, dp], ip),
            "cfs_ring_depth": ([vp, ctypes.POINTER(ip)], ip),
            "cfs_get_ring": ([vp, vp, ip], ip),
            "cfs_set_ring": ([vp, vp, ip], ip),
            "cfs_at_weights": ([ip, ip, dp], ip),
            "cfs_launch_count": ([vp, ctypes.POINTER(ll)], ip),
            "cfs_set_partition": ([vp, ip, ctypes.POINTER(ip), ip], ip),
            "cfs_set_exchange": ([vp, EXCHANGE_FN, vp], ip),
            "cfs_exchange_plan": ([vp, ip, ip, ctypes.POINTER(ll), ctypes.POINTER(ll)], ip),
            "cfs_exchange_count": ([vp, ctypes.POINTER(ll)], ip),
            "cfs_set_timing": ([vp, ip], ip),
            "cfs_set_graph": ([vp, ip], ip),
            "cfs_set_tiles": ([vp, ip, ip, ip], ip),
            "cfs_get_timing": ([vp, dp, ctypes.POINTER(ll)], ip),
            "cfs_mlp_forward": ([vp, vp, vp, ll, vp], ip),
            "cfs_mlp_workspace_bytes": ([ll], ctypes.c_size_t),
            "cfs_mlp_grad": ([vp, vp, vp, ll, vp, vp, vp, vp], ip),
            "cfs_mlp_adamw": ([vp, vp, vp, vp, ip, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, vp], ip),
            "cfs_halo_samples": ([vp, vp, ll, dp, vp, vp, vp], ip),
            "cfs_set_halo_model": ([vp, vp, dp, ip], ip),
            "cfs_diagnostics_static": ([vp, ip, ip, ip, dp, ip, vp, vp, ctypes.c_char_p, ctypes.c_size_t], ip),
            "cfs_last_error": ([vp], ctypes.c_char_p),
            "cfs_destroy": ([vp], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(ctx, status: int) -> None:
    if status != CFS_OK:
        msg = load().cfs_last_error(ctx)
        raise CfsError(status, msg.decode() if msg else "")


# ------------------------------------------------------------------ one-to-one wrappers

def cfs_create(params: CfsParams, stream: int | None = None):
    ctx = ctypes.c_void_p()
    st = load().cfs_create(ctypes.byref(params), ctypes.c_void_p(stream or 0), ctypes.byref(ctx))
    if st != CFS_OK:
        raise CfsError(st, "cfs_create rejected the parameters")
    return ctx


def cfs_set_allocator(ctx, alloc, free, user=None):
    _check(ctx, load().cfs_set_allocator(ctx, alloc, free, user))


def cfs_add_block(ctx, ni: int, nj: int, nk: int, spacing) -> int:
    sp = (ctypes.c_double * 3)(*spacing)
    bid = ctypes.c_int()
    _check(ctx, load().cfs_add_block(ctx, ni, nj, nk, sp, ctypes.byref(bid)))
    return bid.value


def cfs_split_block(ctx, block: int, pi: int, pj: int, pk: int):
    _check(ctx, load().cfs_split_block(ctx, block, pi, pj, pk))


def cfs_set_block_grid(ctx, block: int, xy: np.ndarray, shift):
    """Curvilinear block: xy host [2][nj][ni] point coordinates, shift = (x, y) jumps across the
    periodic wrap in i, then in j."""
    a = np.ascontiguousarray(xy, dtype=np.float64)
    sh = np.ascontiguousarray(shift, dtype=np.float64)
    assert sh.size == 4
    _check(ctx, load().cfs_set_block_grid(ctx, block, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def cfs_connect(ctx, block_a: int, face_a: int, block_b: int, face_b: int, orientation: int = 0):
    _check(ctx, load().cfs_connect(ctx, block_a, face_a, block_b, face_b, orientation))


def cfs_eval_power(x, a: float, y, stream: int | None = None):
    """y = x^a on device tensors (float64, same size) with the library's FP64 power."""
    assert x.dtype == y.dtype and x.numel() == y.numel() and x.is_cuda and y.is_cuda
    st = load().cfs_eval_power(ctypes.c_void_p(x.data_ptr()), float(a), ctypes.c_void_p(y.data_ptr()), x.numel(),
                               ctypes.c_void_p(stream or 0))
    if st != CFS_OK:
        raise CfsError(st, "cfs_eval_power failed")


def cfs_fp64_probe(sink, blocks: int, iters: int, stream: int | None = None):
    """Launch the FP64 pipe probe (blocks x 256 threads x iters x 8 FMAs) into a float64 device
    tensor of blocks x 256 elements."""
    assert sink.dtype.is_floating_point and sink.is_cuda and sink.numel() >= blocks * 256
    st = load().cfs_fp64_probe(ctypes.c_void_p(sink.data_ptr()), blocks, iters, ctypes.c_void_p(stream or 0))
    if st != CFS_OK:
        raise CfsError(st, "cfs_fp64_probe failed")


def cfs_set_partition(ctx, nranks: int, starts, rank: int):
    """Compute sub-domains [starts[rank], starts[rank + 1]) of a grid split over nranks processes."""
    st = (ctypes.c_int * (nranks + 1))(*[int(x) for x in starts])
    _check(ctx, load().cfs_set_partition(ctx, nranks, st, rank))


def cfs_set_exchange(ctx, fn):
    """Install a transport: fn(nranks, send_ptr, send_counts, recv_ptr, recv_counts, stream_ptr) -> None
    (counts in doubles per peer, device pointers as ints); an exception makes cfs_step fail with
    EXCHANGE.  Returns the ctypes callback, which the caller keeps alive."""
    def tramp(user, nranks, send, scnt, recv, rcnt, stream):
        try:
            fn(nranks, send or 0, [scnt[q] for q in range(nranks)], recv or 0, [rcnt[q] for q in range(nranks)],
               stream or 0)
            return 0
        except Exception:  # noqa: BLE001 -- reported to the library as a failed exchange
            import traceback
            traceback.print_exc()
            return 1
    cb = EXCHANGE_FN(tramp)
    _check(ctx, load().cfs_set_exchange(ctx, cb, None))
    return cb


class DeviceDoubles:
    """A device buffer of the library seen by torch (CUDA array interface, no copy)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 2}


def torch_exchange(group=None):
    """A transport for a partitioned context (Solver(..., exchange=...)) over torch.distributed
    point-to-point messages; the ranks of the partition are the ranks of `group`.  With the NCCL
    backend the packed device buffers are sent and received as they are (a batch of isend / irecv
    per exchange); with another backend (gloo) every peer's part is staged through host memory and
    the pairs exchange in rank order (the lower rank sends first), so blocking sends cannot
    deadlock.  The context's stream is synchronised before the messages (the pack kernel has
    written the send buffer) and the device after them (the unpack kernel reads the receive
    buffer).  The NCCL branch needs one GPU per process and is not exercised by the tests, which
    run on one GPU."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    nccl = dist.get_backend(group) == "nccl"

    def transport(nranks, send, scnt, recv, rcnt, stream):
        torch.cuda.synchronize()
        soff = np.concatenate([[0], np.cumsum(scnt)]).astype(np.int64)
        roff = np.concatenate([[0], np.cumsum(rcnt)]).astype(np.int64)
        sdev = torch.as_tensor(DeviceDoubles(send, max(int(soff[-1]), 1)), device="cuda")
        rdev = torch.as_tensor(DeviceDoubles(recv, max(int(roff[-1]), 1)), device="cuda")
        if nccl:
            ops = []
            for q in range(nranks):
                if q == rank:
                    continue
                if scnt[q]:
                    ops.append(dist.P2POp(dist.isend, sdev[soff[q]:soff[q + 1]], q, group))
                if rcnt[q]:
                    ops.append(dist.P2POp(dist.irecv, rdev[roff[q]:roff[q + 1]], q, group))
            if ops:
                for w in dist.batch_isend_irecv(ops):
                    w.wait()
        else:
            for q in range(nranks):
                if q == rank:
                    continue
                sb = sdev[soff[q]:soff[q + 1]].cpu()
                rb = torch.empty(int(rcnt[q]), dtype=torch.float64)
                if rank < q:
                    dist.send(sb, q, group)
                    dist.recv(rb, q, group)
                else:
                    dist.recv(rb, q, group)
                    dist.send(sb, q, group)
                rdev[roff[q]:roff[q + 1]].copy_(rb)
        torch.cuda.synchronize()

    return transport


def cfs_exchange_plan(ctx, peer: int, which: int) -> np.ndarray:
    """State offsets of the points this rank sends to (which = 0) or receives from (1) `peer`."""
    n = ctypes.c_longlong()
    _check(ctx, load().cfs_exchange_plan(ctx, peer, which, None, ctypes.byref(n)))
    out = np.zeros(max(n.value, 1), dtype=np.int64)
    _check(ctx, load().cfs_exchange_plan(ctx, peer, which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                         ctypes.byref(n)))
    return out[: n.value]


def cfs_exchange_count(ctx) -> int:
    n = ctypes.c_longlong()
    _check(ctx, load().cfs_exchange_count(ctx, ctypes.byref(n)))
    return n.value


def cfs_wait_check(ctx, limit: int):
    """Launch the bounded-wait self-test on the context's stream (the next cfs_get_state or
    cfs_diagnostics then reports ETIMEOUT once)."""
    _check(ctx, load().cfs_wait_check(ctx, limit))


def cfs_halo_sources(ctx, block: int, i: int, j: int, k: int):
    """(constant[5], [(block, i, j, k, weight, mirrored, crossed), ...]) of a point beyond a block
    face, as the kernels gather it."""
    out = np.zeros(34)
    _check(ctx, load().cfs_halo_sources(ctx, block, i, j, k, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    n = int(out[0])
    terms = [tuple(out[6 + 7 * t: 13 + 7 * t]) for t in range(n)]
    return out[1:6].copy(), [(int(a), int(b), int(c), int(d), w, int(f), int(x)) for a, b, c, d, w, f, x in terms]


def cfs_metric_terms(ctx, block: int, i: int, j: int) -> np.ndarray:
    """xi^_x, xi^_y, eta^_x, eta^_y, zeta^_z, J^-1, J at (i, j) of a curvilinear block's plane."""
    out = np.zeros(7)
    _check(ctx, load().cfs_metric_terms(ctx, block, i, j, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


BC_PERIODIC, BC_WALL, BC_FARFIELD, BC_OUTFLOW = 0, 1, 2, 3


def cfs_set_bc(ctx, block: int, face: int, bc_type: int, data=None):
    """Physical boundary on a block face: BC_WALL, BC_FARFIELD (data = 5 conserved values),
    BC_OUTFLOW, or BC_PERIODIC (back to the periodic default)."""
    if data is None:
        _check(ctx, load().cfs_set_bc(ctx, block, face, bc_type, None))
    else:
        a = np.ascontiguousarray(data, dtype=np.float64)
        assert a.size == 5
        _check(ctx, load().cfs_set_bc(ctx, block, face, bc_type, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def cfs_set_face_shift(ctx, block: int, face: int, shift):
    a = np.ascontiguousarray(shift, dtype=np.float64)
    assert a.size == 2
    _check(ctx, load().cfs_set_face_shift(ctx, block, face, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def cfs_finalize(ctx, max_delay: int):
    _check(ctx, load().cfs_finalize(ctx, max_delay))


def cfs_set_schedule(ctx, algo: int, at: int, L: int, delays: np.ndarray | None):
    if delays is None:
        _check(ctx, load().cfs_set_schedule(ctx, algo, at, L, 0, None))
        return
    d = np.ascontiguousarray(delays, dtype=np.int8)
    _check(ctx, load().cfs_set_schedule(ctx, algo, at, L, d.shape[0],
                                        d.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))))


def cfs_set_state(ctx, block: int, ptr: int, where: int):
    _check(ctx, load().cfs_set_state(ctx, block, ctypes.c_void_p(ptr), where))


def cfs_get_state(ctx, block: int, ptr: int, where: int):
    _check(ctx, load().cfs_get_state(ctx, block, ctypes.c_void_p(ptr), where))


def cfs_set_dt(ctx, dt: float):
    _check(ctx, load().cfs_set_dt(ctx, dt))


def cfs_get_step(ctx) -> int:
    n = ctypes.c_longlong()
    _check(ctx, load().cfs_get_step(ctx, ctypes.byref(n)))
    return n.value


def cfs_set_step(ctx, n: int):
    _check(ctx, load().cfs_set_step(ctx, n))


def cfs_step(ctx, nsteps: int):
    _check(ctx, load().cfs_step(ctx, nsteps))


def cfs_diagnostics(ctx, check_finite: bool = True) -> np.ndarray:
    out = np.zeros(8)
    st = load().cfs_diagnostics(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st == CFS_ENAN and not check_finite:
        return out
    _check(ctx, st)
    return out


def cfs_ring_depth(ctx) -> int:
    r = ctypes.c_int()
    _check(ctx, load().cfs_ring_depth(ctx, ctypes.byref(r)))
    return r.value


def cfs_get_ring(ctx, ptr: int, where: int):
    _check(ctx, load().cfs_get_ring(ctx, ctypes.c_void_p(ptr), where))


def cfs_set_ring(ctx, ptr: int, where: int):
    _check(ctx, load().cfs_set_ring(ctx, ctypes.c_void_p(ptr), where))


def cfs_at_weights(order: int, kmax: int) -> np.ndarray:
    s = 5 if order == 4 else 2
    C = 5 if order == 4 else 3
    W = np.zeros((kmax + 1) * s * C)
    n = load().cfs_at_weights(order, kmax, W.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if n < 0:
        raise CfsError(CFS_EINVAL, "bad order or kmax")
    return W.reshape(kmax + 1, s, C)


def cfs_launch_count(ctx) -> int:
    n = ctypes.c_longlong()
    _check(ctx, load().cfs_launch_count(ctx, ctypes.byref(n)))
    return n.value


NKINDS = 5
KIND_NAMES = ("view", "flux", "stage_update", "filter", "diagnostics")


def cfs_set_tiles(ctx, fy: int, zc: int, threads: int):
    _check(ctx, load().cfs_set_tiles(ctx, fy, zc, threads))


def cfs_set_graph(ctx, on: bool):
    _check(ctx, load().cfs_set_graph(ctx, int(on)))


def cfs_set_timing(ctx, on: bool):
    _check(ctx, load().cfs_set_timing(ctx, int(on)))


def cfs_get_timing(ctx):
    ms = np.zeros(NKINDS)
    cnt = (ctypes.c_longlong * NKINDS)()
    _check(ctx, load().cfs_get_timing(ctx, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cnt))
    return {KIND_NAMES[k]: (float(ms[k]), int(cnt[k])) for k in range(NKINDS)}


def cfs_diagnostics_static(U_ptr: int, nx: int, ny: int, nz: int, spacing, order: int, out_ptr: int,
                           stream: int | None = None) -> None:
    """Allocation-free diagnostics of a device state into a device buffer of 8 doubles."""
    sp = (ctypes.c_double * 3)(*spacing)
    buf = ctypes.create_string_buffer(256)
    st = load().cfs_diagnostics_static(ctypes.c_void_p(U_ptr), nx, ny, nz, sp, order, ctypes.c_void_p(out_ptr),
                                       ctypes.c_void_p(stream or 0), buf, 256)
    if st != CFS_OK:
        raise CfsError(st, buf.value.decode())


MLP_NIN, MLP_NOUT, MLP_NPARAM = 65, 20, 9684


def cfs_mlp_forward(params_ptr: int, x_ptr: int, y_ptr: int, n: int, stream: int | None = None):
    st = load().cfs_mlp_forward(ctypes.c_void_p(params_ptr), ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), n,
                                ctypes.c_void_p(stream or 0))
    if st != CFS_OK:
        raise CfsError(st, "cfs_mlp_forward failed")


def cfs_mlp_workspace_bytes(n: int) -> int:
    return int(load().cfs_mlp_workspace_bytes(n))


def cfs_mlp_grad(params_ptr, x_ptr, t_ptr, n, ws_ptr, grad_ptr, loss_ptr, stream=None):
    st = load().cfs_mlp_grad(ctypes.c_void_p(params_ptr), ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr), n,
                             ctypes.c_void_p(ws_ptr), ctypes.c_void_p(grad_ptr), ctypes.c_void_p(loss_ptr or 0),
                             ctypes.c_void_p(stream or 0))
    if st != CFS_OK:
        raise CfsError(st, "cfs_mlp_grad failed")


def cfs_mlp_adamw(params_ptr, grad_ptr, m_ptr, v_ptr, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0,
                  stream=None):
    st = load().cfs_mlp_adamw(ctypes.c_void_p(params_ptr), ctypes.c_void_p(grad_ptr), ctypes.c_void_p(m_ptr),
                              ctypes.c_void_p(v_ptr), step, lr, beta1, beta2, eps, wd, ctypes.c_void_p(stream or 0))
    if st != CFS_OK:
        raise CfsError(st, "cfs_mlp_adamw failed")


def cfs_halo_samples(ctx, spec_ptr: int, n: int, scales: np.ndarray, x_ptr: int, t_ptr: int, at4_ptr: int = 0):
    """Training samples (features, residual targets) at the context's current step; at4_ptr (a device
    FP32 [n][20] buffer, or 0) also receives the AT4 stage-0 residuals (Eq. 15) in target units."""
    sc = np.ascontiguousarray(scales, dtype=np.float64)
    _check(ctx, load().cfs_halo_samples(ctx, ctypes.c_void_p(spec_ptr), n, sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr), ctypes.c_void_p(at4_ptr or 0)))


def cfs_set_halo_model(ctx, params: np.ndarray | None, scales: np.ndarray | None, enable: bool = True):
    if not enable:
        _check(ctx, load().cfs_set_halo_model(ctx, None, None, 0))
        return
    p = np.ascontiguousarray(params, dtype=np.float32)
    sc = np.ascontiguousarray(scales, dtype=np.float64)
    _check(ctx, load().cfs_set_halo_model(ctx, ctypes.c_void_p(p.ctypes.data),
                                          sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1))


def cfs_last_error(ctx) -> str:
    m = load().cfs_last_error(ctx)
    return m.decode() if m else ""


def cfs_destroy(ctx):
    load().cfs_destroy(ctx)


# ------------------------------------------------------------------ convenience wrapper

def params_from_case(case, precision: int = 0) -> CfsParams:
    return CfsParams(order=case.order, viscous=int(case.viscous), visc_law=int(case.visc_law),
                     visc_exp=case.visc_exp, gamma=case.gamma, mach=case.mach, re=case.re, pr=case.pr,
                     filter=int(case.filter), alpha_f=case.alpha_f, precision=precision,
                     compact=int(getattr(case, "compact", 0)))


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator (tensors kept alive here)."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            t = self.torch.empty(int(nbytes) + 256, dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        ptr = (t.data_ptr() + 255) // 256 * 256
        self.live[ptr] = t
        return ptr

    def _free(self, ptr, user):
        self.live.pop(ptr, None)


def describe_blocks(ctx, blocks, mb=None):
    """Add the blocks (sizes, splits, curvilinear grids) to a context and, for an
    ``inputs.MultiBlock``, their interfaces and boundary conditions (cfs_connect, cfs_set_bc,
    cfs_set_face_shift)."""
    for i, b in enumerate(blocks):
        bid = cfs_add_block(ctx, b.nx, b.ny, b.nz, (b.dx, b.dy, b.dz))
        cfs_split_block(ctx, bid, b.px, b.py, b.pz)
        gxy = grid_xy(b) if mb is None else mb.xy[i]
        if gxy is not None:
            cfs_set_block_grid(ctx, bid, gxy[0], gxy[1])
    if mb is not None:
        bc = {"wall": BC_WALL, "farfield": BC_FARFIELD, "outflow": BC_OUTFLOW}
        for i, faces in enumerate(mb.faces):
            for f, F in enumerate(faces):
                if F.type == "interface" and (i, f) < (F.nb, F.nf):
                    cfs_connect(ctx, i, f, F.nb, F.nf, int(F.rev))
                elif F.type in bc:
                    cfs_set_bc(ctx, i, f, bc[F.type], F.state if F.type == "farfield" else None)
        for i, faces in enumerate(mb.faces):
            for f, F in enumerate(faces):
                if F.type == "interface" and any(F.shift):
                    cfs_set_face_shift(ctx, i, f, F.shift)


class Solver:
    """A context on the current CUDA device and stream for one periodic block (``case``), for a
    batch of independent periodic blocks (``blocks``: cases sharing the physics and scheme of the
    first, each with its own size, spacing and split), or for a connected multi-block grid
    (``case`` an ``inputs.MultiBlock``: blocks, their coordinates and their faces)."""

    def __init__(self, case, max_delay: int | None = None, precision: int = 0, stream=None,
                 use_torch_allocator: bool = True, blocks=None, tiles=None, graph: bool = False,
                 partition=None, exchange=None):
        import torch
        from .inputs import MultiBlock
        self.torch = torch
        mb = case if isinstance(case, MultiBlock) else None
        if mb is not None:
            blocks = mb.blocks
            case = mb.case
        self.blocks = list(blocks) if blocks is not None else [case]
        case = self.blocks[0]
        self.case = case
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = cfs_create(params_from_case(case, precision), self.stream.cuda_stream)
        self.alloc = None
        if use_torch_allocator:
            self.alloc = TorchAllocator(self.device)
            cfs_set_allocator(self.ctx, self.alloc.alloc_cb, self.alloc.free_cb)
        describe_blocks(self.ctx, self.blocks, mb)
        self._xcb = None
        if partition is not None:
            # (nranks, starts, rank): this process computes sub-domains starts[rank] .. starts[rank+1]-1
            cfs_set_partition(self.ctx, partition[0], partition[1], partition[2])
            if exchange is not None:
                self._xcb = cfs_set_exchange(self.ctx, exchange)
        if tiles is not None:
            cfs_set_tiles(self.ctx, *tiles)
        if max_delay is None:
            max_delay = {"SA": 0, "CAA": case.caa_L - 1, "SAA": case.kmax}[case.algo]
        cfs_finalize(self.ctx, max_delay)
        self.npts = case.nx * case.ny * case.nz
        cfs_set_dt(self.ctx, case.dt)
        if graph:
            cfs_set_graph(self.ctx, True)

    def set_schedule(self, algo: str | None = None, at: bool | None = None, L: int | None = None,
                     delays: np.ndarray | None = None):
        c = self.case
        algo = c.algo if algo is None else algo
        at = c.at if at is None else at
        L = c.caa_L if L is None else L
        cfs_set_schedule(self.ctx, ALGO[algo], int(at), L, delays if algo == "SAA" else None)

    def set_state(self, U, block: int = 0):
        """U: numpy array (host) or CUDA tensor (device), FP64 [5][nz][ny][nx] of the block."""
        b = self.blocks[block]
        n = 5 * b.nx * b.ny * b.nz
        if isinstance(U, np.ndarray):
            a = np.ascontiguousarray(U, dtype=np.float64)
            assert a.size == n
            cfs_set_state(self.ctx, block, a.ctypes.data, HOST)
        else:
            t = U.contiguous()
            assert t.dtype == self.torch.float64 and t.numel() == n and t.is_cuda
            cfs_set_state(self.ctx, block, t.data_ptr(), DEVICE)

    def get_state(self, out=None, block: int = 0):
        """Current state of a block to a new numpy array, or into ``out`` (numpy or CUDA tensor)."""
        c = self.blocks[block]
        if out is None:
            out = np.empty((5, c.nz, c.ny, c.nx), dtype=np.float64)
        if isinstance(out, np.ndarray):
            assert out.flags.c_contiguous and out.dtype == np.float64
            cfs_get_state(self.ctx, block, out.ctypes.data, HOST)
        else:
            cfs_get_state(self.ctx, block, out.data_ptr(), DEVICE)
        return out

    def set_states(self, states):
        """Every block's state, in block order."""
        for i, U in enumerate(states):
            self.set_state(U, block=i)

    def get_states(self) -> list:
        return [self.get_state(block=i) for i in range(len(self.blocks))]

    def step(self, n: int = 1):
        cfs_step(self.ctx, n)

    def diagnostics(self, check_finite: bool = True) -> np.ndarray:
        return cfs_diagnostics(self.ctx, check_finite)

    @property
    def n(self) -> int:
        return cfs_get_step(self.ctx)

    def set_step(self, n: int):
        cfs_set_step(self.ctx, n)

    def launches(self) -> int:
        return cfs_launch_count(self.ctx)

    def close(self):
        if self.ctx is not None:
            cfs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
