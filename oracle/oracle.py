"""Python access to the FP64 CPU oracle (``cfs_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is the plain, slow reference the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this module.  It shares no code with the product library; it is compiled with gcc from
its single C file and loaded with ctypes.

Every function cites the passage of arXiv 2506.03027 it restates (see the C file's header).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cfs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcfs_oracle.so")
_lock = threading.Lock()
_lib = None


class OrFace(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("nb", ctypes.c_int), ("nf", ctypes.c_int), ("rev", ctypes.c_int),
                ("state", ctypes.c_double * 5), ("shift", ctypes.c_double * 2)]


class OrBlock(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("px", ctypes.c_int), ("py", ctypes.c_int), ("pz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("grid_xy", ctypes.POINTER(ctypes.c_double)), ("grid_shift", ctypes.c_double * 4),
        ("face", OrFace * 6),
    ]


class OrParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("px", ctypes.c_int), ("py", ctypes.c_int), ("pz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("gamma", ctypes.c_double), ("mach", ctypes.c_double), ("re", ctypes.c_double),
        ("pr", ctypes.c_double),
        ("viscous", ctypes.c_int), ("visc_law", ctypes.c_int), ("visc_exp", ctypes.c_double),
        ("order", ctypes.c_int), ("algo", ctypes.c_int), ("at", ctypes.c_int),
        ("caa_L", ctypes.c_int), ("kmax", ctypes.c_int),
        ("filter", ctypes.c_int), ("alpha_f", ctypes.c_double), ("dt", ctypes.c_double),
        ("mlp", ctypes.POINTER(ctypes.c_float)), ("mlp_scales", ctypes.POINTER(ctypes.c_double)),
        ("grid_xy", ctypes.POINTER(ctypes.c_double)), ("grid_shift", ctypes.c_double * 4),
        ("nblocks", ctypes.c_int), ("blocks", ctypes.POINTER(OrBlock)),
        ("compact", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + optional OpenMP); returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d = P(ctypes.c_double)
            lib.or_run.argtypes = [P(OrParams), d, P(ctypes.c_int8), ctypes.c_long, ctypes.c_long, d, d]
            lib.or_run.restype = ctypes.c_int
            lib.or_rhs.argtypes = [P(OrParams), d, d]
            lib.or_rhs.restype = ctypes.c_int
            lib.or_diagnostics.argtypes = [P(OrParams), d, d]
            lib.or_extrap_weights.argtypes = [ctypes.c_int, ctypes.c_double, d]
            lib.or_buffer_dudt.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, d]
            lib.or_nu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.or_nu.restype = ctypes.c_double
            lib.or_lserk.argtypes = [ctypes.c_int, d, d]
            lib.or_lserk.restype = ctypes.c_int
            lib.or_filter_coeffs.argtypes = [ctypes.c_double, d]
            lib.or_filter_line.argtypes = [ctypes.c_int, ctypes.c_double, d, d]
            lib.or_compact_line.argtypes = [ctypes.c_int, ctypes.c_double, d, d]
            lib.or_compact_line.restype = None
            lib.or_num_threads.restype = ctypes.c_int
            lib.or_bf16.argtypes = [ctypes.c_double]
            lib.or_bf16.restype = ctypes.c_double
            lib.or_mlp_forward.argtypes = [ctypes.POINTER(ctypes.c_float), d, d]
            lib.or_column_features.argtypes = [P(OrParams), P(d), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, d, d]
            lib.or_column_features.restype = None
            lib.or_set_num_threads.argtypes = [ctypes.c_int]
            lib.or_halo_sources.argtypes = [P(OrParams), ctypes.c_int, ctypes.c_long, P(ctypes.c_int), d]
            lib.or_halo_sources.restype = ctypes.c_int
            lib.or_metric_terms.argtypes = [P(OrParams), ctypes.c_int, ctypes.c_long, P(ctypes.c_int), d]
            lib.or_metric_terms.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


ALGOS = {"SA": 0, "CAA": 1, "SAA": 2}


def params(case) -> OrParams:
    """Translate a ``inputs.Case`` (or ``inputs.MultiBlock``) description into the oracle's
    parameter struct (point coordinates and block tables are kept alive on the struct)."""
    from paper_2506_03027_gb300.inputs import MultiBlock, FACE_TYPES
    if isinstance(case, MultiBlock):
        mb = case
        p = params(mb.case.replace(curv=0.0))
        arr = (OrBlock * len(mb.blocks))()
        keep = []
        for i, (b, faces, g) in enumerate(zip(mb.blocks, mb.faces, mb.xy)):
            B = arr[i]
            B.nx, B.ny, B.nz, B.px, B.py, B.pz = b.nx, b.ny, b.nz, b.px, b.py, b.pz
            B.dx, B.dy, B.dz = b.dx, b.dy, b.dz
            if g is not None:
                xy = np.ascontiguousarray(g[0], dtype=np.float64)
                keep.append(xy)
                B.grid_xy = _dptr(xy)
                for q in range(4):
                    B.grid_shift[q] = float(g[1][q])
            for f, F in enumerate(faces):
                B.face[f].type = FACE_TYPES[F.type]
                B.face[f].nb, B.face[f].nf, B.face[f].rev = F.nb, F.nf, int(F.rev)
                for v in range(5):
                    B.face[f].state[v] = float(F.state[v])
                for q in range(2):
                    B.face[f].shift[q] = float(F.shift[q])
        p._blocks = arr
        p._keep = keep
        p.nblocks = len(mb.blocks)
        p.blocks = ctypes.cast(arr, ctypes.POINTER(OrBlock))
        return p
    p = OrParams(
        nx=case.nx, ny=case.ny, nz=case.nz, px=case.px, py=case.py, pz=case.pz,
        dx=case.dx, dy=case.dy, dz=case.dz, gamma=case.gamma, mach=case.mach, re=case.re,
        pr=case.pr, viscous=int(case.viscous), visc_law=int(case.visc_law),
        visc_exp=case.visc_exp, order=case.order, algo=ALGOS[case.algo], at=int(case.at),
        caa_L=case.caa_L, kmax=case.kmax, filter=int(case.filter), alpha_f=case.alpha_f,
        dt=case.dt, compact=int(getattr(case, "compact", 0)))
    from paper_2506_03027_gb300.inputs import grid_xy
    g = grid_xy(case)
    if g is not None:
        p._xy = g[0]
        p.grid_xy = _dptr(g[0])
        for i in range(4):
            p.grid_shift[i] = float(g[1][i])
    return p


def run(case, U0: np.ndarray, nsteps: int, delays: np.ndarray | None = None, n0: int = 0,
        hist: np.ndarray | None = None, diag: bool = False, model=None):
    """Advance ``nsteps`` steps of the method (Alg. 1-3 with Eq. 3, 8, 14-15); returns U
    (and the per-step diagnostics [nsteps][8] if ``diag``).  ``model`` = (params float32[9684],
    scales float64[15]) replaces the stage-0 face halos of AT steps by the learned predictor."""
    lib = _load()
    p = params(case)
    if model is not None:
        mp = np.ascontiguousarray(model[0], dtype=np.float32)
        ms = np.ascontiguousarray(model[1], dtype=np.float64)
        p.mlp = mp.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        p.mlp_scales = ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    from paper_2506_03027_gb300.inputs import MultiBlock, join_states, split_states
    multi = isinstance(case, MultiBlock)
    U = join_states(U0) if multi else np.ascontiguousarray(U0, dtype=np.float64).copy()
    if delays is None:
        dl = np.zeros(1, dtype=np.int8)
    else:
        dl = np.ascontiguousarray(delays, dtype=np.int8)
    hp = None if hist is None else _dptr(np.ascontiguousarray(hist, dtype=np.float64))
    dg = np.zeros((max(nsteps, 1), 8), dtype=np.float64) if diag else None
    rc = lib.or_run(ctypes.byref(p), _dptr(U), dl.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                    n0, nsteps, hp, _dptr(dg) if diag else None)
    if rc != 0:
        raise ValueError(f"oracle rejected the case (code {rc})")
    if multi:
        U = split_states(case, U)
    return (U, dg[:nsteps]) if diag else U


def rhs(case, U: np.ndarray) -> np.ndarray:
    """R(U) of Eq. 1 with synchronous halos (the CD right-hand side of the whole field)."""
    from paper_2506_03027_gb300.inputs import MultiBlock, join_states, split_states
    lib = _load()
    p = params(case)
    multi = isinstance(case, MultiBlock)
    U = join_states(U) if multi else np.ascontiguousarray(U, dtype=np.float64)
    R = np.zeros_like(U)
    if lib.or_rhs(ctypes.byref(p), _dptr(U), _dptr(R)) != 0:
        raise ValueError("oracle rejected the case")
    return split_states(case, R) if multi else R


def diagnostics(case, U: np.ndarray) -> np.ndarray:
    """[K, enstrophy, sum rho, sum rho u, sum rho v, sum rho w, sum rho E, nan-flag]."""
    from paper_2506_03027_gb300.inputs import MultiBlock, join_states
    lib = _load()
    p = params(case)
    U = join_states(U) if isinstance(case, MultiBlock) else np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros(8)
    if lib.or_diagnostics(ctypes.byref(p), _dptr(U), _dptr(out)) != 0:
        raise ValueError("oracle rejected the case")
    return out


def extrap_weights(order: int, k: float) -> np.ndarray:
    """Eq. 14 (order 2) / Eq. 15 (order 4)."""
    c = np.zeros(5)
    _load().or_extrap_weights(order, float(k), _dptr(c))
    return c[: (5 if order == 4 else 3)]


def buffer_dudt(order: int, e: int, k: float) -> np.ndarray:
    """App. C: dt * dphi/dt at stage e as weights on levels n-k, n-k-1, ..."""
    d = np.zeros(5)
    _load().or_buffer_dudt(order, e, float(k), _dptr(d))
    return d[: (5 if order == 4 else 3)]


def nu(order: int, e: int, j: int) -> float:
    """Eq. 10: nu_j^e."""
    return _load().or_nu(order, e, j)


def lserk(order: int):
    """Table 4 / App. B LSERK coefficients (A, B)."""
    A = np.zeros(5)
    B = np.zeros(5)
    s = _load().or_lserk(order, _dptr(A), _dptr(B))
    return A[:s], B[:s]


def filter_coeffs(alpha: float) -> np.ndarray:
    a = np.zeros(6)
    _load().or_filter_coeffs(alpha, _dptr(a))
    return a


def filter_line(alpha: float, f: np.ndarray) -> np.ndarray:
    """Filter one line: f holds n values plus 5 halo values on each side."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    n = f.size - 10
    out = np.zeros(n)
    _load().or_filter_line(n, alpha, _dptr(f), _dptr(out))
    return out


def compact_line(h: float, f: np.ndarray) -> np.ndarray:
    """Sixth-order compact derivative (Eq. 2, alpha = 1/3) of one line: f holds n values plus 4
    halo values on each side; returns the n derivatives."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    n = f.size - 8
    out = np.zeros(n)
    _load().or_compact_line(n, float(h), _dptr(f), _dptr(out))
    return out


def num_threads() -> int:
    return _load().or_num_threads()


def set_num_threads(n: int) -> None:
    _load().or_set_num_threads(n)


def bf16(x: float) -> float:
    """FP64 -> FP32 -> BF16 (round to nearest even), the feature rounding of the learned halo."""
    return _load().or_bf16(float(x))


def mlp_forward_c(params: np.ndarray, x: np.ndarray) -> np.ndarray:
    """The C oracle's FP64 forward pass of the halo network for one feature vector."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(20)
    _load().or_mlp_forward(p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _dptr(xx), _dptr(y))
    return y


def column_features(case, levels, scales, sub: int, face: int, t1: int, t2: int, k: int):
    """The learned halo's input features of one face column and its 3-level extrapolation, as the
    oracle builds them: levels = (U^n, U^{n-k}, U^{n-k-1}, U^{n-k-2}) full states, scales[15] =
    (in_scale[5], own_scale[5], out_scale[5]).  Returns (x[65], at3[20])."""
    p = params(case)
    sc = np.ascontiguousarray(scales, dtype=np.float64)
    p.mlp_scales = _dptr(sc)
    lv = [np.ascontiguousarray(L, dtype=np.float64) for L in levels]
    ptrs = (ctypes.POINTER(ctypes.c_double) * 4)(*[_dptr(L) for L in lv])
    x = np.zeros(65)
    at3 = np.zeros(20)
    _load().or_column_features(ctypes.byref(p), ptrs, sub, face, t1, t2, k, _dptr(x), _dptr(at3))
    return x, at3


def halo_sources(case, block: int, points):
    """Per point (i, j, k) of ``points`` beyond a block face: (constant[5], [(block, i, j, k, weight,
    mirrored, crossed), ...]) as the oracle resolves it."""
    p = params(case)
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((len(pts), 34))
    if _load().or_halo_sources(ctypes.byref(p), block, len(pts), pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               _dptr(out)) != 0:
        raise ValueError("oracle rejected a point or the description")
    res = []
    for row in out:
        n = int(row[0])
        terms = [tuple(row[6 + 7 * t: 13 + 7 * t]) for t in range(n)]
        res.append((row[1:6].copy(), [(int(a), int(b), int(c), int(d), w, int(f), int(x)) for a, b, c, d, w, f, x in terms]))
    return res


def metric_terms(case, block: int, points) -> np.ndarray:
    """[npts][6] metric terms (xi^_x, xi^_y, eta^_x, eta^_y, zeta^_z, J^-1) at (i, j) points of a
    curvilinear block's extended plane, as the oracle computes them."""
    p = params(case)
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int32).reshape(-1, 2))
    out = np.zeros((len(pts), 6))
    if _load().or_metric_terms(ctypes.byref(p), block, len(pts), pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               _dptr(out)) != 0:
        raise ValueError("oracle rejected the block or the description")
    return out

