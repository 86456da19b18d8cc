"""Plain FP64 CPU oracle of multi-level greedy RBF mesh deformation.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
and by the benchmark's CPU-baseline leg.  The CUDA library never imports,
links or executes anything in this directory, and this directory imports
nothing from the CUDA library.

The arithmetic lives in ``rbfd_oracle.c`` (plain C, every step cited to the
paper's section / equation); this module only compiles it with gcc and
marshals numpy arrays through ctypes.

Parity pins for every function: ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import hashlib
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbfd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "librbfd_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ESINGULAR, ENOTCONV = 0, 1, 2, 3, 4
BASIS = {"C0": 0, "C2": 2, "C4": 4, "C6": 6}


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle C source (gcc, -O2, -ffp-contract=off, OpenMP when
    the compiler supports it) into a shared library; returns its path."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    # the source's hash and the machine: a library built elsewhere or from
    # another source is never taken for current
    with open(src, "rb") as fh:
        stamp = hashlib.sha256(platform.machine().encode() + fh.read()).hexdigest()
    stamp_path = out + ".stamp"
    if not force and os.path.exists(out) and os.path.exists(stamp_path):
        with open(stamp_path) as fh:
            if fh.read().strip() == stamp:
                return out
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]
    tmp = out + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", src, "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [src, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, out)
    with open(stamp_path, "w") as fh:
        fh.write(stamp + "\n")
    return out


def _bind(path: str):
    lib = ctypes.CDLL(path)
    i64p = ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_phi.restype = ctypes.c_double
    lib.orc_phi.argtypes = [ctypes.c_int, ctypes.c_double]
    lib.orc_psi.restype = ctypes.c_double
    lib.orc_psi.argtypes = [ctypes.c_double]
    lib.orc_cholesky.restype = ctypes.c_int
    lib.orc_cholesky.argtypes = [ctypes.c_int64, dp, ctypes.c_int64, dp, ctypes.c_int64]
    lib.orc_chol_solve.restype = None
    lib.orc_chol_solve.argtypes = [ctypes.c_int64, dp, ctypes.c_int64, ctypes.c_int, dp, dp]
    lib.orc_eval.restype = None
    lib.orc_eval.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int64, dp, dp,
                             ctypes.c_int64, dp, dp, ctypes.c_int]
    lib.orc_greedy.restype = ctypes.c_int
    lib.orc_greedy.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int, dp, ctypes.c_double,
                               ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               i64p, i64p, dp, dp, dp, dp, dp, dp]
    lib.orc_replay.restype = ctypes.c_int
    lib.orc_replay.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int, dp, ctypes.c_int,
                               ctypes.c_int64, i64p, i64p, ctypes.c_int, dp, dp, dp, dp, dp, dp]
    lib.orc_support_distances.restype = None
    lib.orc_support_distances.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp]
    lib.orc_deform.restype = ctypes.c_int
    lib.orc_deform.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, i64p, i64p, dp,
                               ctypes.c_int64, dp, ctypes.c_int64, dp, dp, dp, ctypes.c_int]
    lib.orc_max_threads.restype = ctypes.c_int
    lib.orc_max_threads.argtypes = []
    fp = ctypes.POINTER(ctypes.c_float)
    lib.orc_orthogonality.restype = ctypes.c_int
    lib.orc_orthogonality.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                      dp, dp, fp, fp, dp, dp]
    lib.orc_wall_distance.restype = None
    lib.orc_wall_distance.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ctypes.c_int64, dp, dp, ctypes.c_int]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
        return _lib


def load_variant(path: str):
    """Bind another build of the oracle source (used by the mutation tests,
    which compile deliberately broken copies to show that the pins catch
    them).  Returns a ``Variant`` exposing the same functions."""
    return Variant(_bind(path))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def max_threads() -> int:
    return int(_load().orc_max_threads())


def phi(eta, basis: str = "C2", lib=None):
    """Wendland basis of Table 1 at each eta (Eq. 2 for C2)."""
    lib = lib or _load()
    b = BASIS[basis]
    eta = np.asarray(eta, dtype=np.float64)
    return np.vectorize(lambda e: lib.orc_phi(b, float(e)), otypes=[np.float64])(eta)


def psi(xi, lib=None):
    """Wall-distance function of Section 4."""
    lib = lib or _load()
    xi = np.asarray(xi, dtype=np.float64)
    return np.vectorize(lambda x: lib.orc_psi(float(x)), otypes=[np.float64])(xi)


def cholesky(A, lib=None):
    """Row-oriented Cholesky factor L (lower) of SPD A, or None if not SPD."""
    lib = lib or _load()
    A = _f64(A)
    n = A.shape[0]
    L = np.zeros_like(A)
    rc = lib.orc_cholesky(n, _dp(A), n, _dp(L), n)
    return None if rc != 0 else L


def chol_solve(L, B, lib=None):
    """Solve L L^T X = B by forward then back substitution."""
    lib = lib or _load()
    L = _f64(L)
    B = _f64(B)
    n = L.shape[0]
    nrhs = 1 if B.ndim == 1 else B.shape[1]
    X = np.zeros((n, nrhs))
    lib.orc_chol_solve(n, _dp(L), n, nrhs, _dp(B.reshape(n, nrhs)), _dp(X))
    return X.reshape(B.shape)


def evaluate(xyz_c, alpha, xyz_p, R: float, basis: str = "C2", n_threads: int = 1, lib=None):
    """f(r) = sum_j alpha_j phi(|r - r_cj| / R) at each point (Eq. 1)."""
    lib = lib or _load()
    xyz_c = _f64(xyz_c)
    alpha = _f64(alpha)
    xyz_p = _f64(xyz_p)
    dim = xyz_p.shape[1]
    f = np.zeros((xyz_p.shape[0], dim))
    lib.orc_eval(dim, BASIS[basis], float(R), xyz_c.shape[0], _dp(xyz_c), _dp(alpha),
                 xyz_p.shape[0], _dp(xyz_p), _dp(f), int(n_threads))
    return f


@dataclasses.dataclass
class GreedyResult:
    status: int
    idx: list  # per level: int64 array of surface indices, selection order
    alpha: list  # per level: [nc, dim] weights
    smax: np.ndarray  # per level: max_i |dS_l,i|
    emax: np.ndarray  # per level: max_i |E_i| / S0 after the level
    gap: np.ndarray  # per level: smallest relative top-2 key gap seen
    E: np.ndarray  # final error [n_s, dim]
    S0: float
    step_gap: list = None  # per level: [nc] relative top-2 gap of the step that picked control k (k >= 1)

    @property
    def n_levels(self):
        return len(self.idx)


def greedy(xyz_s, dS, R, eps, basis="C2", nc_cap=None, first_rule=0, solve_mode=0, n_threads=1,
           lib=None):
    """Multi-level greedy selection of Section 3 (see rbfd_oracle.c)."""
    lib = lib or _load()
    xyz_s = _f64(xyz_s)
    dS = _f64(dS)
    n_s, dim = xyz_s.shape
    R = _f64(np.atleast_1d(R))
    L = R.shape[0]
    cap = int(min(n_s, 8192) if nc_cap is None else min(nc_cap, n_s))
    nc = np.zeros(L, dtype=np.int64)
    idx = np.zeros(L * cap, dtype=np.int64)
    alpha = np.zeros(L * cap * dim)
    smax = np.zeros(L)
    emax = np.zeros(L)
    gap = np.zeros(L)
    E = np.zeros((n_s, dim))
    sg = np.ones(L * cap)
    rc = lib.orc_greedy(dim, n_s, _dp(xyz_s), _dp(dS), L, _dp(R), float(eps), BASIS[basis], cap,
                        int(first_rule), int(solve_mode), int(n_threads), _ip(nc), _ip(idx), _dp(alpha),
                        _dp(smax), _dp(emax), _dp(E), _dp(gap), _dp(sg))
    if rc in (EINVAL, ENOMEM, ESINGULAR):
        raise RuntimeError(f"oracle greedy failed with status {rc}")
    idx = idx.reshape(L, cap)
    alpha = alpha.reshape(L, cap, dim)
    S0 = float(np.sqrt((dS * dS).sum(1)).max()) if n_s else 0.0
    sg = sg.reshape(L, cap)
    return GreedyResult(rc, [idx[l, : nc[l]].copy() for l in range(L)],
                        [alpha[l, : nc[l]].copy() for l in range(L)], smax, emax, gap, E, S0,
                        [sg[l, : nc[l]].copy() for l in range(L)])


@dataclasses.dataclass
class ReplayResult:
    """Per level l, per slot k = 1 .. n_l (before given control k is added;
    slot n_l after the last one): the largest key among unselected points,
    the key of the given control (of that best point at slot n_l), and the
    rounding scales |dS_l,i| + sum_j |alpha_j| phi_ij of E at both points."""
    best_key: list
    pick_key: list
    best_scale: list
    pick_scale: list
    alpha: list
    smax: np.ndarray


def replay(xyz_s, dS, R, given, basis="C2", n_threads=1, lib=None):
    """Replay the control sequences ``given`` (one index array per level)
    through the greedy of Section 3 (see orc_replay in rbfd_oracle.c)."""
    lib = lib or _load()
    xyz_s = _f64(xyz_s)
    dS = _f64(dS)
    n_s, dim = xyz_s.shape
    R = _f64(np.atleast_1d(R))
    L = R.shape[0]
    if len(given) != L:
        raise ValueError("one given sequence per level")
    cap = max(1, max(len(g) for g in given))
    gnc = np.array([len(g) for g in given], dtype=np.int64)
    gidx = np.zeros((L, cap), dtype=np.int64)
    for l, g in enumerate(given):
        gidx[l, : len(g)] = np.asarray(g, dtype=np.int64)
    alpha = np.zeros(L * cap * dim)
    smax = np.zeros(L)
    bk, pk, bs, ps = (np.zeros(L * (cap + 1)) for _ in range(4))
    rc = lib.orc_replay(dim, n_s, _dp(xyz_s), _dp(dS), L, _dp(R), BASIS[basis], cap, _ip(gnc),
                        _ip(gidx.reshape(-1)), int(n_threads), _dp(alpha), _dp(smax), _dp(bk), _dp(pk), _dp(bs),
                        _dp(ps))
    if rc != OK:
        raise RuntimeError(f"oracle replay failed with status {rc}")
    alpha = alpha.reshape(L, cap, dim)
    cut = lambda a: [a.reshape(L, cap + 1)[l, 1 : gnc[l] + 1].copy() for l in range(L)]
    return ReplayResult(cut(bk), cut(pk), cut(bs), cut(ps), [alpha[l, : gnc[l]].copy() for l in range(L)], smax)


def support_distances(smax, k: float, D: float, lib=None):
    """D_l of Section 4 for each level."""
    lib = lib or _load()
    smax = _f64(smax)
    out = np.zeros_like(smax)
    lib.orc_support_distances(smax.shape[0], _dp(smax), float(k), float(D), _dp(out))
    return out


def deform(res: GreedyResult, xyz_s, R, xyz_v, d_v, k: float, D: float, basis="C2", n_threads=1,
           lib=None):
    """Volume update of Eq. 19 blended by psi (Eq. 23), brute force, FP64."""
    lib = lib or _load()
    xyz_s = _f64(xyz_s)
    xyz_v = _f64(xyz_v)
    d_v = _f64(d_v)
    dim = xyz_s.shape[1]
    L = res.n_levels
    R = _f64(np.atleast_1d(R))
    Dl = support_distances(res.smax, k, D, lib=lib)
    cap = max([len(i) for i in res.idx] + [1])
    nc = np.array([len(i) for i in res.idx], dtype=np.int64)
    idx = np.zeros((L, cap), dtype=np.int64)
    al = np.zeros((L, cap, dim))
    for l in range(L):
        idx[l, : nc[l]] = res.idx[l]
        al[l, : nc[l]] = res.alpha[l]
    out = np.zeros((xyz_v.shape[0], dim))
    rc = lib.orc_deform(dim, BASIS[basis], L, _dp(R), _dp(Dl), _ip(nc), _ip(idx.reshape(-1)),
                        _dp(al.reshape(-1)), cap, _dp(xyz_s), xyz_v.shape[0], _dp(xyz_v), _dp(d_v),
                        _dp(out), int(n_threads))
    if rc != OK:
        raise RuntimeError(f"oracle deform failed with status {rc}")
    return out


def wall_distance(xyz_s, xyz_v, n_threads=1, lib=None):
    """Distance from each volume point to its nearest surface point (brute force)."""
    lib = lib or _load()
    xyz_s = _f64(xyz_s)
    xyz_v = _f64(xyz_v)
    d = np.zeros(xyz_v.shape[0])
    lib.orc_wall_distance(xyz_s.shape[1], xyz_s.shape[0], _dp(xyz_s), xyz_v.shape[0], _dp(xyz_v), _dp(d),
                          int(n_threads))
    return d


@dataclasses.dataclass
class Quality:
    theta: np.ndarray     # per cell, degrees in [0, 90]
    min_deg: float
    mean_deg: float
    argmin: int
    cells: int
    tangled: int
    hist: np.ndarray      # cells per 10-degree bin


def orthogonality(wall, vol, n_layers, periodic_i=True, wall_disp=None, vol_disp=None, n_k=1, lib=None):
    """Orthogonality angle of each cell of the structured grid grown off the
    surface: ``wall`` [n_k * n_i][dim] (FP64), ``vol`` [n_k * n_i * n_layers][dim]
    (FP32, wall-normal index fastest), displacements optional."""
    lib = lib or _load()
    wall = _f64(wall)
    dim = wall.shape[1]
    n_i = wall.shape[0] // n_k
    vol = np.ascontiguousarray(vol, dtype=np.float32)
    wd = None if wall_disp is None else _f64(wall_disp)
    vd = None if vol_disp is None else np.ascontiguousarray(vol_disp, dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    fptr = lambda a: None if a is None else a.ctypes.data_as(fp)
    n_ci = n_i if periodic_i else n_i - 1
    n_ck = n_k - 1 if dim == 3 else 1
    theta = np.zeros(max(n_ck * n_ci * n_layers, 0))
    summ = np.zeros(14)
    rc = lib.orc_orthogonality(dim, n_i, n_k, n_layers, 1 if periodic_i else 0, _dp(wall),
                               None if wd is None else _dp(wd), fptr(vol), fptr(vd), _dp(theta), _dp(summ))
    if rc != OK:
        raise ValueError(f"oracle orthogonality: bad arguments (status {rc})")
    return Quality(theta, summ[0], summ[1], int(summ[2]), int(summ[3]), int(summ[4]), summ[5:].astype(np.int64))


class Variant:
    """The oracle's functions bound to one specific build of its source."""

    def __init__(self, lib):
        self.lib = lib

    def __getattr__(self, name):
        fn = globals()[name]
        return lambda *a, **kw: fn(*a, lib=self.lib, **kw)
