"""ctypes binding of the rbfd C ABI (``include/rbfd.h``).

Argument marshalling only: every step of the method runs in the CUDA library
``_build/librbfd.so``.  The functions keep the C names; ``Mesh`` wraps a handle.
Host arrays are numpy arrays; device arrays are torch CUDA tensors (pass
``inputs_on_device=True`` at creation).  If the library cannot be built or
loaded, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ESINGULAR, ENOTCONV, ETIMEOUT, EBUSY, ECUDA, ESTATE, ECOMM, ECANCELED = range(11)
FP64, MIXED = 0, 1
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ESINGULAR", 4: "ENOTCONV", 5: "ETIMEOUT", 6: "EBUSY",
                7: "ECUDA", 8: "ESTATE", 9: "ECOMM", 10: "ECANCELED"}


class RbfdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class rbfd_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("basis", ctypes.c_int),
        ("first_point", ctypes.c_int),
        ("inputs_on_device", ctypes.c_int),
        ("nc_cap", ctypes.c_int64),
        ("stream", ctypes.c_void_p),
        ("eps_absolute", ctypes.c_int),
        ("refine_iters", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("engine", ctypes.c_int),
        ("grid_ctas", ctypes.c_int),
        ("prune", ctypes.c_int),
    ]


class rbfd_stats(ctypes.Structure):
    _fields_ = [
        ("greedy_ms", ctypes.c_double),
        ("deform_ms", ctypes.c_double),
        ("greedy_steps", ctypes.c_int64),
        ("pairs_useful", ctypes.c_int64),
        ("pairs_visited", ctypes.c_int64),
        ("deform_points", ctypes.c_int64),
        ("refine_sweeps", ctypes.c_int64),
        ("confirm_resumes", ctypes.c_int64),
        ("launches", ctypes.c_int64),
        ("sweep_ms", ctypes.c_double),
        ("grow_ms", ctypes.c_double),
        ("vol_ms", ctypes.c_double),
        ("sweep_launches", ctypes.c_int64),
        ("grow_launches", ctypes.c_int64),
        ("vol_launches", ctypes.c_int64),
        ("sweep_pairs_useful", ctypes.c_int64),
        ("sweep_pairs_visited", ctypes.c_int64),
        ("vol_pairs_useful", ctypes.c_int64),
        ("vol_pairs_visited", ctypes.c_int64),
        ("persist_ms", ctypes.c_double),
        ("persist_launches", ctypes.c_int64),
        ("persist_ctas", ctypes.c_int64),
        ("persist_phase_ms", ctypes.c_double * 8),
        ("wall_ms", ctypes.c_double),
        ("wall_launches", ctypes.c_int64),
        ("wall_pairs_search", ctypes.c_int64),
        ("wall_pairs_exact", ctypes.c_int64),
        ("newton_steps", ctypes.c_int64),
        ("newton_ms", ctypes.c_double),
        ("newton_launches", ctypes.c_int64),
        ("newton_terms", ctypes.c_int64),
        ("greedy_host_ms", ctypes.c_double * 4),
        ("newton_pairs_useful", ctypes.c_int64),
        ("newton_pairs_formed", ctypes.c_int64),
        ("eq12_pairs", ctypes.c_int64),
        ("persist_grow_fma", ctypes.c_int64),
        ("sweep_pairs_skipped", ctypes.c_int64),
        ("sweep_warps_skipped", ctypes.c_int64),
    ]


class rbfd_quality(ctypes.Structure):
    _fields_ = [
        ("min_deg", ctypes.c_double),
        ("mean_deg", ctypes.c_double),
        ("argmin", ctypes.c_int64),
        ("cells", ctypes.c_int64),
        ("tangled", ctypes.c_int64),
        ("hist", ctypes.c_int64 * 9),
    ]


class rbfd_server_options(ctypes.Structure):
    _fields_ = [
        ("slots", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("mem_budget_bytes", ctypes.c_int64),
        ("max_queue", ctypes.c_int64),
        ("fuse_volume", ctypes.c_int),
    ]


class rbfd_request(ctypes.Structure):
    _fields_ = [("dS", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class rbfd_job(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n_levels", ctypes.c_int),
        ("n_s", ctypes.c_int64),
        ("xyz_s", ctypes.c_void_p),
        ("dS", ctypes.c_void_p),
        ("R", ctypes.c_void_p),
        ("eps", ctypes.c_double),
        ("opt", ctypes.POINTER(rbfd_options)),
        ("n_v", ctypes.c_int64),
        ("xyz_v", ctypes.c_void_p),
        ("d_v", ctypes.c_void_p),
        ("D", ctypes.c_double),
        ("k", ctypes.c_double),
        ("out", ctypes.c_void_p),
    ]


class rbfd_worklist_tune(ctypes.Structure):
    _fields_ = [
        ("autotune", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("item_blocks", ctypes.c_int),
        ("cell_div", ctypes.c_int * 16),
        ("cached", ctypes.c_int),
        ("trials", ctypes.c_int),
        ("launch_ms", ctypes.c_double),
        ("items", ctypes.c_int64),
    ]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = 0, 1, 2, 3, 4

# int maxloc(void *user, double *key, int64_t *idx) (rbfd_greedy_split)
MAXLOC_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_int64))

# (name, restype, argtypes) of every function include/rbfd.h declares
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_d = ctypes.c_double
SIGNATURES = [
    ("rbfd_options_default", None, [ctypes.POINTER(rbfd_options)]),
    ("rbfd_create", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _i64, _vp, _vp, ctypes.c_int, _vp, _d,
                                   ctypes.POINTER(rbfd_options)]),
    ("rbfd_greedy", ctypes.c_int, [_vp]),
    ("rbfd_greedy_warm", ctypes.c_int, [_vp]),
    ("rbfd_greedy_split", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, MAXLOC_FN, _vp]),
    ("rbfd_get_level", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_i64), _vp, _vp, ctypes.POINTER(_d)]),
    ("rbfd_num_levels", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    ("rbfd_level_info", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_d), ctypes.POINTER(_d),
                                       ctypes.POINTER(_d)]),
    ("rbfd_get_stats", ctypes.c_int, [_vp, ctypes.POINTER(rbfd_stats)]),
    ("rbfd_deform", ctypes.c_int, [_vp, _i64, _vp, _vp, _d, _d, _vp]),
    ("rbfd_deform_f64", ctypes.c_int, [_vp, _i64, _vp, _vp, _d, _d, _vp]),
    ("rbfd_deform_noalloc", ctypes.c_int, [_vp, _i64, _vp, _vp, _d, _d, _vp]),
    ("rbfd_wall_distance", ctypes.c_int, [_vp, _i64, _vp, _vp]),
    ("rbfd_orthogonality", ctypes.c_int, [ctypes.c_int, _i64, _i64, _i64, ctypes.c_int, _vp, _vp, _vp, _vp, _vp,
                                          ctypes.POINTER(rbfd_quality), ctypes.c_int, _vp]),
    ("rbfd_wall_distance_f64", ctypes.c_int, [_vp, _i64, _vp, _vp]),
    ("rbfd_sort_pairs", ctypes.c_int, [_vp, _vp, _i64, ctypes.c_int, _vp]),
    ("rbfd_set_displacement", ctypes.c_int, [_vp, _vp]),
    ("rbfd_set_volume", ctypes.c_int, [_vp, _i64, _vp, _vp]),
    ("rbfd_deform_volume", ctypes.c_int, [_vp, _d, _d, _vp]),
    ("rbfd_greedy_batch", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int]),
    ("rbfd_deform_batch", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_i64),
                                         ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_d),
                                         ctypes.POINTER(_d), ctypes.POINTER(_vp)]),
    ("rbfd_deform_worklist", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_i64),
                                             ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_d),
                                             ctypes.POINTER(_d), ctypes.POINTER(_vp),
                                             ctypes.POINTER(rbfd_worklist_tune)]),
    ("rbfd_greedy_deform_batch", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_i64),
                                                ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_d),
                                                ctypes.POINTER(_d), ctypes.POINTER(_vp)]),
    ("rbfd_run_jobs", ctypes.c_int, [ctypes.POINTER(rbfd_job), ctypes.c_int, ctypes.POINTER(_vp)]),
    ("rbfd_destroy", ctypes.c_int, [_vp]),
    ("rbfd_server_options_default", None, [ctypes.POINTER(rbfd_server_options)]),
    ("rbfd_server_create", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(rbfd_server_options)]),
    ("rbfd_server_add_mesh", ctypes.c_int, [_vp, ctypes.c_int, _i64, _vp, _i64, _vp, _vp, ctypes.c_int, _vp, _d,
                                            _d, _d, ctypes.POINTER(ctypes.c_int)]),
    ("rbfd_submit", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(rbfd_request), ctypes.POINTER(ctypes.c_uint64)]),
    ("rbfd_poll", ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
    ("rbfd_wait", ctypes.c_int, [_vp, ctypes.c_uint64, _d, ctypes.POINTER(ctypes.c_int)]),
    ("rbfd_cancel", ctypes.c_int, [_vp, ctypes.c_uint64]),
    ("rbfd_request_times", ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(_d), ctypes.POINTER(_d),
                                          ctypes.POINTER(_d)]),
    ("rbfd_server_destroy", ctypes.c_int, [_vp]),
    ("rbfd_last_error", ctypes.c_char_p, []),
    ("rbfd_version", ctypes.c_char_p, []),
]

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library; raises on failure."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"rbfd CUDA library missing: {_build.LIB} (run paper_2107_13887_gb300.build)")
        lib = ctypes.CDLL(_build.LIB)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc):
    if rc != OK:
        msg = load().rbfd_last_error().decode(errors="replace")
        raise RbfdError(rc, msg)


def rbfd_last_error() -> str:
    return load().rbfd_last_error().decode(errors="replace")


def _ptr(a):
    """Data pointer of a numpy array or a torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _is_torch_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def default_options() -> rbfd_options:
    o = rbfd_options()
    load().rbfd_options_default(ctypes.byref(o))
    return o


def _create_args(xyz_s, dS, R, precision=MIXED, basis=2, first_point=0, nc_cap=0, stream=None,
                 eps_absolute=False, refine_iters=3, profile=False, engine=0, grid_ctas=0, prune=True):
    """rbfd_create's arrays (FP64, contiguous) and options."""
    on_dev = _is_torch_cuda(xyz_s)
    if on_dev:
        import torch

        xyz_s = xyz_s.to(torch.float64).contiguous()
        dS = dS.to(torch.float64).contiguous()
    else:
        xyz_s = np.ascontiguousarray(xyz_s, dtype=np.float64)
        dS = np.ascontiguousarray(dS, dtype=np.float64)
    Rv = np.ascontiguousarray(np.atleast_1d(R), dtype=np.float64)
    o = default_options()
    o.precision = int(precision)
    o.basis = int(basis)
    o.first_point = int(first_point)
    o.inputs_on_device = 1 if on_dev else 0
    o.nc_cap = int(nc_cap)
    o.stream = stream
    o.eps_absolute = 1 if eps_absolute else 0
    o.refine_iters = int(refine_iters)
    o.profile = 1 if profile else 0
    o.engine = int(engine)
    o.grid_ctas = int(grid_ctas)
    o.prune = 1 if prune else 0
    return xyz_s, dS, Rv, o


@dataclasses.dataclass
class LevelResult:
    idx: np.ndarray
    alpha: np.ndarray
    e_max: float
    R: float
    smax: float
    tau: float


class Mesh:
    """One surface set up for deformation: ``rbfd_create`` on construction,
    ``rbfd_destroy`` on ``close()`` / garbage collection."""

    def __init__(self, xyz_s, dS, R, eps, precision=MIXED, basis=2, first_point=0, nc_cap=0, stream=None,
                 eps_absolute=False, refine_iters=3, profile=False, engine=0, grid_ctas=0, prune=True):
        lib = load()
        self._lib = lib
        xyz_s, dS, Rv, o = _create_args(xyz_s, dS, R, precision=precision, basis=basis, first_point=first_point,
                                        nc_cap=nc_cap, stream=stream, eps_absolute=eps_absolute,
                                        refine_iters=refine_iters, profile=profile, engine=engine,
                                        grid_ctas=grid_ctas, prune=prune)
        self._keep = (xyz_s, dS)
        self.n_s, self.dim = (int(x) for x in xyz_s.shape)
        self.on_device = bool(o.inputs_on_device)
        h = ctypes.c_void_p()
        _check(lib.rbfd_create(ctypes.byref(h), self.dim, self.n_s, _ptr(xyz_s), _ptr(dS), len(Rv),
                               _ptr(Rv), float(eps), ctypes.byref(o)))
        self.h = h

    @classmethod
    def _wrap(cls, h, xyz_s, dS, on_device):
        """A Mesh for a handle made by the library (rbfd_run_jobs)."""
        m = cls.__new__(cls)
        m._lib = load()
        m._keep = (xyz_s, dS)
        m.n_s, m.dim = (int(x) for x in xyz_s.shape)
        m.on_device = bool(on_device)
        m.h = h
        return m

    def close(self):
        if getattr(self, "h", None):
            self._lib.rbfd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def greedy(self, allow_not_converged: bool = True) -> int:
        rc = self._lib.rbfd_greedy(self.h)
        if rc == ENOTCONV and allow_not_converged:
            return rc
        _check(rc)
        return rc

    def greedy_warm(self, allow_not_converged: bool = True) -> int:
        """``rbfd_greedy_warm``: the greedy for the current displacement,
        every level started from the previous run's controls and factor."""
        rc = self._lib.rbfd_greedy_warm(self.h)
        if rc == ENOTCONV and allow_not_converged:
            return rc
        _check(rc)
        return rc

    def greedy_split(self, rank: int, world: int, maxloc, allow_not_converged: bool = True) -> int:
        """``rbfd_greedy_split``: the greedy with the surface sweep split over
        ``world`` ranks; ``maxloc(key, idx) -> (key, idx)`` combines this rank's
        best candidate with the other ranks' (largest key, lowest index on
        ties), once per greedy step."""
        err = []

        def cb(_user, key_p, idx_p):
            try:
                k, i = maxloc(float(key_p[0]), int(idx_p[0]))
                key_p[0] = float(k)
                idx_p[0] = int(i)
                return 0
            except Exception as exc:  # reported as RBFD_ECOMM
                err.append(exc)
                return 1

        fn = MAXLOC_FN(cb)
        rc = self._lib.rbfd_greedy_split(self.h, int(rank), int(world), fn, None)
        if err and rc == ECOMM:
            raise RbfdError(ECOMM, f"maxloc callback raised {err[0]!r}") from err[0]
        if rc == ENOTCONV and allow_not_converged:
            return rc
        _check(rc)
        return rc

    def num_levels(self) -> int:
        n = ctypes.c_int()
        _check(self._lib.rbfd_num_levels(self.h, ctypes.byref(n)))
        return n.value

    def level(self, l: int) -> LevelResult:
        nc = ctypes.c_int64()
        e = ctypes.c_double()
        _check(self._lib.rbfd_get_level(self.h, l, ctypes.byref(nc), None, None, ctypes.byref(e)))
        idx = np.zeros(nc.value, dtype=np.int64)
        al = np.zeros((nc.value, self.dim))
        _check(self._lib.rbfd_get_level(self.h, l, ctypes.byref(nc), _ptr(idx), _ptr(al), ctypes.byref(e)))
        R, sm, tau = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self._lib.rbfd_level_info(self.h, l, ctypes.byref(R), ctypes.byref(sm), ctypes.byref(tau)))
        return LevelResult(idx, al, e.value, R.value, sm.value, tau.value)

    def levels(self):
        return [self.level(l) for l in range(self.num_levels())]

    def stats(self) -> dict:
        s = rbfd_stats()
        _check(self._lib.rbfd_get_stats(self.h, ctypes.byref(s)))
        out = {f: getattr(s, f) for f, _ in rbfd_stats._fields_}
        out["persist_phase_ms"] = list(s.persist_phase_ms)
        out["greedy_host_ms"] = list(s.greedy_host_ms)
        return out

    def deform(self, xyz_v, d_v, D: float, k: float, out=None):
        """Volume update (Eq. 19 / Eq. 23).  numpy in -> numpy out (host
        pointers); torch CUDA tensors in -> tensor out (device pointers).
        ``d_v=None``: the wall distances are computed on the device."""
        if self.on_device:
            import torch

            f64 = xyz_v.dtype == torch.float64
            n_v = xyz_v.shape[0]
            if out is None:
                out = torch.empty((n_v, self.dim), dtype=xyz_v.dtype, device=xyz_v.device)
        else:
            f64 = np.asarray(xyz_v).dtype == np.float64
            dt = np.float64 if f64 else np.float32
            xyz_v = np.ascontiguousarray(xyz_v, dtype=dt)
            if d_v is not None:
                d_v = np.ascontiguousarray(d_v, dtype=dt)
            n_v = xyz_v.shape[0]
            if out is None:
                out = np.empty((n_v, self.dim), dtype=dt)
        fn = self._lib.rbfd_deform_f64 if f64 else self._lib.rbfd_deform
        _check(fn(self.h, int(n_v), _ptr(xyz_v), _ptr(d_v), float(D), float(k), _ptr(out)))
        return out

    def set_displacement(self, dS):
        """``rbfd_set_displacement``: a new surface displacement on the same surface."""
        if self.on_device:
            import torch

            dS = dS.to(torch.float64).contiguous()
        else:
            dS = np.ascontiguousarray(dS, dtype=np.float64)
        self._keep_dS = dS
        _check(self._lib.rbfd_set_displacement(self.h, _ptr(dS)))

    def set_volume(self, xyz_v, d_v):
        """``rbfd_set_volume``: register a float32 volume mesh for repeated updates."""
        if not self.on_device:
            xyz_v = np.ascontiguousarray(xyz_v, dtype=np.float32)
            if d_v is not None:
                d_v = np.ascontiguousarray(d_v, dtype=np.float32)
        self.n_v_reg = int(xyz_v.shape[0])
        _check(self._lib.rbfd_set_volume(self.h, self.n_v_reg, _ptr(xyz_v), _ptr(d_v)))

    def deform_volume(self, D: float, k: float, out=None):
        """``rbfd_deform_volume`` on the registered volume."""
        if out is None:
            if self.on_device:
                import torch

                out = torch.empty((self.n_v_reg, self.dim), dtype=torch.float32, device="cuda")
            else:
                out = np.empty((self.n_v_reg, self.dim), dtype=np.float32)
        _check(self._lib.rbfd_deform_volume(self.h, float(D), float(k), _ptr(out)))
        return out

    def wall_distance(self, xyz_v, out=None):
        """``rbfd_wall_distance``: distance of each volume point from the
        nearest surface point, FP64.  float32 or float64 coordinates; numpy in
        -> numpy out, torch CUDA tensors in -> tensor out."""
        if self.on_device:
            import torch

            f64 = xyz_v.dtype == torch.float64
            n_v = xyz_v.shape[0]
            if out is None:
                out = torch.empty((n_v,), dtype=torch.float64, device=xyz_v.device)
        else:
            f64 = np.asarray(xyz_v).dtype == np.float64
            xyz_v = np.ascontiguousarray(xyz_v, dtype=np.float64 if f64 else np.float32)
            n_v = xyz_v.shape[0]
            if out is None:
                out = np.empty((n_v,), dtype=np.float64)
        fn = self._lib.rbfd_wall_distance_f64 if f64 else self._lib.rbfd_wall_distance
        _check(fn(self.h, int(n_v), _ptr(xyz_v), _ptr(out)))
        return out

    def deform_noalloc(self, xyz_v, d_v, D: float, k: float, out):
        """``rbfd_deform_noalloc``: float32 torch CUDA tensors in, result written
        into ``out`` (a preallocated float32 CUDA tensor); at most 131,072 points.
        The shapes, dtypes and layout are checked here, since the library sees
        only pointers: xyz_v and out [n_v, dim], d_v [n_v], all contiguous."""
        import torch

        n_v = int(xyz_v.shape[0]) if xyz_v.dim() == 2 else -1
        for name, t, shape in (("xyz_v", xyz_v, (n_v, self.dim)), ("d_v", d_v, (n_v,)),
                               ("out", out, (n_v, self.dim))):
            if t is None or not isinstance(t, torch.Tensor):
                raise RbfdError(EINVAL, f"rbfd_deform_noalloc: {name} must be a tensor")
            if t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shape:
                raise RbfdError(EINVAL, f"rbfd_deform_noalloc: {name} must be a contiguous float32 tensor of "
                                        f"shape {shape}, got {t.dtype} {tuple(t.shape)}")
        _check(self._lib.rbfd_deform_noalloc(self.h, n_v, _ptr(xyz_v), _ptr(d_v), float(D), float(k), _ptr(out)))
        return out


def orthogonality(wall, vol, n_layers, periodic_i=True, wall_disp=None, vol_disp=None, n_k=1, theta=True,
                  stream=None):
    """``rbfd_orthogonality``: orthogonality angle (degrees) of each cell of
    the structured grid grown off the surface, and a summary dict.  ``wall``
    [n_k * n_i][dim] (float64), ``vol`` [n_k * n_i * n_layers][dim] (float32),
    displacements optional; numpy arrays (host) or torch CUDA tensors (device)."""
    lib = load()
    on_dev = _is_torch_cuda(vol)
    if on_dev:
        import torch

        wall = wall.to(torch.float64).contiguous()
        vol = vol.to(torch.float32).contiguous()
        wall_disp = None if wall_disp is None else wall_disp.to(torch.float64).contiguous()
        vol_disp = None if vol_disp is None else vol_disp.to(torch.float32).contiguous()
    else:
        wall = np.ascontiguousarray(wall, dtype=np.float64)
        vol = np.ascontiguousarray(vol, dtype=np.float32)
        wall_disp = None if wall_disp is None else np.ascontiguousarray(wall_disp, dtype=np.float64)
        vol_disp = None if vol_disp is None else np.ascontiguousarray(vol_disp, dtype=np.float32)
    dim = int(wall.shape[1])
    n_i = int(wall.shape[0]) // (n_k if dim == 3 else 1)
    n_ci = n_i if periodic_i else n_i - 1
    cells = max(0, (n_k - 1 if dim == 3 else 1) * n_ci * int(n_layers))
    th = None
    if theta:
        if on_dev:
            th = torch.empty(cells, dtype=torch.float32, device=vol.device)
        else:
            th = np.empty(cells, dtype=np.float32)
    q = rbfd_quality()
    _check(lib.rbfd_orthogonality(dim, n_i, n_k if dim == 3 else 1, int(n_layers), 1 if periodic_i else 0,
                                  _ptr(wall), _ptr(wall_disp), _ptr(vol), _ptr(vol_disp), _ptr(th),
                                  ctypes.byref(q), 1 if on_dev else 0, stream))
    summ = {f: getattr(q, f) for f, _ in rbfd_quality._fields_}
    summ["hist"] = list(q.hist)
    return th, summ


def sort_pairs(keys, vals, key_bits=32, stream=None):
    """``rbfd_sort_pairs``: stable in-place sort of (key, value) pairs, int32 or
    uint32 torch CUDA tensors of one length, by the low ``key_bits`` bits of
    the key."""
    lib = load()
    if not (_is_torch_cuda(keys) and _is_torch_cuda(vals)) or keys.numel() != vals.numel():
        raise ValueError("sort_pairs: keys and vals must be CUDA tensors of one length")
    if keys.element_size() != 4 or vals.element_size() != 4 or not keys.is_contiguous() or not vals.is_contiguous():
        raise ValueError("sort_pairs: contiguous 32-bit tensors expected")
    _check(lib.rbfd_sort_pairs(_ptr(keys), _ptr(vals), int(keys.numel()), int(key_bits), stream))
    return keys, vals


def greedy_batch(meshes, allow_not_converged: bool = True) -> int:
    """``rbfd_greedy_batch``: the greedy selection of several meshes at once."""
    lib = load()
    arr = (_vp * len(meshes))(*[m.h.value for m in meshes])
    rc = lib.rbfd_greedy_batch(arr, len(meshes))
    if rc == ENOTCONV and allow_not_converged:
        return rc
    _check(rc)
    return rc


def deform_batch(meshes, xyz_v, d_v, D, k, out):
    """``rbfd_deform_batch``: float32 arrays (numpy for host meshes, torch CUDA
    tensors for device meshes), one per mesh; results written into ``out``."""
    lib = load()
    n = len(meshes)
    nv = (_i64 * n)(*[int(x.shape[0]) for x in xyz_v])
    px = (_vp * n)(*[_ptr(x).value for x in xyz_v])
    pd = (_vp * n)(*[None if x is None else _ptr(x).value for x in d_v])
    po = (_vp * n)(*[_ptr(x).value for x in out])
    Dv = (_d * n)(*[float(x) for x in D])
    kv = (_d * n)(*[float(x) for x in k])
    arr = (_vp * n)(*[m.h.value for m in meshes])
    _check(lib.rbfd_deform_batch(arr, n, nv, px, pd, Dv, kv, po))
    return out


def deform_worklist(meshes, xyz_v, d_v, D, k, out, autotune=True, ctas_per_sm=2, item_blocks=1, cell_div=None):
    """``rbfd_deform_worklist``: the volume updates of several meshes in one
    work-list launch; float32 arrays as in ``deform_batch`` (``d_v`` may be
    None, or hold None entries).  Returns the settings used as a dict
    (autotuned and cached per batch shape, or the ones given)."""
    lib = load()
    n = len(meshes)
    arr = (_vp * n)(*[m.h.value for m in meshes])
    nv = (_i64 * n)(*[int(x.shape[0]) for x in xyz_v])
    px = (_vp * n)(*[_ptr(x).value for x in xyz_v])
    pd = None if d_v is None else (_vp * n)(*[None if x is None else _ptr(x).value for x in d_v])
    Dv = (_d * n)(*[float(x) for x in D])
    kv = (_d * n)(*[float(x) for x in k])
    po = (_vp * n)(*[_ptr(x).value for x in out])
    t = rbfd_worklist_tune()
    t.autotune = 1 if autotune else 0
    t.ctas_per_sm = int(ctas_per_sm)
    t.item_blocks = int(item_blocks)
    for i in range(min(n, 16)):
        t.cell_div[i] = int(cell_div[i]) if cell_div is not None else 1
    _check(lib.rbfd_deform_worklist(arr, n, nv, px, pd, Dv, kv, po, ctypes.byref(t)))
    return {"autotune": bool(t.autotune), "ctas_per_sm": t.ctas_per_sm, "item_blocks": t.item_blocks,
            "cell_div": list(t.cell_div)[:n], "cached": bool(t.cached), "trials": t.trials,
            "launch_ms": t.launch_ms, "items": t.items}


def greedy_deform_batch(meshes, xyz_v, d_v, D, k, out, allow_not_converged: bool = True) -> int:
    """``rbfd_greedy_deform_batch``: greedy then volume update per mesh, the
    meshes side by side; float32 arrays as in ``deform_batch`` (``d_v`` may be
    None, or hold None entries, to compute wall distances)."""
    lib = load()
    n = len(meshes)
    arr = (_vp * n)(*[m.h.value for m in meshes])
    nv = (_i64 * n)(*[int(x.shape[0]) for x in xyz_v])
    px = (_vp * n)(*[_ptr(x).value for x in xyz_v])
    pd = None if d_v is None else (_vp * n)(*[None if x is None else _ptr(x).value for x in d_v])
    Dv = (_d * n)(*[float(x) for x in D])
    kv = (_d * n)(*[float(x) for x in k])
    po = (_vp * n)(*[_ptr(x).value for x in out])
    rc = lib.rbfd_greedy_deform_batch(arr, n, nv, px, pd, Dv, kv, po)
    if rc == ENOTCONV and allow_not_converged:
        return rc
    _check(rc)
    return rc


def run_jobs(jobs, allow_not_converged: bool = True):
    """``rbfd_run_jobs``: create, greedy and volume update for each job, the
    jobs side by side, in one library call.  Each job is a dict with the
    arguments of ``Mesh`` (xyz_s, dS, R, eps and options) and of
    ``Mesh.deform`` (xyz_v, d_v (may be None), D, k, out: float32 arrays of
    the same kind as xyz_s).  Returns (meshes, status): the ``Mesh`` objects
    (None where creation failed) for reading levels and statistics."""
    lib = load()
    n = len(jobs)
    arr = (rbfd_job * n)()
    keep = []
    for i, j in enumerate(jobs):
        opts = {key: j[key] for key in ("precision", "basis", "first_point", "nc_cap", "stream", "eps_absolute",
                                        "refine_iters", "profile", "engine", "grid_ctas", "prune") if key in j}
        xyz_s, dS, Rv, o = _create_args(j["xyz_s"], j["dS"], j["R"], **opts)
        keep.append((xyz_s, dS, Rv, o, j))
        a = arr[i]
        a.dim, a.n_levels, a.n_s = int(xyz_s.shape[1]), len(Rv), int(xyz_s.shape[0])
        a.xyz_s, a.dS, a.R = _ptr(xyz_s).value, _ptr(dS).value, _ptr(Rv).value
        a.eps = float(j["eps"])
        a.opt = ctypes.pointer(o)
        a.n_v = int(j["xyz_v"].shape[0])
        a.xyz_v = _ptr(j["xyz_v"]).value
        a.d_v = None if j.get("d_v") is None else _ptr(j["d_v"]).value
        a.D, a.k = float(j["D"]), float(j["k"])
        a.out = _ptr(j["out"]).value
    handles = (_vp * n)()
    rc = lib.rbfd_run_jobs(arr, n, handles)
    meshes = [Mesh._wrap(ctypes.c_void_p(handles[i]), xyz_s, dS, o.inputs_on_device) if handles[i] else None
              for i, (xyz_s, dS, Rv, o, j) in enumerate(keep)]
    if not (rc == ENOTCONV and allow_not_converged):
        if rc != 0:
            for m in meshes:
                if m is not None:
                    m.close()
        _check(rc)
    return meshes, rc


class Server:
    """The request loop of ``rbfd_server_*``: register meshes, submit
    displacements (host numpy arrays), poll / wait for the volume results."""

    def __init__(self, slots=4, precision=MIXED, mem_budget_bytes=0, max_queue=4096, fuse_volume=False):
        lib = load()
        self._lib = lib
        o = rbfd_server_options()
        lib.rbfd_server_options_default(ctypes.byref(o))
        o.slots = int(slots)
        o.precision = int(precision)
        o.mem_budget_bytes = int(mem_budget_bytes)
        o.max_queue = int(max_queue)
        o.fuse_volume = 1 if fuse_volume else 0
        h = ctypes.c_void_p()
        _check(lib.rbfd_server_create(ctypes.byref(h), ctypes.byref(o)))
        self.h = h
        self.meshes = {}
        self._live = {}

    def add_mesh(self, xyz_s, xyz_v, d_v, R, eps, D, k) -> int:
        xyz_s = np.ascontiguousarray(xyz_s, dtype=np.float64)
        xyz_v = np.ascontiguousarray(xyz_v, dtype=np.float32)
        if d_v is not None:  # None: wall distances computed on the device
            d_v = np.ascontiguousarray(d_v, dtype=np.float32)
        Rv = np.ascontiguousarray(np.atleast_1d(R), dtype=np.float64)
        mid = ctypes.c_int()
        _check(self._lib.rbfd_server_add_mesh(self.h, xyz_s.shape[1], xyz_s.shape[0], _ptr(xyz_s), xyz_v.shape[0],
                                              _ptr(xyz_v), _ptr(d_v), len(Rv), _ptr(Rv), float(eps), float(D),
                                              float(k), ctypes.byref(mid)))
        self.meshes[mid.value] = (xyz_s.shape[0], xyz_v.shape[0], xyz_s.shape[1])
        return mid.value

    def submit(self, mesh_id: int, dS, out=None):
        if mesh_id not in self.meshes:
            raise RbfdError(EINVAL, f"rbfd_submit: unknown mesh {mesh_id}")
        n_s, n_v, dim = self.meshes[mesh_id]
        dS = np.ascontiguousarray(dS, dtype=np.float64)
        if out is None:
            out = np.empty((n_v, dim), dtype=np.float32)
        req = rbfd_request(_ptr(dS).value, _ptr(out).value)
        t = ctypes.c_uint64()
        _check(self._lib.rbfd_submit(self.h, int(mesh_id), ctypes.byref(req), ctypes.byref(t)))
        self._live[t.value] = out  # the server writes it when the request completes
        return t.value

    def poll(self, ticket: int) -> int:
        st = ctypes.c_int()
        _check(self._lib.rbfd_poll(self.h, ticket, ctypes.byref(st)))
        return st.value

    def wait(self, ticket: int, timeout_s: float = 0.0):
        """Block until done; returns (status, result array)."""
        st = ctypes.c_int()
        rc = self._lib.rbfd_wait(self.h, ticket, float(timeout_s), ctypes.byref(st))
        if rc not in (OK, ENOTCONV):
            raise RbfdError(rc, rbfd_last_error())
        return rc, self._live.pop(ticket)

    def cancel(self, ticket: int):
        """``rbfd_cancel``: drop a queued request (its result array is never written)."""
        _check(self._lib.rbfd_cancel(self.h, ticket))
        self._live.pop(ticket, None)

    def times(self, ticket: int):
        q, r, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self._lib.rbfd_request_times(self.h, ticket, ctypes.byref(q), ctypes.byref(r), ctypes.byref(t)))
        return q.value, r.value, t.value

    def close(self):
        if getattr(self, "h", None):
            self._lib.rbfd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
