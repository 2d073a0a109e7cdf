"""ctypes binding of libamrmg (include/amrmg.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; importing this
module raises if ``libamrmg.so`` has not been built, and nothing here falls
back to a CPU path.  Particle and output arrays are contiguous float64 CUDA
tensors (torch is used for device memory and streams only).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libamrmg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; g.build()'` "
                      "(the CUDA library is required; there is no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

AMR_OK, AMR_EINVAL, AMR_ENOMEM, AMR_ENOCONV, AMR_ECUDA, AMR_ETIMEOUT, AMR_ENESTING, AMR_EOUTSIDE = range(8)
STATUS = {0: "AMR_OK", 1: "AMR_EINVAL", 2: "AMR_ENOMEM", 3: "AMR_ENOCONV", 4: "AMR_ECUDA", 5: "AMR_ETIMEOUT",
          6: "AMR_ENESTING", 7: "AMR_EOUTSIDE"}
TAG = {"rel": 0, "abs": 1, "boxes": 2, "phi": 3, "efield": 4}
PRECISION = {"fp64": 0, "mixed": 1}
FIELD = {"rho": 0, "phi": 1, "res": 2, "ex": 3, "ey": 4, "ez": 5}
NORM = {"inf": 0, 0: 0, 1: 1, 2: 2}
MAX_LEVELS = 6


class AmrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Desc(ctypes.Structure):
    _fields_ = [("n0", ctypes.c_int), ("max_level", ctypes.c_int), ("brick", ctypes.c_int),
                ("tag_mode", ctypes.c_int), ("tag_lambda", ctypes.c_double), ("buffer_cells", ctypes.c_int),
                ("n_boxes", ctypes.c_int), ("boxes_host", ctypes.POINTER(ctypes.c_int)),
                ("precision", ctypes.c_int), ("eps0", ctypes.c_double), ("bc", ctypes.c_int),
                ("robin_d", ctypes.c_double), ("max_device_bytes", ctypes.c_int64)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("norm", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("bottom_cycles", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("use_graph", ctypes.c_int), ("persistent", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("n0", ctypes.c_int), ("max_level", ctypes.c_int), ("precision", ctypes.c_int),
                ("n_particles", ctypes.c_int64), ("sigma", ctypes.c_double), ("centre", ctypes.c_double * 3),
                ("seed", ctypes.c_uint64), ("arrival_s", ctypes.c_double),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p), ("q", ctypes.c_void_p),
                ("field_out", ctypes.c_void_p)]


class RequestResult(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("status", ctypes.c_int), ("iters", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("retried", ctypes.c_int), ("rel_res_max", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("checksum", ctypes.c_double * 4)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int), ("realtime", ctypes.c_int),
                ("admit_fraction", ctypes.c_double)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("rel_res", ctypes.c_double * MAX_LEVELS), ("ms_total", ctypes.c_double)]


_P = ctypes.c_void_p
_D = ctypes.c_void_p  # device or host double pointer
_I64 = ctypes.c_int64
_SIGS = {
    "amr_desc_default": ([ctypes.POINTER(Desc)], ctypes.c_int),
    "amr_solve_opts_default": ([ctypes.POINTER(SolveOpts)], ctypes.c_int),
    "amr_create_hierarchy": ([ctypes.POINTER(Desc), _D, _D, _D, _D, _I64, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "amr_destroy": ([_P], None),
    "amr_deposit": ([_P, _D, _D, _D, _D, _I64], ctypes.c_int),
    "amr_solve": ([_P, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats)], ctypes.c_int),
    "amr_gather": ([_P, _D, _D, _D, _I64, _D, _D, _D, _D], ctypes.c_int),
    "amr_step": ([_P, _D, _D, _D, _D, _I64, ctypes.POINTER(SolveOpts), _D, _D, _D, ctypes.POINTER(SolveStats)],
                 ctypes.c_int),
    "amr_residual": ([_P, ctypes.c_int, _D], ctypes.c_int),
    "amr_field_from_phi": ([_P], ctypes.c_int),
    "amr_num_levels": ([_P, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "amr_level_box": ([_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(_I64)], ctypes.c_int),
    "amr_get_level": ([_P, ctypes.c_int, ctypes.c_int, _D], ctypes.c_int),
    "amr_set_level": ([_P, ctypes.c_int, ctypes.c_int, _D], ctypes.c_int),
    "amr_get_mask": ([_P, ctypes.c_int, _D], ctypes.c_int),
    "amr_ghost_stats": ([_P, ctypes.POINTER(_I64)], ctypes.c_int),
    "amr_hierarchy_bytes": ([ctypes.POINTER(Desc), ctypes.c_double, ctypes.POINTER(_I64)], ctypes.c_int),
    "amr_device_bytes": ([_P, ctypes.POINTER(_I64)], ctypes.c_int),
    "amr_kernel_launches": ([_P, ctypes.POINTER(_I64)], ctypes.c_int),
    "amr_bottom_solver": ([_P, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "amr_bin": ([_P, _P, _P, _P, _I64, _P, _P, ctypes.POINTER(_I64)], ctypes.c_int),
    "amr_profile": ([_P, ctypes.c_int], ctypes.c_int),
    "amr_profile_num_kinds": ([], ctypes.c_int),
    "amr_profile_kind_name": ([ctypes.c_int], ctypes.c_char_p),
    "amr_profile_read": ([_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64),
                          ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "amr_profile_read_flops": ([_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "amr_profile_read_ops": ([_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "amr_batch_create": ([ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(SolveOpts), ctypes.POINTER(_P)],
                         ctypes.c_int),
    "amr_batch_solve": ([_P, ctypes.POINTER(SolveStats)], ctypes.c_int),
    "amr_batch_destroy": ([_P], None),
    "amr_selftest_barrier_timeout": ([_P, ctypes.c_int], ctypes.c_int),
    "amr_serve": ([ctypes.POINTER(ServeConfig), ctypes.POINTER(Request), ctypes.c_int, ctypes.POINTER(SolveOpts),
                   ctypes.POINTER(RequestResult)], ctypes.c_int),
    "amr_request_bytes": ([ctypes.POINTER(Request), ctypes.POINTER(_I64)], ctypes.c_int),
    "amr_masked_norms_noalloc": ([_D, _D, _I64, ctypes.c_int, _D, _P], ctypes.c_int),
    "amr_regrid_boxes": ([_P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                          ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "amr_transfer_phi": ([_P, _P], ctypes.c_int),
    "amr_set_gather_buffer": ([_P, ctypes.c_int], ctypes.c_int),
    "amr_solve_many": ([ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(SolveOpts), ctypes.c_int,
                        ctypes.POINTER(SolveStats)], ctypes.c_int),
    "amr_domain_transform": ([_D, _D, _D, _I64, ctypes.POINTER(ctypes.c_double), ctypes.c_double, _D, _D, _D,
                              ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "amr_rescale_fields": ([_P, ctypes.c_double], ctypes.c_int),
    "amr_push": ([_D, _D, _D, _D, _D, _D, _D, _D, _D, _I64, ctypes.c_double, ctypes.c_double, _P], ctypes.c_int),
    "amr_moments": ([_D, _D, _D, _I64, ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "amr_probe_fp64_fma": ([_I64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _P],
                           ctypes.c_int),
    "amr_last_error": ([], ctypes.c_char_p),
}
for _name, (_args, _ret) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _ret


def last_error() -> str:
    return _lib.amr_last_error().decode()


def _check(rc, allow=()):
    if rc != AMR_OK and rc not in allow:
        raise AmrError(rc, last_error())
    return rc


def _dev(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def make_desc(n0, max_level, *, boxes=None, tag_mode="rel", tag_lambda=0.1, buffer_cells=1, brick=8,
              precision="fp64", eps0=1.0, robin_d=None, periodic=False, max_device_bytes=0):
    """robin_d: None for homogeneous Dirichlet faces, else the distance d of
    the Robin faces d phi/dn + phi/d = 0 (Eq. robin_bc); periodic=True for
    periodic faces; max_device_bytes > 0 caps the hierarchy's device bytes
    (creation fails with AMR_ENOMEM instead)."""
    d = Desc()
    _lib.amr_desc_default(ctypes.byref(d))
    d.max_device_bytes = int(max_device_bytes)
    d.n0, d.max_level, d.brick = int(n0), int(max_level), int(brick)
    d.tag_mode = TAG["boxes" if boxes is not None else tag_mode]
    d.tag_lambda, d.buffer_cells = float(tag_lambda), int(buffer_cells)
    d.precision, d.eps0 = PRECISION[precision], float(eps0)
    if robin_d is not None:
        d.bc, d.robin_d = 1, float(robin_d)
    if periodic:
        d.bc = 2
    flat = []
    for lev, lo, hi in boxes or []:
        flat += [int(lev), *map(int, lo), *map(int, hi)]
    arr = (ctypes.c_int * max(len(flat), 1))(*flat)
    d.n_boxes = len(flat) // 7
    d.boxes_host = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int))
    return d, arr


def solve_opts(eps=1e-10, norm=2, max_iter=100, nu_pre=2, nu_post=2, bottom_cycles=2, warm_start=False,
               use_graph=True, persistent=False):
    o = SolveOpts()
    _lib.amr_solve_opts_default(ctypes.byref(o))
    o.eps, o.norm, o.max_iter = float(eps), NORM[norm], int(max_iter)
    o.nu_pre, o.nu_post, o.bottom_cycles, o.warm_start = int(nu_pre), int(nu_post), int(bottom_cycles), int(warm_start)
    o.use_graph = int(bool(use_graph))
    o.persistent = int(bool(persistent))
    return o


def hierarchy_bytes(n0, max_level, fill=0.05, **kw):
    d, _keep = make_desc(n0, max_level, **kw)
    out = _I64()
    _check(_lib.amr_hierarchy_bytes(ctypes.byref(d), float(fill), ctypes.byref(out)))
    return int(out.value)


class Hierarchy:
    """An AMR hierarchy owned by libamrmg, bound to a CUDA stream."""

    def __init__(self, n0, max_level, *, particles=None, boxes=None, tag_mode="rel", tag_lambda=0.1,
                 buffer_cells=1, brick=8, precision="fp64", eps0=1.0, robin_d=None, periodic=False,
                 stream=None, max_device_bytes=0):
        import torch
        d, keep = make_desc(n0, max_level, boxes=boxes, tag_mode=tag_mode, tag_lambda=tag_lambda,
                            buffer_cells=buffer_cells, brick=brick, precision=precision, eps0=eps0,
                            robin_d=robin_d, periodic=periodic, max_device_bytes=max_device_bytes)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        if particles is not None:
            x, y, z, q = particles
            ptrs = [_dev(t, n) for t, n in zip((x, y, z, q), "xyzq")]
            n = x.numel()
        else:
            ptrs = [None] * 4
            n = 0
        h = _P()
        _check(_lib.amr_create_hierarchy(ctypes.byref(d), *ptrs, n, ctypes.c_void_p(stream.cuda_stream),
                                         ctypes.byref(h)))
        self._h = h
        self.n0 = int(n0)

    def close(self):
        if getattr(self, "_h", None):
            _lib.amr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nlevels(self):
        n = ctypes.c_int()
        _check(_lib.amr_num_levels(self._h, ctypes.byref(n)))
        return n.value

    def level_box(self, level):
        lo, hi, nv = (ctypes.c_int * 3)(), (ctypes.c_int * 3)(), _I64()
        _check(_lib.amr_level_box(self._h, level, lo, hi, ctypes.byref(nv)))
        return np.array(lo[:]), np.array(hi[:]), int(nv.value)

    def shape(self, level):
        lo, hi, _ = self.level_box(level)
        e = hi - lo + 1
        return int(e[2]), int(e[1]), int(e[0])

    def h(self, level):
        return 1.0 / (self.n0 * 2 ** level)

    def regrid_boxes(self, policy, tag_lambda, max_level, buffer_cells=1):
        """Boxes (level, lo, hi) of a regridded hierarchy from this one's
        current fields (Sec. 4.2 policies 'rel', 'abs', 'phi', 'efield')."""
        n = ctypes.c_int(0)
        rc = _lib.amr_regrid_boxes(self._h, TAG[policy], float(tag_lambda), int(buffer_cells), int(max_level),
                                   None, 0, ctypes.byref(n))
        if rc == AMR_OK:
            return []
        if rc != AMR_EINVAL or n.value == 0:
            _check(rc)
        cap = max(n.value, 1)
        arr = (ctypes.c_int * (7 * cap))()
        _check(_lib.amr_regrid_boxes(self._h, TAG[policy], float(tag_lambda), int(buffer_cells), int(max_level),
                                     arr, cap, ctypes.byref(n)))
        return [(arr[7 * b], tuple(arr[7 * b + 1:7 * b + 4]), tuple(arr[7 * b + 4:7 * b + 7]))
                for b in range(n.value)]

    def rescale_fields(self, S):
        """phi /= S and E /= S^2 on every level (back to particle space)."""
        _check(_lib.amr_rescale_fields(self._h, float(S)))

    def set_gather_buffer(self, buffer_cells):
        """Gather from a refined level only buffer_cells inside it."""
        _check(_lib.amr_set_gather_buffer(self._h, int(buffer_cells)))

    def transfer_phi_from(self, src):
        """Warm start: phi of every level from src where it holds the cell,
        else from the parent on this hierarchy's coarser level."""
        _check(_lib.amr_transfer_phi(src._h, self._h))

    def deposit(self, x, y, z, q):
        _check(_lib.amr_deposit(self._h, _dev(x, "x"), _dev(y, "y"), _dev(z, "z"), _dev(q, "q"), x.numel()))

    def solve(self, raise_on_noconv=False, **kw):
        o = solve_opts(**kw)
        st = SolveStats()
        rc = _lib.amr_solve(self._h, ctypes.byref(o), ctypes.byref(st))
        _check(rc, allow=() if raise_on_noconv else (AMR_ENOCONV,))
        return {"iters": st.iters, "status": STATUS[st.status], "rel_res": np.array(st.rel_res[:st.n_levels]),
                "ms_total": st.ms_total}

    def gather(self, x, y, z, with_phi=False):
        import torch
        n = x.numel()
        ex, ey, ez = (torch.empty(n, dtype=torch.float64, device=x.device) for _ in range(3))
        ph = torch.empty(n, dtype=torch.float64, device=x.device) if with_phi else None
        _check(_lib.amr_gather(self._h, _dev(x, "x"), _dev(y, "y"), _dev(z, "z"), n, _dev(ex, "ex"), _dev(ey, "ey"),
                               _dev(ez, "ez"), _dev(ph, "phi") if with_phi else None))
        return (ex, ey, ez, ph) if with_phi else (ex, ey, ez)

    def step_host(self, x, y, z, q, out=None, **kw):
        """deposit + solve + gather through host arrays (float64, ideally
        pinned); returns (ex, ey, ez, stats)."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, q)]
        n = len(arrs[0])
        if out is None:
            out = tuple(np.empty(n) for _ in range(3))
        o = solve_opts(**kw)
        st = SolveStats()
        rc = _lib.amr_step(self._h, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs], n, ctypes.byref(o),
                           *[a.ctypes.data_as(ctypes.c_void_p) for a in out], ctypes.byref(st))
        _check(rc, allow=(AMR_ENOCONV,))
        return out[0], out[1], out[2], {"iters": st.iters, "rel_res": np.array(st.rel_res[:st.n_levels])}

    def step_ptrs(self, xp, yp, zp, qp, n, exp, eyp, ezp, opts):
        """Host-pointer step without numpy conversions (benchmark loop)."""
        st = SolveStats()
        rc = _lib.amr_step(self._h, xp, yp, zp, qp, n, ctypes.byref(opts), exp, eyp, ezp, ctypes.byref(st))
        _check(rc, allow=(AMR_ENOCONV,))
        return st

    def residual(self, norm=2):
        out = (ctypes.c_double * MAX_LEVELS)()
        _check(_lib.amr_residual(self._h, NORM[norm], ctypes.cast(out, ctypes.c_void_p)))
        return np.array(out[:self.nlevels])

    def field_from_phi(self):
        _check(_lib.amr_field_from_phi(self._h))

    def get(self, level, field):
        out = np.zeros(self.shape(level))
        _check(_lib.amr_get_level(self._h, level, FIELD[field], out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set(self, level, field, arr):
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(arr, dtype=np.float64), self.shape(level)))
        _check(_lib.amr_set_level(self._h, level, FIELD[field], a.ctypes.data_as(ctypes.c_void_p)))

    def mask(self, level):
        out = np.zeros(self.shape(level), np.int8)
        _check(_lib.amr_get_mask(self._h, level, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def ghost_stats(self):
        out = (_I64 * 3)()
        _check(_lib.amr_ghost_stats(self._h, out))
        return {"quadratic": out[0], "linear": out[1], "constant": out[2]}

    def device_bytes(self):
        out = _I64()
        _check(_lib.amr_device_bytes(self._h, ctypes.byref(out)))
        return int(out.value)

    def profile(self, enable=True, mode="eager"):
        """Per-launch timers: mode "eager" runs solves host-driven with an
        event pair around every launch; mode "graph" runs each solve as the
        captured graph unrolled to the last solve's V-cycle count, with
        event-record nodes around every kernel node."""
        m = 0 if not enable else (2 if mode == "graph" else 1)
        _check(_lib.amr_profile(self._h, m))

    def profile_read(self):
        """{kind: (ms_total, launches, algorithmic_bytes, algorithmic_flops)} of the timed launches."""
        out = {}
        for k in range(_lib.amr_profile_num_kinds()):
            ms, n, b, f = ctypes.c_double(), _I64(), ctypes.c_double(), ctypes.c_double()
            _check(_lib.amr_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)))
            _check(_lib.amr_profile_read_flops(self._h, k, ctypes.byref(f)))
            if n.value:
                out[_lib.amr_profile_kind_name(k).decode()] = (ms.value, int(n.value), b.value, f.value)
        return out

    def profile_read_ops(self):
        """{kind: algorithmic arithmetic instructions (an FMA counts 1)} of the
        timed launches, for the kinds with a flop count."""
        out = {}
        for k in range(_lib.amr_profile_num_kinds()):
            o = ctypes.c_double()
            _check(_lib.amr_profile_read_ops(self._h, k, ctypes.byref(o)))
            if o.value:
                out[_lib.amr_profile_kind_name(k).decode()] = o.value
        return out

    def selftest_barrier_timeout(self, limit_ms=50):
        """Runs the solve program with a barrier that cannot complete;
        returns the status code (AMR_ETIMEOUT when the bounded wait works)."""
        return int(_lib.amr_selftest_barrier_timeout(self._h, int(limit_ms)))

    def bin(self, x, y, z):
        """(keys, perm, nkeys): keys as int32 device tensor holding the uint32
        bit patterns (0xFFFFFFFF = no key), perm int64 sorted by key."""
        import torch
        n = x.numel()
        keys = torch.empty(max(n, 1), dtype=torch.int32, device=x.device)
        perm = torch.empty(max(n, 1), dtype=torch.int64, device=x.device)
        nk = _I64()
        _check(_lib.amr_bin(self._h, _dev(x, "x"), _dev(y, "y"), _dev(z, "z"), n, ctypes.c_void_p(keys.data_ptr()),
                            ctypes.c_void_p(perm.data_ptr()), ctypes.byref(nk)))
        return keys[:n], perm[:n], int(nk.value)

    def bottom_solver(self):
        """'exact' (sine transforms + tridiagonal solves) or 'gmg'."""
        out = ctypes.c_int()
        _check(_lib.amr_bottom_solver(self._h, ctypes.byref(out)))
        return "exact" if out.value == 1 else "gmg"

    def kernel_launches(self):
        out = _I64()
        _check(_lib.amr_kernel_launches(self._h, ctypes.byref(out)))
        return int(out.value)


class Batch:
    """Many hierarchies solved by one graph launch per solve (the form is
    picked at creation by AMR_BATCH: "graphs" (default) independent graph
    branches, "clusters" a persistent cluster program, "rounds" a
    cooperative program of lock-step rounds; all give each hierarchy its solo
    result, bit for bit)."""

    def __init__(self, hierarchies, mode=None, **opts):
        import os
        self.hs = list(hierarchies)
        if mode is not None:
            prev = os.environ.get("AMR_BATCH")
            os.environ["AMR_BATCH"] = mode
            try:
                self._create(opts)
            finally:
                if prev is None:
                    os.environ.pop("AMR_BATCH", None)
                else:
                    os.environ["AMR_BATCH"] = prev
        else:
            self._create(opts)

    def _create(self, opts):
        arr = (_P * len(self.hs))(*[h._h for h in self.hs])
        o = solve_opts(**opts)
        b = _P()
        _check(_lib.amr_batch_create(arr, len(self.hs), ctypes.byref(o), ctypes.byref(b)))
        self._b = b

    def solve(self):
        st = (SolveStats * len(self.hs))()
        rc = _lib.amr_batch_solve(self._b, st)
        _check(rc, allow=(AMR_ENOCONV,))
        return [{"iters": s.iters, "status": STATUS[s.status], "rel_res": np.array(s.rel_res[:s.n_levels]),
                 "ms_total": s.ms_total} for s in st]

    def close(self):
        if getattr(self, "_b", None):
            _lib.amr_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_request(n0, max_level, n_particles, sigma, seed, arrival_s=0.0, precision="fp64",
                 centre=(0.5, 0.5, 0.5), particles=None, field_out=None):
    """One request of the served form.  particles: optional (x, y, z, q)
    CUDA float64 tensors solved instead of the seeded bunch; field_out:
    optional CUDA float64 tensor of 4 n_particles values that receives the
    gathered Ex, Ey, Ez and phi.  Both must outlive the serve call."""
    r = Request()
    r.n0, r.max_level, r.precision = int(n0), int(max_level), PRECISION[precision]
    r.n_particles, r.sigma = int(n_particles), float(sigma)
    for d in range(3):
        r.centre[d] = float(centre[d])
    r.seed, r.arrival_s = int(seed) & ((1 << 64) - 1), float(arrival_s)
    if particles is not None:
        for name, t in zip("xyzq", particles):
            setattr(r, name, _dev(t, name).value)
    if field_out is not None:
        if field_out.numel() < 4 * int(n_particles):
            raise ValueError("field_out needs 4 n_particles values")
        r.field_out = _dev(field_out, "field_out").value
    return r


def request_bytes(r):
    out = _I64()
    _check(_lib.amr_request_bytes(ctypes.byref(r), ctypes.byref(out)))
    return int(out.value)


def serve(requests, budget_bytes, max_slots, realtime=True, admit_fraction=1.0, **opts):
    """Run the continuous-batching request loop; one dict per request."""
    n = len(requests)
    arr = (Request * n)(*requests)
    res = (RequestResult * n)()
    cfg = ServeConfig()
    cfg.budget_bytes, cfg.max_slots, cfg.realtime = int(budget_bytes), int(max_slots), int(bool(realtime))
    cfg.admit_fraction = float(admit_fraction)
    o = solve_opts(**opts)
    _check(_lib.amr_serve(ctypes.byref(cfg), arr, n, ctypes.byref(o), res))
    return [{"arrival_s": r.arrival_s, "admit_s": r.admit_s, "done_s": r.done_s, "status": r.status,
             "iters": r.iters, "n_levels": r.n_levels, "retried": bool(r.retried), "rel_res_max": r.rel_res_max,
             "device_bytes": r.device_bytes, "checksum": np.array(r.checksum[:])} for r in res]


def domain_transform(x, y, z, centre=(0.0, 0.0, 0.0), delta=0.2, out=None, stream=None):
    """Map particle-space positions into the unit cube (Sec. 4.1): returns
    (u, v, w, S) with u = 1/2 + (x - centre) / S."""
    import torch
    n = x.numel()
    u, v, w = out if out is not None else (torch.empty_like(x), torch.empty_like(y), torch.empty_like(z))
    c = (ctypes.c_double * 3)(*map(float, centre))
    S = ctypes.c_double(0.0)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(_lib.amr_domain_transform(_dev(x, "x"), _dev(y, "y"), _dev(z, "z"), n, c, float(delta), _dev(u, "u"),
                                     _dev(v, "v"), _dev(w, "w"), ctypes.byref(S), ctypes.c_void_p(st.cuda_stream)))
    return u, v, w, S.value


def push(pos, mom, field, q_over_m, dt, stream=None):
    """Kick-drift push in place: mom += (q/m) dt E; pos += dt mom."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    n = pos[0].numel()
    _check(_lib.amr_push(*[_dev(t, "pos") for t in pos], *[_dev(t, "mom") for t in mom],
                         *[_dev(t, "E") for t in field], n, float(q_over_m), float(dt), ctypes.c_void_p(st.cuda_stream)))


def moments(x, y, z, stream=None):
    """Centroid, rms size and beam-profile parameter per axis (Eqs. rms_sigma,
    halo): dict of three 3-arrays."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    out = (ctypes.c_double * 9)()
    _check(_lib.amr_moments(_dev(x, "x"), _dev(y, "y"), _dev(z, "z"), x.numel(), out,
                            ctypes.c_void_p(st.cuda_stream)))
    return {"centroid": np.array(out[0:3]), "sigma": np.array(out[3:6]), "xi": np.array(out[6:9])}


def solve_many(hierarchies, n_streams=16, **opts):
    """Solve independent hierarchies side by side (their captured graphs on
    n_streams streams); one stats dict per hierarchy."""
    hs = list(hierarchies)
    arr = (_P * len(hs))(*[h._h for h in hs])
    o = solve_opts(**opts)
    st = (SolveStats * len(hs))()
    _check(_lib.amr_solve_many(arr, len(hs), ctypes.byref(o), int(n_streams), st), allow=(AMR_ENOCONV,))
    return [{"iters": s.iters, "status": STATUS[s.status], "rel_res": np.array(s.rel_res[:s.n_levels]),
             "ms_total": s.ms_total} for s in st]


def probe_fp64_fma(iters=16384, stream=None):
    """The device's FP64 FMA rate (amr_probe_fp64_fma): (GFMA/s, ms of the
    timed launch)."""
    import torch
    g, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(_lib.amr_probe_fp64_fma(int(iters), ctypes.byref(g), ctypes.byref(ms), ctypes.c_void_p(st.cuda_stream)))
    return float(g.value), float(ms.value)
