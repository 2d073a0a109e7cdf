"""Plain FP64 CPU oracle of the AMR multigrid Poisson solve (arXiv 1812.03689).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path: the C source ``amr_oracle.c`` builds its own hierarchy,
assembles the paper's per-level matrices explicitly (Sec. 5.3) and runs
Alg. 1-3 literally.  This module is argument marshalling over ctypes plus the
numpy view of the dense per-level layout.

Dense layout of a level (shared convention with the C-ABI, written
independently on each side): the valid cells' bounding box ``[lo, hi]``
(inclusive, level index space, level spacing ``h_l = 1 / (n0 * 2**l)``), as a
numpy array of shape ``(nz, ny, nx)`` indexed ``[k, j, i]``; cells outside the
level read as 0.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "amr_oracle.c")

FIELDS = {"rho": 0, "phi": 1, "res": 2, "ex": 3, "ey": 4, "ez": 5, "err": 6}
MATRICES = {"A_nf": 0, "A_comp": 1, "B_crse": 2, "B_fine": 3, "R": 4, "I": 5,
            "G_x": 6, "G_y": 7, "G_z": 8, "Gc_x": 9, "Gc_y": 10, "Gc_z": 11}
TAG_MODES = {"rel": 0, "abs": 1, "boxes": 2, "phi": 3, "efield": 4}
NORMS = {1: 1, 2: 2, "inf": 0, 0: 0}


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no FMA contraction, so both hosts
    round alike), with OpenMP when the compiler has it (the parallel loops
    give the serial loops' results; see the C source)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB_PATH, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
    return _LIB_PATH


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def set_threads(n: int | None = None) -> int:
    """Threads of the oracle's parallel loops (default: every core this
    process may run on); returns the number in use (1 without OpenMP)."""
    return int(_load().orc_set_threads(int(n if n else host_cores())))


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_int, ip, dp, dp, dp, dp, ctypes.c_long, ctypes.c_double]
        lib.orc_create_bc.restype = P
        lib.orc_create_bc.argtypes = lib.orc_create.argtypes + [ctypes.c_double]
        lib.orc_regrid.restype = P
        lib.orc_regrid.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp,
                                   ctypes.c_long]
        lib.orc_set_gather_buffer.argtypes = [P, ctypes.c_int]
        lib.orc_last_error.restype = ctypes.c_char_p
        lib.orc_destroy.argtypes = [P]
        lib.orc_bin.argtypes = [P, dp, dp, dp, ctypes.c_long, ctypes.POINTER(ctypes.c_uint),
                                ctypes.POINTER(ctypes.c_long)]
        lib.orc_bin.restype = ctypes.c_long
        lib.orc_nlevels.argtypes = [P]
        lib.orc_level_box.argtypes = [P, ctypes.c_int, ip, ip, ip]
        lib.orc_get_field.argtypes = [P, ctypes.c_int, ctypes.c_int, dp]
        lib.orc_set_field.argtypes = [P, ctypes.c_int, ctypes.c_int, dp]
        lib.orc_get_mask.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int8)]
        lib.orc_deposit.argtypes = [P, dp, dp, dp, dp, ctypes.c_long]
        lib.orc_solve.argtypes = [P, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_int, dp]
        lib.orc_solve.restype = ctypes.c_int
        lib.orc_residual.argtypes = [P, ctypes.c_int, dp]
        lib.orc_average_down.argtypes = [P]
        lib.orc_efield.argtypes = [P]
        lib.orc_gather.argtypes = [P, dp, dp, dp, ctypes.c_long, dp, dp, dp, dp]
        lib.orc_matrix.argtypes = [P, ctypes.c_int, ctypes.c_int, ip, ip, ip, ip, ip, dp]
        lib.orc_cells.argtypes = [P, ctypes.c_int, ip]
        lib.orc_ghost_stats.argtypes = [P, ctypes.POINTER(ctypes.c_long)]
        lib.orc_quad_pattern.restype = ctypes.c_ulong
        lib.orc_quad_pattern.argtypes = [ctypes.c_int]
        lib.orc_lin_pattern.restype = ctypes.c_ulong
        lib.orc_lin_pattern.argtypes = [ctypes.c_int]
        lib.orc_ghost_stencil.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ip, dp, ip]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = ctypes.c_int
        _lib = lib
        lib.orc_set_threads(host_cores())
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def quad_pattern(case: int) -> int:
    return int(_load().orc_quad_pattern(case))


def lin_pattern(case: int) -> int:
    return int(_load().orc_lin_pattern(case))


class OracleHierarchy:
    """One AMR hierarchy on the unit cube, owned by the C oracle.

    ``boxes``: list of ``(level, lo3, hi3)`` (inclusive, level index space)
    for ``tag_mode='boxes'``; otherwise levels are made by tagging the
    deposited charge density (``'rel'``: rho > lambda * max rho, ``'abs'``:
    |rho| >= lambda, Eq. tag_charge) with ``brick``-cell fine bricks.
    ``robin_d``: 0 for homogeneous Dirichlet faces, else the artificial
    distance d > 0 of the Robin faces d phi/dn + phi/d = 0 (Eq. robin_bc);
    ``periodic=True`` makes the faces periodic instead.
    """

    def __init__(self, n0, lmax, *, particles=None, boxes=None, tag_mode="rel", tag_lambda=0.1,
                 buffer=1, brick=8, eps0=1.0, robin_d=0.0, periodic=False):
        lib = _load()
        if boxes is not None:
            tag_mode = "boxes"
        flat = []
        for b in boxes or []:
            lev, lo, hi = b
            flat += [int(lev), *map(int, lo), *map(int, hi)]
        barr = np.ascontiguousarray(np.array(flat if flat else [0], dtype=np.int32))
        if particles is None:
            x = y = z = q = np.zeros(1)
            npart = 0
        else:
            x, y, z, q = (np.ascontiguousarray(a, dtype=np.float64) for a in particles)
            npart = len(x)
        self._keep = (x, y, z, q, barr)
        h = lib.orc_create_bc(int(n0), int(lmax), int(brick), TAG_MODES[tag_mode], float(tag_lambda),
                              int(buffer), len(flat) // 7, _iptr(barr), _dptr(x), _dptr(y), _dptr(z), _dptr(q),
                              npart, float(eps0), -1.0 if periodic else float(robin_d))
        if not h:
            raise ValueError("oracle: " + lib.orc_last_error().decode())
        self._h = ctypes.c_void_p(h)
        self.n0 = int(n0)
        self.robin_d = float(robin_d)

    def regrid(self, policy, tag_lambda, lmax, *, particles=None, buffer=1):
        """New hierarchy (Sec. 4.2): level l+1 from the blocks that ``policy``
        ('rel', 'abs', 'phi' or 'efield') tags on THIS hierarchy's level l
        from its current fields, nested in the new level l; the particles
        are deposited on the new levels."""
        lib = _load()
        if particles is None:
            x = y = z = q = np.zeros(1)
            npart = 0
        else:
            x, y, z, q = (np.ascontiguousarray(a, dtype=np.float64) for a in particles)
            npart = len(x)
        h = lib.orc_regrid(self._h, TAG_MODES[policy], float(tag_lambda), int(buffer), int(lmax),
                           _dptr(x), _dptr(y), _dptr(z), _dptr(q), npart)
        if not h:
            raise ValueError("oracle: " + lib.orc_last_error().decode())
        new = OracleHierarchy.__new__(OracleHierarchy)
        new._keep = (x, y, z, q)
        new._h = ctypes.c_void_p(h)
        new.n0 = self.n0
        new.robin_d = self.robin_d
        return new

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().orc_destroy(h)
            self._h = None

    @property
    def nlevels(self) -> int:
        return int(_load().orc_nlevels(self._h))

    def level_box(self, l):
        lo = np.zeros(3, np.int32)
        hi = np.zeros(3, np.int32)
        n = np.zeros(1, np.int32)
        _load().orc_level_box(self._h, l, _iptr(lo), _iptr(hi), _iptr(n))
        return lo.copy(), hi.copy(), int(n[0])

    def h(self, l):
        return 1.0 / (self.n0 * 2 ** l)

    def shape(self, l):
        lo, hi, _ = self.level_box(l)
        ext = hi - lo + 1
        return int(ext[2]), int(ext[1]), int(ext[0])

    def get(self, l, field):
        out = np.zeros(self.shape(l), np.float64)
        _load().orc_get_field(self._h, l, FIELDS[field], _dptr(out))
        return out

    def set(self, l, field, arr):
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(arr, np.float64), self.shape(l)))
        _load().orc_set_field(self._h, l, FIELDS[field], _dptr(a))

    def mask(self, l):
        out = np.zeros(self.shape(l), np.int8)
        _load().orc_get_mask(self._h, l, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
        return out

    def centres(self, l):
        """Cell-centre coordinates (x, y, z) of the dense layout of level l."""
        lo, hi, _ = self.level_box(l)
        h = self.h(l)
        ax = [(np.arange(lo[d], hi[d] + 1) + 0.5) * h for d in range(3)]
        Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return X, Y, Z

    def deposit(self, x, y, z, q):
        x, y, z, q = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, q))
        _load().orc_deposit(self._h, _dptr(x), _dptr(y), _dptr(z), _dptr(q), len(x))

    def solve(self, eps=1e-10, p=2, max_iter=100, nu1=2, nu2=2, bottom_rtol=1e-14, warm=False):
        rel = np.zeros(8)
        it = _load().orc_solve(self._h, float(eps), NORMS[p], int(max_iter), int(nu1), int(nu2),
                               float(bottom_rtol), int(bool(warm)), _dptr(rel))
        return int(it), rel[: self.nlevels].copy()

    def residual(self, p=2):
        rel = np.zeros(8)
        _load().orc_residual(self._h, NORMS[p], _dptr(rel))
        return rel[: self.nlevels].copy()

    def average_down(self):
        _load().orc_average_down(self._h)

    def efield(self):
        _load().orc_efield(self._h)

    def set_gather_buffer(self, b):
        """Interpolate from a refined level only b cells inside it."""
        _load().orc_set_gather_buffer(self._h, int(b))

    def gather(self, x, y, z, with_phi=False):
        x, y, z = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z))
        n = len(x)
        ex, ey, ez, ph = (np.zeros(n) for _ in range(4))
        _load().orc_gather(self._h, _dptr(x), _dptr(y), _dptr(z), n, _dptr(ex), _dptr(ey), _dptr(ez),
                           _dptr(ph) if with_phi else ctypes.cast(None, ctypes.POINTER(ctypes.c_double)))
        return (ex, ey, ez, ph) if with_phi else (ex, ey, ez)

    def bin(self, x, y, z):
        """(keys uint32, perm int64 stable by key, number of keys)."""
        x, y, z = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z))
        n = len(x)
        keys = np.zeros(max(n, 1), np.uint32)
        perm = np.zeros(max(n, 1), np.int64)
        lib = _load()
        nk = lib.orc_bin(self._h, _dptr(x), _dptr(y), _dptr(z), n,
                         keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)),
                         perm.ctypes.data_as(ctypes.POINTER(ctypes.c_long)))
        return keys[:n], perm[:n], int(nk)

    def matrix(self, l, which):
        lib = _load()
        nr, nc, nnz = (np.zeros(1, np.int32) for _ in range(3))
        lib.orc_matrix(self._h, l, MATRICES[which], _iptr(nr), _iptr(nc), _iptr(nnz), None, None, None)
        ptr = np.zeros(int(nr[0]) + 1, np.int32)
        col = np.zeros(max(int(nnz[0]), 1), np.int32)
        val = np.zeros(max(int(nnz[0]), 1), np.float64)
        lib.orc_matrix(self._h, l, MATRICES[which], _iptr(nr), _iptr(nc), _iptr(nnz), _iptr(ptr), _iptr(col),
                       _dptr(val))
        k = int(nnz[0])
        return sp.csr_matrix((val[:k], col[:k], ptr), shape=(int(nr[0]), int(nc[0])))

    def cells(self, l):
        n = self.level_box(l)[2]
        out = np.zeros((max(n, 1), 3), np.int32)
        _load().orc_cells(self._h, l, _iptr(out))
        return out[:n]

    def ghost_stats(self):
        out = (ctypes.c_long * 3)()
        _load().orc_ghost_stats(self._h, out)
        return {"quadratic": out[0], "linear": out[1], "constant": out[2]}

    def ghost_stencil(self, l, f, d, s):
        cols = np.zeros(9, np.int32)
        w = np.zeros(9)
        order = np.zeros(1, np.int32)
        n = _load().orc_ghost_stencil(self._h, l, int(f[0]), int(f[1]), int(f[2]), int(d), int(s), _iptr(cols),
                                      _dptr(w), _iptr(order))
        return cols[:n].copy(), w[:n].copy(), int(order[0])

    # -- helpers on the vector (row) layout ------------------------------
    def to_rows(self, l, dense):
        lo = self.level_box(l)[0]
        c = self.cells(l) - lo
        return dense[c[:, 2], c[:, 1], c[:, 0]]

    def from_rows(self, l, v):
        lo = self.level_box(l)[0]
        c = self.cells(l) - lo
        out = np.zeros(self.shape(l))
        out[c[:, 2], c[:, 1], c[:, 0]] = v
        return out
