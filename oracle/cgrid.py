"""ctypes wrapper and build step for the plain C oracle loops (cgrid.c).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .index import index_vis
from .wkernel import KernelTables, Params

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cgrid.c")
_LIB = os.path.join(_HERE, "_cgrid.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile cgrid.c (gcc, -O2 -ffp-contract=off, OpenMP) next to this file."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
               "-fPIC", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        lib.oracle_grid.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, p, p, p,
                                    ctypes.c_int64, p, p, p, p, p, p, p, p, p, ctypes.c_int]
        lib.oracle_grid_lattice.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, p, p, p,
                                            ctypes.c_int64, p, p, p, p, p, p, p, p,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int, p]
        lib.oracle_degrid.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, p, p, p,
                                      ctypes.c_int64, p, p, p, p, p, p, p, p, ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class Oracle:
    """FP64 gridder/degridder for one set of imaging parameters."""

    def __init__(self, prm: Params, tables: KernelTables | None = None):
        self.prm = prm
        self.tables = KernelTables(prm) if tables is None else tables
        flat, offs = self.tables.flat()
        self._table = np.ascontiguousarray(flat.view(np.float64))
        self._offs = np.ascontiguousarray(offs[:-1].astype(np.int64))
        self._support = np.ascontiguousarray(self.tables.support.astype(np.int32))

    def index(self, uvw_m, freq_hz):
        return index_vis(uvw_m, freq_hz, self.prm)

    def _idx_arrays(self, idx):
        cvt = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        return (cvt(idx["ku"]), cvt(idx["kv"]), cvt(idx["ou"]), cvt(idx["ov"]),
                cvt(idx["plane"]), np.ascontiguousarray(idx["flags"], dtype=np.uint8))

    def grid(self, uvw_m, freq_hz, vis, weight=None, grid=None, idx=None, nthreads=None):
        """Accumulate vis [nrow, nchan, npol] onto grid [npol, N, N] (complex128)."""
        prm = self.prm
        N, npol = prm.grid_n, prm.npol
        if idx is None:
            idx = self.index(uvw_m, freq_hz)
        nvis = idx["ku"].shape[0]
        v = np.ascontiguousarray(np.asarray(vis, dtype=np.complex128).reshape(nvis, npol))
        wt = None
        if weight is not None:
            wt = np.ascontiguousarray(np.asarray(weight, dtype=np.float64).reshape(nvis, npol))
        if grid is None:
            grid = np.zeros((npol, N, N), dtype=np.complex128)
        assert grid.dtype == np.complex128 and grid.flags.c_contiguous
        a = self._idx_arrays(idx)
        _load().oracle_grid(N, npol, prm.oversample, _ptr(self._support), _ptr(self._offs),
                            _ptr(self._table), nvis, *[_ptr(x) for x in a], _ptr(v), _ptr(wt),
                            _ptr(grid), nthreads or default_threads())
        return grid

    def degrid(self, uvw_m, freq_hz, grid, idx=None, nthreads=None):
        """Visibilities [nrow * nchan, npol] (complex128) from grid [npol, N, N]."""
        prm = self.prm
        N, npol = prm.grid_n, prm.npol
        if idx is None:
            idx = self.index(uvw_m, freq_hz)
        nvis = idx["ku"].shape[0]
        g = np.ascontiguousarray(np.asarray(grid, dtype=np.complex128))
        assert g.shape == (npol, N, N)
        out = np.zeros((nvis, npol), dtype=np.complex128)
        a = self._idx_arrays(idx)
        _load().oracle_degrid(N, npol, prm.oversample, _ptr(self._support), _ptr(self._offs),
                              _ptr(self._table), nvis, *[_ptr(x) for x in a], _ptr(g),
                              _ptr(out), nthreads or default_threads())
        return out

    def grid_lattice(self, uvw_m, freq_hz, vis, off: int, step: int, m: int, weight=None, idx=None):
        """The grid at lattice points (off + step*a, off + step*b): [npol, m, m]
        (row index b = v), the same per-point sums as ``grid``."""
        prm = self.prm
        npol = prm.npol
        if idx is None:
            idx = self.index(uvw_m, freq_hz)
        nvis = idx["ku"].shape[0]
        v = np.ascontiguousarray(np.asarray(vis, dtype=np.complex128).reshape(nvis, npol))
        wt = None
        if weight is not None:
            wt = np.ascontiguousarray(np.asarray(weight, dtype=np.float64).reshape(nvis, npol))
        out = np.zeros((npol, m, m), dtype=np.complex128)
        a = self._idx_arrays(idx)
        _load().oracle_grid_lattice(prm.grid_n, npol, prm.oversample, _ptr(self._support),
                                    _ptr(self._offs), _ptr(self._table), nvis,
                                    *[_ptr(x) for x in a], _ptr(v), _ptr(wt), off, step, m,
                                    _ptr(out))
        return out
