"""ctypes front end of the plain C oracle (``lj_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by the smoke check and
by the benchmark's CPU-baseline leg, never by the CUDA library or its Python
binding.  Every function returns fresh numpy arrays and never touches a GPU.

Functions and the passages of Watanabe & Nakagawa (arXiv 1806.05713) they
follow:

* ``pairlist(..., method="brute")``: the O(N^2) definition of the Verlet list
  (section "Verlet List and Bookkeeping Method"): all j != i (j > i for the
  half list) with minimum-image r^2 < r_s^2, rows sorted by j.
* ``pairlist(..., method="cells")``: the linked-list cell method of the same
  section; must give the identical list.
* ``force``: Algorithm 3 (sorted list) with Algorithm 1 per pair; the
  momentum change of one call, p_i -= df r, p_j += df r (half list).
* ``pairlist_rows`` / ``force_rows``: the same two functions restricted to
  a block of rows (a bounded sample of a large system for CPU timing).
* ``force_atoms``: the momentum change of chosen atoms straight from the
  definition, summed over every other atom (no list; checks sampled atoms
  of systems too large to list on the CPU quickly).
* ``energy``: Eq. (1) truncated at r_c, optionally shifted to V(r_c) = 0.
* ``virial``: the pair virial sum r F(r) of the same truncated Eq. (1).
* ``force_vjp``: the adjoint of the force map F(q; eps, sigma), derived from
  Eq. (1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lj_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblj_oracle.so")
_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_int = ctypes.c_int
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile lj_oracle.c with gcc (no fused multiply-add) and return the path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.oracle_pairlist_brute.restype = _i64
        lib.oracle_pairlist_brute.argtypes = [_i64, _vp, _i64, _vp, _dbl, _int, _vp, _vp, _i64]
        lib.oracle_pairlist_cells.restype = _i64
        lib.oracle_pairlist_cells.argtypes = [_i64, _vp, _i64, _vp, _dbl, _int, _vp, _vp, _i64]
        lib.oracle_pairlist_cells_rows.restype = _i64
        lib.oracle_pairlist_cells_rows.argtypes = [_i64, _vp, _i64, _vp, _dbl, _int, _i64, _i64,
                                                   _vp, _vp, _i64]
        lib.oracle_force_rows.restype = None
        lib.oracle_force_rows.argtypes = [_i64, _vp, _i64, _vp, _i64, _i64, _i64, _vp, _vp, _int,
                                          _dbl, _dbl, _vp, _dbl, _dbl]
        lib.oracle_force_atoms.restype = None
        lib.oracle_force_atoms.argtypes = [_i64, _vp, _i64, _vp, _dbl, _dbl, _dbl, _dbl, _vp, _i64,
                                           _vp]
        lib.oracle_force.restype = None
        lib.oracle_force.argtypes = [_i64, _vp, _i64, _vp, _i64, _vp, _vp, _int, _dbl, _dbl,
                                     _vp, _dbl, _dbl]
        lib.oracle_energy.restype = _dbl
        lib.oracle_energy.argtypes = [_i64, _vp, _i64, _vp, _vp, _int, _dbl, _vp, _dbl, _dbl,
                                      _int]
        lib.oracle_virial.restype = _dbl
        lib.oracle_virial.argtypes = [_i64, _vp, _i64, _vp, _vp, _int, _dbl, _vp, _dbl, _dbl]
        lib.oracle_force_fs.restype = None
        lib.oracle_force_fs.argtypes = [_i64, _vp, _i64, _vp, _i64, _vp, _vp, _int, _dbl, _dbl,
                                        _vp, _dbl, _dbl]
        lib.oracle_energy_fs.restype = _dbl
        lib.oracle_energy_fs.argtypes = [_i64, _vp, _i64, _vp, _vp, _int, _dbl, _vp, _dbl, _dbl]
        lib.oracle_force_vjp.restype = None
        lib.oracle_force_vjp.argtypes = [_i64, _vp, _i64, _vp, _i64, _vp, _vp, _int, _dbl, _vp,
                                         _dbl, _dbl, _vp, _vp]
        _lib = lib
        return lib


def _rows(a: np.ndarray, name: str) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] < 3:
        raise ValueError(f"{name} must be (n, >=3) float64")
    return a


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def pairlist(q, box, rs: float, half: bool = True, method: str = "cells"):
    """Sorted CSR Verlet list (row_ptr int32[n+1], col int32[nnz])."""
    lib = _load()
    q = _rows(q, "q")
    L = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    n = q.shape[0]
    fn = {"brute": lib.oracle_pairlist_brute, "cells": lib.oracle_pairlist_cells}[method]
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    cap = max(1, 160 * n if half else 320 * n)
    while True:
        col = np.empty(cap, dtype=np.int32)
        nnz = fn(n, _ptr(q), q.shape[1], _ptr(L), float(rs), int(bool(half)), _ptr(row_ptr),
                 _ptr(col), cap)
        if nnz <= cap:
            return row_ptr, col[:nnz].copy()
        cap = int(nnz)


def pairlist_rows(q, box, rs: float, half: bool, i0: int, i1: int):
    """Rows i0 .. i1-1 of the cell-method list: (row_ptr int32[i1-i0+1]
    starting at 0, col int32 with global atom indices)."""
    lib = _load()
    q = _rows(q, "q")
    L = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    n = q.shape[0]
    if not 0 <= i0 <= i1 <= n:
        raise ValueError("row range outside the system")
    row_ptr = np.zeros(i1 - i0 + 1, dtype=np.int32)
    cap = max(1, (160 if half else 320) * (i1 - i0))
    while True:
        col = np.empty(cap, dtype=np.int32)
        nnz = lib.oracle_pairlist_cells_rows(n, _ptr(q), q.shape[1], _ptr(L), float(rs),
                                             int(bool(half)), int(i0), int(i1), _ptr(row_ptr),
                                             _ptr(col), cap)
        if nnz <= cap:
            return row_ptr, col[:nnz].copy()
        cap = int(nnz)


def force_rows(q, p, row_ptr, col, half: bool, dt: float, rc: float, box, i0: int, i1: int,
               eps: float = 1.0, sigma: float = 1.0, inplace: bool = False) -> np.ndarray:
    """Momenta after one force call over rows i0 .. i1-1 of a list given in
    the pairlist_rows form; p is not modified unless inplace (then p, a
    C-contiguous float64 (n, >=3) array, is updated and returned -- the
    timing loops use this so that no copy of p is made per call)."""
    lib = _load()
    q = _rows(q, "q")
    if inplace:
        if not (isinstance(p, np.ndarray) and p.dtype == np.float64 and p.ndim == 2
                and p.shape[1] >= 3 and p.flags["C_CONTIGUOUS"]):
            raise ValueError("inplace needs a C-contiguous float64 (n, >=3) array")
        out = p
    else:
        out = _rows(p, "p").copy()
    L = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if row_ptr.size != i1 - i0 + 1 or not 0 <= i0 <= i1 <= q.shape[0]:
        raise ValueError("row_ptr does not match the row range")
    lib.oracle_force_rows(q.shape[0], _ptr(q), q.shape[1], _ptr(out), out.shape[1], int(i0),
                          int(i1), _ptr(row_ptr), _ptr(col), int(bool(half)), float(dt), float(rc),
                          _ptr(L), float(eps), float(sigma))
    return out


def force_atoms(q, idx, dt: float, rc: float, box, eps: float = 1.0,
                sigma: float = 1.0) -> np.ndarray:
    """Momentum change (m, 3) of the atoms idx in one force call, from the
    definition over all atoms (no list)."""
    lib = _load()
    q = _rows(q, "q")
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    if idx.size and (idx.min() < 0 or idx.max() >= q.shape[0]):
        raise ValueError("atom index outside the system")
    L = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    out = np.zeros((idx.size, 3))
    lib.oracle_force_atoms(q.shape[0], _ptr(q), q.shape[1], _ptr(L), float(dt), float(rc),
                           float(eps), float(sigma), _ptr(idx), idx.size, _ptr(out))
    return out


def force(q, p, row_ptr, col, half: bool, dt: float, rc: float, box, eps: float = 1.0,
          sigma: float = 1.0) -> np.ndarray:
    """Momenta after one force call (Algorithm 3); p is not modified."""
    lib = _load()
    q = _rows(q, "q")
    out = _rows(p, "p").copy()
    L = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    lib.oracle_force(q.shape[0], _ptr(q), q.shape[1], _ptr(out), out.shape[1], _ptr(row_ptr),
                     _ptr(col), int(bool(half)), float(dt), float(rc), _ptr(L), float(eps),
                     float(sigma))
    return out


def forces(q, row_ptr, col, half: bool, rc: float, box, eps: float = 1.0,
           sigma: float = 1.0) -> np.ndarray:
    """Forces F (n, 3): the momentum change of one call with p = 0, dt = 1."""
    p0 = np.zeros((np.asarray(q).shape[0], 3))
    return force(q, p0, row_ptr, col, half, 1.0, rc, box, eps, sigma)


def energy(q, row_ptr, col, half: bool, rc: float, box, eps: float = 1.0, sigma: float = 1.0,
           shifted: bool = False) -> float:
    """Potential energy, Eq. (1), over unique pairs with r < r_c."""
    lib = _load()
    q = _rows(q, "q")
    L = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return float(lib.oracle_energy(q.shape[0], _ptr(q), q.shape[1], _ptr(row_ptr), _ptr(col),
                                   int(bool(half)), float(rc), _ptr(L), float(eps),
                                   float(sigma), int(bool(shifted))))


def virial(q, row_ptr, col, half: bool, rc: float, box, eps: float = 1.0,
           sigma: float = 1.0) -> float:
    """Pair virial W = sum over unique pairs with r < r_c of r F(r),
    F = -dV/dr of Eq. (1)."""
    lib = _load()
    q = _rows(q, "q")
    L = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return float(lib.oracle_virial(q.shape[0], _ptr(q), q.shape[1], _ptr(row_ptr), _ptr(col),
                                   int(bool(half)), float(rc), _ptr(L), float(eps), float(sigma)))


def force_fs(q, p, row_ptr, col, half: bool, dt: float, rc: float, box, eps: float = 1.0,
             sigma: float = 1.0) -> np.ndarray:
    """Momenta after one force call with the force-shifted truncation (the
    pair force -V'(r) + V'(r_c), zero at r_c); p is not modified."""
    lib = _load()
    q = _rows(q, "q")
    out = _rows(p, "p").copy()
    L = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    lib.oracle_force_fs(q.shape[0], _ptr(q), q.shape[1], _ptr(out), out.shape[1], _ptr(row_ptr),
                        _ptr(col), int(bool(half)), float(dt), float(rc), _ptr(L), float(eps),
                        float(sigma))
    return out


def energy_fs(q, row_ptr, col, half: bool, rc: float, box, eps: float = 1.0,
              sigma: float = 1.0) -> float:
    """Force-shifted potential energy: sum of V(r) - V(r_c) - (r - r_c) V'(r_c)
    over unique pairs with r < r_c."""
    lib = _load()
    q = _rows(q, "q")
    L = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return float(lib.oracle_energy_fs(q.shape[0], _ptr(q), q.shape[1], _ptr(row_ptr), _ptr(col),
                                      int(bool(half)), float(rc), _ptr(L), float(eps),
                                      float(sigma)))


def force_vjp(q, R, row_ptr, col, half: bool, rc: float, box, eps: float = 1.0,
              sigma: float = 1.0):
    """(dLoss/dq (n,3), dLoss/deps, dLoss/dsigma) for R = dLoss/dF."""
    lib = _load()
    q = _rows(q, "q")
    R = _rows(R, "R")
    n = q.shape[0]
    L = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    gq = np.zeros((n, 3))
    ges = np.zeros(2)
    lib.oracle_force_vjp(n, _ptr(q), q.shape[1], _ptr(R), R.shape[1], _ptr(row_ptr), _ptr(col),
                         int(bool(half)), float(rc), _ptr(L), float(eps), float(sigma),
                         _ptr(gq), _ptr(ges))
    return gq, float(ges[0]), float(ges[1])
