"""Thin Python binding of the C ABI in ``include/lj_gb300.h``.

Each function has the name of the C entry point it calls and only
marshals arguments: torch CUDA tensors provide device memory and the
current CUDA stream; every step of the computation runs in the library's
kernels.  The library is loaded from the package's ``_build`` folder; if it
is missing or no CUDA device is present the functions raise -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

LJ_OK = 0
LJ_ERR_ARG = 1
LJ_ERR_BOX = 2
LJ_ERR_RANGE = 3
LJ_ERR_CAPACITY = 4
LJ_ERR_CUDA = 5
LJ_ERR_DEVICE = 6

LJ_FP64 = 0
LJ_MIXED = 1
LJ_DFLOAT = 2
LJ_TPI_AUTO = 0
LJ_SCHED_SWP2 = 128
LJ_SCHED_SORTED = 512
LJ_SCHED_IMAGES = 1024
LJ_SCHED_FIXED = 2048
LJ_SCHED_STREAM = 8192
LJ_SCHED_CELLS = 16384
LJ_MD_LAST_HALF_KICK = 1
LJ_PEAK_DFMA = 0
LJ_PEAK_FFMA = 1
LJ_PEAK_FFMA2 = 2
LJ_PEAK_L2_READ = 3
LJ_RCP_FP64_FAST = 1
LJ_RSQRT_FP64 = 2
LJ_RCP_DF = 3
LJ_RCP_DF2 = 4
LJ_RCP_FP32 = 5
LJ_RCP_FP64_INT = 6
LJ_STATIC_MAX_ATOMS = 131072

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "liblj_gb300.so")
_lib = None

_i64, _dbl, _int, _vp, _sz = ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
_dbl3 = ctypes.c_double * 3
_i64p = ctypes.POINTER(ctypes.c_int64)

class LjSystem(ctypes.Structure):
    """Mirror of the C struct lj_system."""
    _fields_ = [("atom_offset", ctypes.c_int64), ("n", ctypes.c_int64),
                ("row_offset", ctypes.c_int64), ("entry_offset", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("box", ctypes.c_double * 3), ("r_cut", ctypes.c_double),
                ("eps", ctypes.c_double), ("sigma", ctypes.c_double), ("half", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class LjBatch(ctypes.Structure):
    """Mirror of the C struct lj_batch."""
    _fields_ = [("plan_dev", ctypes.c_void_p), ("plan_bytes", ctypes.c_size_t),
                ("nitems", ctypes.c_int64), ("total_atoms", ctypes.c_int64),
                ("dt", ctypes.c_double), ("nsys", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("tpi", ctypes.c_int32), ("rows_per_item", ctypes.c_int32),
                ("blocks", ctypes.c_int32), ("flags", ctypes.c_int32)]


_sysp = ctypes.POINTER(LjSystem)
_batchp = ctypes.POINTER(LjBatch)
_intp = ctypes.POINTER(ctypes.c_int)
_fltp = ctypes.POINTER(ctypes.c_float)

# (name, restype, argtypes) of every exported entry point.
SIGNATURES = {
    "lj_status_string": (ctypes.c_char_p, [_int]),
    "lj_last_cuda_error": (ctypes.c_char_p, []),
    "lj_version": (_int, []),
    "lj_kernel_launch_count": (ctypes.c_ulonglong, []),
    "lj_pairlist_workspace_bytes": (_sz, [_i64, _dbl3, _dbl]),
    "lj_build_pairlist": (_int, [_vp, _i64, _dbl3, _dbl, _int, _vp, _vp, _i64, _vp, _sz, _i64p,
                                 _i64p, _vp]),
    "lj_build_pairlist_static": (_int, [_vp, _i64, _dbl3, _dbl, _int, _vp, _vp, _i64, _i64p, _i64p,
                                        _vp]),
    "lj_force_workspace_bytes": (_sz, [_i64, _dbl3, _int]),
    "lj_force": (_int, [_vp, _vp, _i64, _vp, _vp, _i64, _int, _dbl, _dbl, _dbl3, _dbl, _dbl, _int,
                        _int, _vp, _sz, _vp]),
    "lj_batch_plan_bytes": (_sz, [_sysp, _int, _int]),
    "lj_batch_init": (_int, [_batchp, _sysp, _int, _dbl, _int, _int, _int, _vp, _sz, _vp]),
    "lj_force_batched_workspace_bytes": (_sz, [_batchp]),
    "lj_force_batched": (_int, [_batchp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "lj_autotune_force": (_int, [_vp, _vp, _i64, _vp, _vp, _i64, _int, _dbl, _dbl, _dbl3, _dbl, _dbl,
                                 _int, _intp, _int, _int, _vp, _sz, _intp, _fltp, _fltp, _vp]),
    "lj_autotune_batched": (_int, [_sysp, _int, _dbl, _int, _intp, _int, _intp, _int, _vp, _vp, _vp,
                                   _vp, _vp, _sz, _vp, _sz, _int, _intp, _intp, _fltp, _vp]),
    "lj_drift": (_int, [_vp, _vp, _i64, _dbl, _dbl3, _vp, _vp]),
    "lj_md_steps": (_int, [_vp, _vp, _i64, _vp, _vp, _i64, _int, _dbl, _dbl, _dbl, _dbl3, _dbl, _dbl,
                           _int, _int, _i64, _int, _vp, _vp, _vp, _vp, _sz, _vp]),
    "lj_force_vjp_workspace_bytes": (_sz, [_i64, _int]),
    "lj_force_vjp": (_int, [_vp, _vp, _i64, _vp, _vp, _i64, _int, _dbl, _dbl3, _dbl, _dbl, _int,
                            _vp, _vp, _vp, _sz, _vp]),
    "lj_force_strided": (_int, [_vp, _vp, _i64, _i64, _i64, _vp, _vp, _i64, _int, _dbl, _dbl, _dbl3,
                                _dbl, _dbl, _int, _vp]),
    "lj_force_energy_workspace_bytes": (_sz, [_i64]),
    "lj_force_energy": (_int, [_vp, _vp, _i64, _vp, _vp, _i64, _int, _dbl, _dbl, _dbl3, _dbl, _dbl,
                               _int, _vp, _vp, _sz, _vp]),
    "lj_force_energy_virial": (_int, [_vp, _vp, _i64, _vp, _vp, _i64, _int, _dbl, _dbl, _dbl3, _dbl,
                                      _dbl, _int, _vp, _vp, _vp, _sz, _vp]),
    "lj_force_shifted_workspace_bytes": (_sz, [_i64]),
    "lj_force_shifted": (_int, [_vp, _vp, _i64, _vp, _vp, _i64, _int, _dbl, _dbl, _dbl3, _dbl, _dbl,
                                _vp, _vp, _sz, _vp]),
    "lj_measure_peak": (_int, [_int, _vp, _sz, _i64, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), _vp]),
    "lj_eval_reciprocal": (_int, [_int, _vp, _i64, _vp, _vp, _vp]),
    "lj_energy_workspace_bytes": (_sz, [_i64]),
    "lj_energy": (_int, [_vp, _i64, _vp, _vp, _i64, _int, _dbl, _dbl3, _dbl, _dbl, _int, _vp, _vp,
                         _sz, _vp]),
}


class LJError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _lib
        msg = lib.lj_status_string(status).decode() if lib else f"status {status}"
        if status == LJ_ERR_CUDA and lib:
            msg += " -- " + lib.lj_last_cuda_error().decode()
        super().__init__(f"{where}: {msg}")
        self.status = status


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"CUDA library not built ({_LIB_PATH} missing); "
                           "run paper_1806_05713_gb300.build.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != LJ_OK:
        raise LJError(status, where)


def _box3(box) -> ctypes.Array:
    b = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    return _dbl3(*[float(x) for x in b])


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str, shape=None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous {dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")
    return t.data_ptr()


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


@dataclass
class PairList:
    """CSR Verlet list on the device (row_ptr int32[n+1], col int32[nnz]).

    ``workspace`` is the builder's scratch, kept so that a rebuild can reuse
    every buffer (pass the list as ``reuse=``)."""
    row_ptr: torch.Tensor
    col: torch.Tensor
    n: int
    nnz: int
    half: bool
    r_search: float
    max_row: int
    workspace: torch.Tensor | None = None

    @property
    def col_view(self) -> torch.Tensor:
        return self.col[: self.nnz]


def lj_pairlist_workspace_bytes(n: int, box, r_search: float) -> int:
    return int(load().lj_pairlist_workspace_bytes(int(n), _box3(box), float(r_search)))


def lj_build_pairlist(q4: torch.Tensor, box, r_search: float, half: bool = True,
                      col_capacity: int | None = None, stream=None,
                      reuse: PairList | None = None) -> PairList:
    """Build the sorted CSR list.  Buffers of ``reuse`` are used when large
    enough; a too-small column buffer is regrown to the reported size and
    the build retried once."""
    lib = load()
    n = int(q4.shape[0]) if q4.dim() == 2 else 0
    qp = _dev(q4, torch.float64, "q4", (n, 4))
    dev = q4.device
    bx = _box3(box)
    wsb = int(lib.lj_pairlist_workspace_bytes(n, bx, float(r_search)))
    if reuse is not None and reuse.row_ptr.numel() == n + 1:
        row_ptr = reuse.row_ptr
    else:
        row_ptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
    if reuse is not None and reuse.workspace is not None and reuse.workspace.numel() >= wsb:
        ws = reuse.workspace
    else:
        ws = _workspace(wsb, dev)
    if col_capacity is None:
        col_capacity = max(1, (90 if half else 180) * n)
    col = reuse.col if reuse is not None else None
    for _ in range(2):
        if col is None or col.numel() < col_capacity:
            col = torch.empty(max(1, int(col_capacity)), dtype=torch.int32, device=dev)
        nnz = ctypes.c_int64(0)
        mrow = ctypes.c_int64(0)
        st = lib.lj_build_pairlist(qp, n, bx, float(r_search), int(bool(half)),
                                   row_ptr.data_ptr(), col.data_ptr(), int(col.numel()),
                                   ws.data_ptr(), ws.numel(), ctypes.byref(nnz), ctypes.byref(mrow),
                                   _stream(stream))
        if st == LJ_ERR_CAPACITY and nnz.value > col.numel():
            col_capacity = nnz.value
            col = None
            continue
        _check(st, "lj_build_pairlist")
        return PairList(row_ptr, col, n, int(nnz.value), bool(half), float(r_search),
                        int(mrow.value), ws)
    raise LJError(LJ_ERR_CAPACITY, "lj_build_pairlist")


def lj_build_pairlist_static(q4: torch.Tensor, box, r_search: float, half: bool,
                             row_ptr: torch.Tensor, col: torch.Tensor, stream=None):
    """The allocation-free builder: scratch comes from the library's fixed
    device array; the caller passes the row_ptr (n+1) and col outputs.
    Returns (nnz, max_row)."""
    lib = load()
    n = int(q4.shape[0])
    nnz = ctypes.c_int64(0)
    mrow = ctypes.c_int64(0)
    st = lib.lj_build_pairlist_static(_dev(q4, torch.float64, "q4", (n, 4)), n, _box3(box),
                                      float(r_search), int(bool(half)),
                                      _dev(row_ptr, torch.int32, "row_ptr", (n + 1,)),
                                      _dev(col, torch.int32, "col"), int(col.numel()),
                                      ctypes.byref(nnz), ctypes.byref(mrow), _stream(stream))
    _check(st, "lj_build_pairlist_static")
    return int(nnz.value), int(mrow.value)


def lj_force_workspace_bytes(n: int, box, precision: int = LJ_FP64) -> int:
    return int(load().lj_force_workspace_bytes(int(n), _box3(box), int(precision)))


def lj_force(q4: torch.Tensor, p4: torch.Tensor, plist: PairList, dt: float, r_cut: float, box,
             eps: float = 1.0, sigma: float = 1.0, precision: int = LJ_FP64, tpi: int = LJ_TPI_AUTO,
             workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """p4 += impulses (in place); returns p4."""
    lib = load()
    n = plist.n
    qp = _dev(q4, torch.float64, "q4", (n, 4))
    pp = _dev(p4, torch.float64, "p4", (n, 4))
    need = lib.lj_force_workspace_bytes(n, _box3(box), int(precision))
    if workspace is None and need > 0:
        workspace = _workspace(need, q4.device)
    wsp = workspace.data_ptr() if workspace is not None else None
    wsb = workspace.numel() if workspace is not None else 0
    st = lib.lj_force(qp, pp, n, plist.row_ptr.data_ptr(), plist.col.data_ptr(), plist.nnz,
                      int(plist.half), float(dt), float(r_cut), _box3(box), float(eps),
                      float(sigma), int(precision), int(tpi), wsp, wsb, _stream(stream))
    _check(st, "lj_force")
    return p4


def lj_force_prepared(q4: torch.Tensor, p4: torch.Tensor, plist: PairList, dt: float,
                      r_cut: float, box, eps: float = 1.0, sigma: float = 1.0,
                      precision: int = LJ_FP64, tpi: int = LJ_TPI_AUTO,
                      workspace: torch.Tensor | None = None, stream=None):
    """lj_force with its arguments marshalled once; returns a no-argument
    callable that enqueues the same call again (for tight loops)."""
    lib = load()
    n = plist.n
    qp = _dev(q4, torch.float64, "q4", (n, 4))
    pp = _dev(p4, torch.float64, "p4", (n, 4))
    need = lib.lj_force_workspace_bytes(n, _box3(box), int(precision))
    if workspace is None and need > 0:
        workspace = _workspace(need, q4.device)
    args = (qp, pp, n, plist.row_ptr.data_ptr(), plist.col.data_ptr(), plist.nnz,
            int(plist.half), float(dt), float(r_cut), _box3(box), float(eps), float(sigma),
            int(precision), int(tpi), workspace.data_ptr() if workspace is not None else None,
            workspace.numel() if workspace is not None else 0, _stream(stream))
    keep = (q4, p4, plist, workspace)
    fn = lib.lj_force

    def call():
        st = fn(*args)
        if st != LJ_OK:
            raise LJError(st, "lj_force")
        return keep[1]
    return call


def lj_energy_workspace_bytes(n: int) -> int:
    return int(load().lj_energy_workspace_bytes(int(n)))


def lj_energy(q4: torch.Tensor, plist: PairList, r_cut: float, box, eps: float = 1.0,
              sigma: float = 1.0, shifted: bool = False, out: torch.Tensor | None = None,
              workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Potential energy into a 1-element device tensor (returned)."""
    lib = load()
    n = plist.n
    qp = _dev(q4, torch.float64, "q4", (n, 4))
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=q4.device)
    if workspace is None:
        workspace = _workspace(lib.lj_energy_workspace_bytes(n), q4.device)
    st = lib.lj_energy(qp, n, plist.row_ptr.data_ptr(), plist.col.data_ptr(), plist.nnz,
                       int(plist.half), float(r_cut), _box3(box), float(eps), float(sigma),
                       int(bool(shifted)), _dev(out, torch.float64, "out"), workspace.data_ptr(),
                       workspace.numel(), _stream(stream))
    _check(st, "lj_energy")
    return out


def lj_force_vjp_workspace_bytes(n: int, precision: int = LJ_FP64) -> int:
    return int(load().lj_force_vjp_workspace_bytes(int(n), int(precision)))


def lj_force_vjp(q4: torch.Tensor, gradF4: torch.Tensor, plist: PairList, r_cut: float, box,
                 eps: float = 1.0, sigma: float = 1.0, precision: int = LJ_FP64,
                 gradq4: torch.Tensor | None = None, grad_eps_sigma: torch.Tensor | None = None,
                 workspace: torch.Tensor | None = None, stream=None):
    """(dLoss/dq (n, 4), dLoss/d(eps, sigma) (2,)) for dLoss/dF = gradF4."""
    lib = load()
    n = plist.n
    if gradq4 is None:
        gradq4 = torch.empty((n, 4), dtype=torch.float64, device=q4.device)
    if grad_eps_sigma is None:
        grad_eps_sigma = torch.empty(2, dtype=torch.float64, device=q4.device)
    if workspace is None:
        workspace = _workspace(lib.lj_force_vjp_workspace_bytes(n, int(precision)), q4.device)
    st = lib.lj_force_vjp(_dev(q4, torch.float64, "q4", (n, 4)),
                          _dev(gradF4, torch.float64, "gradF4", (n, 4)), n,
                          plist.row_ptr.data_ptr(), plist.col.data_ptr(), plist.nnz,
                          int(plist.half), float(r_cut), _box3(box), float(eps), float(sigma),
                          int(precision), _dev(gradq4, torch.float64, "gradq4", (n, 4)),
                          _dev(grad_eps_sigma, torch.float64, "grad_eps_sigma", (2,)),
                          workspace.data_ptr(), workspace.numel(), _stream(stream))
    _check(st, "lj_force_vjp")
    return gradq4, grad_eps_sigma


def lj_autotune_force(q4: torch.Tensor, plist: PairList, dt: float, r_cut: float, box,
                      eps: float = 1.0, sigma: float = 1.0, precision: int = LJ_FP64,
                      candidates=None, reps: int = 5, stream=None):
    """Fastest schedule among `candidates` for this system and list (times
    each with CUDA events on a scratch momentum array).  Returns
    (best_tpi, best_ms, {tpi: ms})."""
    lib = load()
    if candidates is None:
        S, W, I, F = LJ_SCHED_SORTED, LJ_SCHED_SWP2, LJ_SCHED_IMAGES, LJ_SCHED_FIXED
        # the fixed-point schedules are refused (and skipped) for boxes wider
        # than 1024 r_c, where the image-selected ones take over
        R, C = LJ_SCHED_STREAM, LJ_SCHED_CELLS
        candidates = ([F | 4, F | 8, F | 16, S | F | 8, F | R | 8, F | R | 16, F | R | 32, I | 4,
                       I | 8, I | 16, I | W | 8]
                      if precision == LJ_FP64 else
                      [W | 8, W | 4, W | 16, S | W | 8, 4, 8, 16, S | 4, S | 8]
                      if precision == LJ_DFLOAT else
                      [4, 8, 16, W | 4, W | 8, W | 16, S | 8, S | W | 8, C | 8, C | W | 4, C | W | 8])
    n = plist.n
    scratch = torch.zeros((n, 4), dtype=torch.float64, device=q4.device)
    ws = _workspace(lib.lj_force_workspace_bytes(n, _box3(box), int(precision)), q4.device)
    arr = (ctypes.c_int * len(candidates))(*candidates)
    ms = (ctypes.c_float * len(candidates))()
    best = ctypes.c_int(0)
    best_ms = ctypes.c_float(0)
    st = lib.lj_autotune_force(_dev(q4, torch.float64, "q4", (n, 4)), scratch.data_ptr(), n,
                               plist.row_ptr.data_ptr(), plist.col.data_ptr(), plist.nnz,
                               int(plist.half), float(dt), float(r_cut), _box3(box), float(eps),
                               float(sigma), int(precision), arr, len(candidates), int(reps),
                               ws.data_ptr(), ws.numel(), ctypes.byref(best), ctypes.byref(best_ms),
                               ms, _stream(stream))
    _check(st, "lj_autotune_force")
    return int(best.value), float(best_ms.value), {c: float(m) for c, m in zip(candidates, ms)}


def lj_autotune_layout(q4: torch.Tensor, box, r_search: float, dt: float, r_cut: float,
                       eps: float = 1.0, sigma: float = 1.0, precision: int = LJ_FP64,
                       reps: int = 5, stream=None):
    """The list layout chosen by measurement: builds the half list (p_j by
    atomics) and the full list (no p_j writes), tunes the schedule on each
    with lj_autotune_force and keeps the faster.  Returns (plist, tpi, ms,
    {(half, tpi): ms})."""
    best, table = None, {}
    for half in (True, False):
        pl = lj_build_pairlist(q4, box, r_search, half, stream=stream)
        t, ms, tab = lj_autotune_force(q4, pl, dt, r_cut, box, eps, sigma, precision, reps=reps,
                                       stream=stream)
        table.update({(half, c): m for c, m in tab.items()})
        if best is None or ms < best[2]:
            best = (pl, t, ms)
    return best[0], best[1], best[2], table


def lj_drift(q4: torch.Tensor, p4: torch.Tensor, dt: float, box,
             max_disp2: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """q += dt p (wrapped); returns the 1-element device tensor max |dt p|^2."""
    lib = load()
    n = int(q4.shape[0])
    if max_disp2 is None:
        max_disp2 = torch.empty(1, dtype=torch.float64, device=q4.device)
    st = lib.lj_drift(_dev(q4, torch.float64, "q4", (n, 4)), _dev(p4, torch.float64, "p4", (n, 4)),
                      n, float(dt), _box3(box), _dev(max_disp2, torch.float64, "max_disp2"),
                      _stream(stream))
    _check(st, "lj_drift")
    return max_disp2


def lj_md_state_new(device) -> torch.Tensor:
    """A zeroed lj_md_state (48 bytes) in device memory."""
    return torch.zeros(6, dtype=torch.float64, device=device)


def lj_md_state_read(state: torch.Tensor) -> dict:
    """The fields of an lj_md_state (one device-to-host copy; synchronises)."""
    a = state.cpu().numpy()
    ints = a.view(np.int32)
    return {"moved": float(a[0]), "last_disp2": float(a[2]), "stale": int(ints[8]),
            "steps": int(ints[9])}


def lj_md_steps(q4: torch.Tensor, p4: torch.Tensor, plist: PairList, steps: int, dt: float,
                r_cut: float, r_search: float, box, eps: float = 1.0, sigma: float = 1.0,
                precision: int = LJ_FP64, tpi: int = LJ_TPI_AUTO, state: torch.Tensor | None = None,
                workspace: torch.Tensor | None = None, last_half_kick: bool = False,
                q_build: torch.Tensor | None = None, energies: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """Enqueue `steps` leapfrog steps (drift, then a kick by dt; dt/2 on the
    last one with last_half_kick) with the bookkeeping test on the device;
    returns the lj_md_state tensor.  q_build: the positions the list was
    built from (the displacement bound) or None (the summed fastest-atom
    bound).  energies: a device tensor of `steps` doubles for U(q) of each
    step (FP64).  Once the margin is used up the library empties plist's
    rows and the remaining steps do nothing: read the state, rebuild, kick
    once, continue."""
    lib = load()
    n = int(q4.shape[0])
    if state is None:
        state = lj_md_state_new(q4.device)
    if state.dtype != torch.float64 or state.numel() != 6 or not state.is_cuda:
        raise TypeError("state must be a 6-element CUDA float64 tensor (lj_md_state_new)")
    if workspace is None:
        nb = lj_force_workspace_bytes(n, box, precision)
        if energies is not None:
            nb = max(nb, lj_force_energy_workspace_bytes(n))
        workspace = _workspace(nb, q4.device)
    qb = 0 if q_build is None else _dev(q_build, torch.float64, "q_build", (n, 4))
    if energies is not None and energies.numel() < int(steps):
        raise ValueError("energies must hold one double per step")
    ep = 0 if energies is None else _dev(energies, torch.float64, "energies")
    st = lib.lj_md_steps(_dev(q4, torch.float64, "q4", (n, 4)), _dev(p4, torch.float64, "p4", (n, 4)),
                         n, plist.row_ptr.data_ptr(), plist.col.data_ptr(), plist.nnz,
                         int(plist.half), float(dt), float(r_cut), float(r_search), _box3(box),
                         float(eps), float(sigma), int(precision), int(tpi), int(steps),
                         LJ_MD_LAST_HALF_KICK if last_half_kick else 0, qb, ep, state.data_ptr(),
                         workspace.data_ptr(), workspace.numel(), _stream(stream))
    _check(st, "lj_md_steps")
    return state


def lj_force_strided(q: torch.Tensor, p: torch.Tensor, n: int, row_stride: int, comp_stride: int,
                     plist: PairList, dt: float, r_cut: float, box, eps: float = 1.0,
                     sigma: float = 1.0, lanes_per_row: int = 8, p_offset: int = 0, stream=None):
    """FP64 force with q and p in a strided layout (AoS4, AoS8, SoA, ...);
    p is read at p.data_ptr() + 8 * p_offset (p_offset = 4 for AoS8 records)."""
    lib = load()
    for t, name in ((q, "q"), (p, "p")):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
            raise TypeError(f"{name} must be a CUDA float64 tensor")
    st = lib.lj_force_strided(q.data_ptr(), p.data_ptr() + 8 * int(p_offset), int(n),
                              int(row_stride), int(comp_stride), plist.row_ptr.data_ptr(),
                              plist.col.data_ptr(), plist.nnz, int(plist.half), float(dt),
                              float(r_cut), _box3(box), float(eps), float(sigma),
                              int(lanes_per_row), _stream(stream))
    _check(st, "lj_force_strided")
    return p


def lj_force_energy_workspace_bytes(n: int) -> int:
    return int(load().lj_force_energy_workspace_bytes(int(n)))


def lj_force_energy(q4: torch.Tensor, p4: torch.Tensor, plist: PairList, dt: float, r_cut: float,
                    box, eps: float = 1.0, sigma: float = 1.0, shifted: bool = False,
                    out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """p4 += impulses (FP64) and the potential energy into a 1-element tensor."""
    lib = load()
    n = plist.n
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=q4.device)
    if workspace is None:
        workspace = _workspace(lib.lj_force_energy_workspace_bytes(n), q4.device)
    st = lib.lj_force_energy(_dev(q4, torch.float64, "q4", (n, 4)),
                             _dev(p4, torch.float64, "p4", (n, 4)), n, plist.row_ptr.data_ptr(),
                             plist.col.data_ptr(), plist.nnz, int(plist.half), float(dt),
                             float(r_cut), _box3(box), float(eps), float(sigma), int(bool(shifted)),
                             _dev(out, torch.float64, "out"), workspace.data_ptr(),
                             workspace.numel(), _stream(stream))
    _check(st, "lj_force_energy")
    return out


def lj_force_energy_virial(q4: torch.Tensor, p4: torch.Tensor, plist: PairList, dt: float,
                           r_cut: float, box, eps: float = 1.0, sigma: float = 1.0,
                           shifted: bool = False, out: torch.Tensor | None = None,
                           workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """p4 += impulses (FP64); returns a 2-element tensor (potential energy,
    pair virial sum r F(r))."""
    lib = load()
    n = plist.n
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=q4.device)
    if out.numel() < 2:
        raise ValueError("out must hold two doubles (energy, virial)")
    if workspace is None:
        workspace = _workspace(lib.lj_force_energy_workspace_bytes(n), q4.device)
    ep = _dev(out, torch.float64, "out")
    st = lib.lj_force_energy_virial(_dev(q4, torch.float64, "q4", (n, 4)),
                                    _dev(p4, torch.float64, "p4", (n, 4)), n,
                                    plist.row_ptr.data_ptr(), plist.col.data_ptr(), plist.nnz,
                                    int(plist.half), float(dt), float(r_cut), _box3(box),
                                    float(eps), float(sigma), int(bool(shifted)), ep, ep + 8,
                                    workspace.data_ptr(), workspace.numel(), _stream(stream))
    _check(st, "lj_force_energy_virial")
    return out


def lj_force_shifted_workspace_bytes(n: int) -> int:
    return int(load().lj_force_shifted_workspace_bytes(int(n)))


def lj_force_shifted(q4: torch.Tensor, p4: torch.Tensor, plist: PairList, dt: float,
                     r_cut: float, box, eps: float = 1.0, sigma: float = 1.0,
                     out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor | None:
    """p4 += impulses with the force-shifted truncation (FP64); if `out` (a
    1-element float64 device tensor) is given it receives the force-shifted
    potential energy.  Returns `out`."""
    lib = load()
    n = plist.n
    if workspace is None:
        workspace = _workspace(lib.lj_force_shifted_workspace_bytes(n), q4.device)
    st = lib.lj_force_shifted(_dev(q4, torch.float64, "q4", (n, 4)),
                              _dev(p4, torch.float64, "p4", (n, 4)), n, plist.row_ptr.data_ptr(),
                              plist.col.data_ptr(), plist.nnz, int(plist.half), float(dt),
                              float(r_cut), _box3(box), float(eps), float(sigma),
                              _dev(out, torch.float64, "out") if out is not None else None,
                              workspace.data_ptr(), workspace.numel(), _stream(stream))
    _check(st, "lj_force_shifted")
    return out


# ---- remaining entry points, same names, argument marshalling only --------

def lj_status_string(status: int) -> str:
    return load().lj_status_string(int(status)).decode()


def lj_last_cuda_error() -> str:
    return load().lj_last_cuda_error().decode()


def lj_version() -> int:
    return int(load().lj_version())


def lj_kernel_launch_count() -> int:
    return int(load().lj_kernel_launch_count())


def lj_batch_plan_bytes(systems, rows_per_item: int) -> int:
    """systems: a ctypes array of LjSystem."""
    return int(load().lj_batch_plan_bytes(systems, len(systems), int(rows_per_item)))


def lj_batch_init(batch: LjBatch, systems, dt: float, precision: int, tpi: int,
                  rows_per_item: int, plan: torch.Tensor, stream=None) -> LjBatch:
    _check(load().lj_batch_init(ctypes.byref(batch), systems, len(systems), float(dt),
                                int(precision), int(tpi), int(rows_per_item), plan.data_ptr(),
                                plan.numel(), _stream(stream)), "lj_batch_init")
    return batch


def lj_force_batched_workspace_bytes(batch: LjBatch) -> int:
    return int(load().lj_force_batched_workspace_bytes(ctypes.byref(batch)))


def lj_force_batched(batch: LjBatch, q4: torch.Tensor, p4: torch.Tensor, row_ptr: torch.Tensor,
                     col: torch.Tensor, workspace: torch.Tensor, stream=None) -> torch.Tensor:
    _check(load().lj_force_batched(ctypes.byref(batch), q4.data_ptr(), p4.data_ptr(),
                                   row_ptr.data_ptr(), col.data_ptr(), workspace.data_ptr(),
                                   workspace.numel(), _stream(stream)), "lj_force_batched")
    return p4


def lj_autotune_batched(systems, dt: float, precision: int, tpis, rows_per_item,
                        q4: torch.Tensor, p4_scratch: torch.Tensor, row_ptr: torch.Tensor,
                        col: torch.Tensor, plan: torch.Tensor, workspace: torch.Tensor,
                        reps: int = 5, stream=None):
    """Returns (best_tpi, best_rows_per_item, best_ms)."""
    ta = (ctypes.c_int * len(tpis))(*tpis)
    ra = (ctypes.c_int * len(rows_per_item))(*rows_per_item)
    bt, br, bm = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_float(0)
    _check(load().lj_autotune_batched(systems, len(systems), float(dt), int(precision), ta,
                                      len(tpis), ra, len(rows_per_item), q4.data_ptr(),
                                      p4_scratch.data_ptr(), row_ptr.data_ptr(), col.data_ptr(),
                                      plan.data_ptr(), plan.numel(), workspace.data_ptr(),
                                      workspace.numel(), int(reps), ctypes.byref(bt),
                                      ctypes.byref(br), ctypes.byref(bm), _stream(stream)),
           "lj_autotune_batched")
    return bt.value, br.value, bm.value


def lj_measure_peak(kind: int, work: int, buf: torch.Tensor | None = None, stream=None):
    """One timed run of the ceiling probe ``kind`` (LJ_PEAK_*); returns
    (rate, ms): flop/s for the FMA kinds, bytes/s for LJ_PEAK_L2_READ (which
    reads ``buf``, a CUDA byte tensor)."""
    lib = load()
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    bp = buf.data_ptr() if buf is not None else None
    nb = buf.numel() * buf.element_size() if buf is not None else 0
    st = lib.lj_measure_peak(int(kind), bp, nb, int(work), ctypes.byref(rate), ctypes.byref(ms),
                             _stream(stream))
    _check(st, "lj_measure_peak")
    return float(rate.value), float(ms.value)


def lj_eval_reciprocal(kind: int, a: torch.Tensor, stream=None):
    """Evaluate the reciprocal approximation ``kind`` (LJ_RCP_*, LJ_RSQRT_FP64)
    on the float64 CUDA tensor ``a``; returns (out (n, 2) float64: value or
    double-float head, and tail; ok (n,) uint8: 1 inside the function's
    range)."""
    lib = load()
    n = int(a.numel())
    ap = _dev(a, torch.float64, "a")
    out = torch.empty((n, 2), dtype=torch.float64, device=a.device)
    ok = torch.empty(n, dtype=torch.uint8, device=a.device)
    st = lib.lj_eval_reciprocal(int(kind), ap, n, out.data_ptr(), ok.data_ptr(), _stream(stream))
    _check(st, "lj_eval_reciprocal")
    return out, ok
