"""Many independent LJ systems in one persistent launch (``lj_force_batched``).

``Batch`` lays the systems out in packed device arrays (positions and
momenta AoS4, one CSR list per system at its own offsets), builds every
system's list in place with ``lj_build_pairlist``, writes the device plan
with ``lj_batch_init``, and runs the force for all systems with one
``lj_force_batched`` call -- which can be captured once in a CUDA graph and
replayed.  ``autotune`` picks lanes-per-row and rows-per-work-item with the
library's ``lj_autotune_batched``.  Host-side orchestration only: every
step of the computation runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import lj


class Batch:
    def __init__(self, systems, dt: float, precision: int = lj.LJ_FP64, half: bool = True,
                 tpi: int = 8, rows_per_item: int = 64, eps: float = 1.0, sigma: float = 1.0,
                 device="cuda", plan_rows_min: int = 8):
        lib = lj.load()
        self.lib = lib
        self.dt, self.precision, self.half = float(dt), int(precision), bool(half)
        self.device = torch.device(device)
        self.systems = list(systems)
        nsys = len(self.systems)
        ns = [s.n for s in self.systems]
        self.atom_offset = np.concatenate([[0], np.cumsum(ns)[:-1]]).astype(np.int64)
        self.row_offset = self.atom_offset + np.arange(nsys, dtype=np.int64)
        total = int(sum(ns))
        self.total_atoms = total
        q = np.concatenate([s.q for s in self.systems], axis=0)
        self.q4 = torch.from_numpy(q).to(self.device)
        self.p4 = torch.zeros((total, 4), dtype=torch.float64, device=self.device)
        self.row_ptr = torch.empty(total + nsys, dtype=torch.int32, device=self.device)
        ws_bytes = max(lib.lj_pairlist_workspace_bytes(s.n, lj._box3(s.box), s.rs) for s in self.systems)
        self.list_ws = lj._workspace(ws_bytes, self.device)
        self.eps, self.sigma = float(eps), float(sigma)
        self.plan_rows_min = int(plan_rows_min)
        self._build_lists(self.half)
        self.c_batch = lj.LjBatch()
        self.init(tpi, rows_per_item)

    def _build_lists(self, half: bool):
        """Every system's list (half or full) in place, and the host
        descriptors and device plan for it."""
        lib, st, nsys = self.lib, lj._stream(None), len(self.systems)
        self.half = bool(half)
        # pass 1: list sizes (capacity 0 reports the size needed)
        nnz = np.zeros(nsys, dtype=np.int64)
        qbase, rbase = self.q4.data_ptr(), self.row_ptr.data_ptr()
        for k, s in enumerate(self.systems):
            c = ctypes.c_int64(0)
            code = lib.lj_build_pairlist(qbase + 32 * int(self.atom_offset[k]), s.n, lj._box3(s.box),
                                         float(s.rs), int(half), rbase + 4 * int(self.row_offset[k]),
                                         None, 0, self.list_ws.data_ptr(), self.list_ws.numel(),
                                         ctypes.byref(c), None, st)
            if code not in (lj.LJ_OK, lj.LJ_ERR_CAPACITY):
                lj._check(code, "lj_build_pairlist")
            nnz[k] = c.value
        self.nnz = nnz
        self.entry_offset = np.concatenate([[0], np.cumsum(nnz)[:-1]]).astype(np.int64)
        self.col = torch.empty(max(1, int(nnz.sum())), dtype=torch.int32, device=self.device)
        cbase = self.col.data_ptr()
        # pass 2: fill each list at its offsets
        for k, s in enumerate(self.systems):
            c = ctypes.c_int64(0)
            lj._check(lib.lj_build_pairlist(qbase + 32 * int(self.atom_offset[k]), s.n,
                                            lj._box3(s.box), float(s.rs), int(half),
                                            rbase + 4 * int(self.row_offset[k]),
                                            cbase + 4 * int(self.entry_offset[k]), int(nnz[k]),
                                            self.list_ws.data_ptr(), self.list_ws.numel(),
                                            ctypes.byref(c), None, st), "lj_build_pairlist")
        self.c_systems = (lj.LjSystem * nsys)()
        for k, s in enumerate(self.systems):
            y = self.c_systems[k]
            y.atom_offset, y.n = int(self.atom_offset[k]), int(s.n)
            y.row_offset, y.entry_offset, y.nnz = int(self.row_offset[k]), int(self.entry_offset[k]), int(nnz[k])
            for a in range(3):
                y.box[a] = float(s.box[a])
            y.r_cut, y.eps, y.sigma, y.half = float(s.rc), self.eps, self.sigma, int(half)
        self.plan = lj._workspace(lib.lj_batch_plan_bytes(self.c_systems, nsys, self.plan_rows_min),
                                  self.device)

    @property
    def pairs(self) -> int:
        """Unique pairs per call (half-list entries)."""
        return int(self.nnz.sum()) if self.half else int(self.nnz.sum()) // 2

    def init(self, tpi: int, rows_per_item: int):
        if rows_per_item < self.plan_rows_min:
            raise ValueError("rows_per_item below the plan size this batch was created with")
        lj._check(self.lib.lj_batch_init(ctypes.byref(self.c_batch), self.c_systems, len(self.systems),
                                         self.dt, self.precision, int(tpi), int(rows_per_item),
                                         self.plan.data_ptr(), self.plan.numel(), lj._stream(None)),
                  "lj_batch_init")
        need = self.lib.lj_force_batched_workspace_bytes(ctypes.byref(self.c_batch))
        if getattr(self, "ws", None) is None or self.ws.numel() < need:
            self.ws = lj._workspace(need, self.device)

    def force(self, p4: torch.Tensor | None = None, stream=None):
        """p += impulses for every system (one persistent launch)."""
        p4 = self.p4 if p4 is None else p4
        lj._check(self.lib.lj_force_batched(ctypes.byref(self.c_batch), self.q4.data_ptr(),
                                            lj._dev(p4, torch.float64, "p4", (self.total_atoms, 4)),
                                            self.row_ptr.data_ptr(), self.col.data_ptr(),
                                            self.ws.data_ptr(), self.ws.numel(), lj._stream(stream)),
                  "lj_force_batched")
        return p4

    def force_per_system(self, p4: torch.Tensor | None = None, tpi: int = lj.LJ_TPI_AUTO,
                         stream=None):
        """The same update as separate lj_force calls, one per system."""
        p4 = self.p4 if p4 is None else p4
        ws = getattr(self, "_ws1", None)
        need = max(self.lib.lj_force_workspace_bytes(s.n, lj._box3(s.box), self.precision)
                   for s in self.systems)
        if ws is None or ws.numel() < need:
            ws = self._ws1 = lj._workspace(need, self.device)
        st = lj._stream(stream)
        for k, s in enumerate(self.systems):
            lj._check(self.lib.lj_force(self.q4.data_ptr() + 32 * int(self.atom_offset[k]),
                                        p4.data_ptr() + 32 * int(self.atom_offset[k]), s.n,
                                        self.row_ptr.data_ptr() + 4 * int(self.row_offset[k]),
                                        self.col.data_ptr() + 4 * int(self.entry_offset[k]),
                                        int(self.nnz[k]), int(self.half), self.dt, float(s.rc),
                                        lj._box3(s.box), self.c_systems[k].eps,
                                        self.c_systems[k].sigma, self.precision, int(tpi),
                                        ws.data_ptr(), ws.numel(), st), "lj_force")
        return p4

    def capture_graph(self, p4: torch.Tensor | None = None) -> torch.cuda.CUDAGraph:
        """A CUDA graph of one batched force call (replay with .replay())."""
        p4 = self.p4 if p4 is None else p4
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self.force(p4)  # warm-up outside capture
        torch.cuda.current_stream(self.device).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.force(p4)
        return g

    def capture_per_system_graph(self, p4: torch.Tensor | None = None,
                                 tpi: int = lj.LJ_TPI_AUTO) -> torch.cuda.CUDAGraph:
        """A CUDA graph of the per-system calls (force_per_system): replaying
        it issues the same kernels as the separate lj_force calls with no
        host work between them, so its time against the persistent launch's
        is the GPU-side difference of the two ways of running the batch."""
        p4 = self.p4 if p4 is None else p4
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self.force_per_system(p4, tpi=tpi)  # sizes the workspace outside capture
        torch.cuda.current_stream(self.device).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.force_per_system(p4, tpi=tpi)
        return g

    def autotune(self, tpis=None, rows=(16, 32, 64, 128), reps: int = 5, layouts=None):
        """Pick lanes-per-row and rows-per-item -- and, with layouts=(True,
        False), the list layout (half list with p_j atomics, or full list
        without) -- by timing; applies them and returns (tpi, rows, ms)."""
        layouts = (self.half,) if layouts is None else tuple(bool(h) for h in layouts)
        best = None
        for half in layouts:
            if half != self.half:
                self._build_lists(half)
                self.init(self.c_batch.tpi, self.c_batch.rows_per_item)
            t, r, ms = self._autotune_layout(tpis, rows, reps)
            if best is None or ms < best[3]:
                best = (half, t, r, ms)
        if best[0] != self.half:
            self._build_lists(best[0])
        self.init(best[1], best[2])
        return best[1], best[2], best[3]

    def _autotune_layout(self, tpis, rows, reps):
        if tpis is None:
            tpis = ((4, 8, 16) if self.precision == lj.LJ_DFLOAT else
                    (2, 4, 8, 16, lj.LJ_SCHED_STREAM) if self.precision == lj.LJ_FP64 else
                    (2, 4, 8, 16))
        scratch = torch.zeros_like(self.p4)
        ta = (ctypes.c_int * len(tpis))(*tpis)
        ra = (ctypes.c_int * len(rows))(*rows)
        bt, br, bm = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_float(0)
        lj._check(self.lib.lj_autotune_batched(self.c_systems, len(self.systems), self.dt,
                                               self.precision, ta, len(tpis), ra, len(rows),
                                               self.q4.data_ptr(), scratch.data_ptr(),
                                               self.row_ptr.data_ptr(), self.col.data_ptr(),
                                               self.plan.data_ptr(), self.plan.numel(),
                                               self.ws.data_ptr(), self.ws.numel(), int(reps),
                                               ctypes.byref(bt), ctypes.byref(br), ctypes.byref(bm),
                                               lj._stream(None)), "lj_autotune_batched")
        return bt.value, br.value, bm.value
