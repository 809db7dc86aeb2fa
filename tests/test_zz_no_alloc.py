"""The allocation-free pair-list builder, lj_build_pairlist_static.

It exists for callers that cannot allocate device memory (no cudaMalloc in
their context, no workspace handed to them): its scratch is a fixed array in
the library's device memory.  It must produce exactly the list of the
regular entry point, lj_build_pairlist, call after call -- the shared array
keeps the previous call's contents, so a second call on a different system
checks that everything that must start at zero is cleared.  Both calls (the
paper-size system of 119,164 atoms, then the 4,000-atom one) go through the
builder's two-walk path, count -> scan -> fill, the only path this entry
point takes; the regular builder it is compared with takes its one-walk
path, so the two routes check each other.  This file sorts last so that a
run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1806_05713_gb300 import inputs

pytestmark = pytest.mark.gpu


def _static_list(lj, q, box, rs, half, cap):
    n = q.shape[0]
    row_ptr = torch.full((n + 1,), -7, dtype=torch.int32, device="cuda")
    col = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    nnz = ctypes.c_int64(-1)
    mrow = ctypes.c_int64(-1)
    st = lj.load().lj_build_pairlist_static(
        q.data_ptr(), n, lj._box3(box), float(rs), int(half), row_ptr.data_ptr(), col.data_ptr(),
        cap, ctypes.byref(nnz), ctypes.byref(mrow), torch.cuda.current_stream().cuda_stream)
    assert st == lj.LJ_OK, lj.load().lj_status_string(st)
    torch.cuda.synchronize()
    return row_ptr.cpu().numpy(), col[: nnz.value].cpu().numpy(), int(mrow.value)


@pytest.mark.parametrize("half", [True, False])
def test_static_builder_matches_regular_builder_twice(cuda_lib, half):
    lj = cuda_lib
    systems = [inputs.workload_paper(order="random"), inputs.workload_small(order="cell")]
    for s in systems:   # two calls in a row, the second on a smaller system
        q = torch.from_numpy(s.q).cuda()
        ref = lj.lj_build_pairlist(q, s.box, s.rs, half)
        torch.cuda.synchronize()
        rp, col, mrow = _static_list(lj, q, s.box, s.rs, half, ref.nnz + 16)
        assert np.array_equal(rp, ref.row_ptr.cpu().numpy())
        assert np.array_equal(col, ref.col_view.cpu().numpy())
        assert mrow == ref.max_row


def test_static_builder_rejects_too_many_atoms(cuda_lib):
    lj = cuda_lib
    n = lj.LJ_STATIC_MAX_ATOMS + 1
    nnz, mrow = ctypes.c_int64(), ctypes.c_int64()
    st = lj.load().lj_build_pairlist_static(ctypes.c_void_p(256), n, lj._box3([100.0] * 3), 3.3,
                                            1, ctypes.c_void_p(256), ctypes.c_void_p(256), 0,
                                            ctypes.byref(nnz), ctypes.byref(mrow), None)
    assert st == lj.LJ_ERR_CAPACITY
