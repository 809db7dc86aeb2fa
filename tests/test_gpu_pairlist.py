"""GPU pair list vs the oracle: bit-exact CSR (row_ptr and sorted col)."""
import math

import numpy as np
import pytest
import torch

from paper_1806_05713_gb300 import inputs
from conftest import to_dev

pytestmark = pytest.mark.gpu


def _gpu_list(lj, q, box, rs, half, **kw):
    pl = lj.lj_build_pairlist(to_dev(q), box, rs, half, **kw)
    torch.cuda.synchronize()
    return pl.row_ptr.cpu().numpy(), pl.col_view.cpu().numpy(), pl


def _assert_same(lj, oracle_lib, q, box, rs, half, method="cells"):
    rp, col, pl = _gpu_list(lj, q, box, rs, half)
    orp, ocol = oracle_lib.pairlist(q, box, rs, half, method)
    assert pl.nnz == ocol.size
    assert np.array_equal(rp, orp)
    assert np.array_equal(col, ocol)
    return pl


@pytest.mark.parametrize("order", ["random", "cell", "lattice"])
@pytest.mark.parametrize("half", [True, False])
def test_small_fcc_bit_exact(cuda_lib, oracle_lib, order, half):
    s = inputs.workload_small(order=order)
    pl = _assert_same(cuda_lib, oracle_lib, s.q, s.box, s.rs, half)
    assert pl.max_row > 0


@pytest.mark.parametrize("k,rho,rs", [(3, 1.0, 2.2), (4, 0.8, 2.6), (5, 1.0, 3.3), (6, 1.2, 1.3),
                                      (7, 1.0, 1.1)])
@pytest.mark.parametrize("half", [True, False])
def test_degenerate_cell_grids_bit_exact(cuda_lib, oracle_lib, k, rho, rs, half):
    s = inputs.fcc_system(k, rho, 0.07, seed=11 + k)
    rs = min(rs, 0.5 * s.box[0])
    _assert_same(cuda_lib, oracle_lib, s.q, s.box, rs, half, "brute")


def test_nonuniform_box_and_uniform_gas(cuda_lib, oracle_lib):
    rng = np.random.default_rng(3)
    box = np.array([6.7, 9.1, 13.4])
    q = np.zeros((700, 4))
    q[:, :3] = rng.random((700, 3)) * box
    for half in (True, False):
        _assert_same(cuda_lib, oracle_lib, q, box, 3.3, half, "brute")


@pytest.mark.parametrize("box", [(9.9, 11.55, 14.85), (8.3, 8.3, 21.0), (16.6, 8.4, 8.5)])
def test_forward_stencil_noncubic_boxes(cuda_lib, oracle_lib, box):
    """Boxes with five or more cells on every axis (the forward-stencil
    walk), with five exactly on some axes and unequal sides, against brute
    force, half and full lists."""
    rng = np.random.default_rng(int(sum(box) * 10))
    box = np.array(box)
    n = int(0.9 * np.prod(box))
    q = np.zeros((n, 4))
    q[:, :3] = rng.random((n, 3)) * box
    for half in (True, False):
        _assert_same(cuda_lib, oracle_lib, q, box, 3.3, half, "brute")


def test_atoms_on_cell_and_box_faces(cuda_lib, oracle_lib):
    """Positions exactly on cell boundaries, at 0 and just below L."""
    L = 13.2  # 4 cells of exactly r_s = 3.3
    g = np.array([0.0, 3.3, 6.6, 9.9, np.nextafter(L, 0.0), 1.65, 4.95])
    xs, ys, zs = np.meshgrid(g, g, g, indexing="ij")
    q = np.zeros((xs.size, 4))
    q[:, 0], q[:, 1], q[:, 2] = xs.ravel(), ys.ravel(), zs.ravel()
    box = np.array([L, L, L])
    for half in (True, False):
        _assert_same(cuda_lib, oracle_lib, q, box, 3.3, half, "brute")


def test_exact_ties_at_search_length(cuda_lib, oracle_lib):
    """Pairs at exactly r_s are excluded on both sides (strict '<')."""
    q = np.zeros((4, 4))
    q[0, :3] = [1.0, 1.0, 1.0]
    q[1, :3] = [1.0 + 3.25, 1.0, 1.0]     # r_s = 3.25 exactly representable
    q[2, :3] = [1.0, 1.0 + 3.0, 1.0]
    q[3, :3] = [1.0, 1.0, 1.0 + np.nextafter(3.25, 0.0)]
    box = np.array([20.0, 20.0, 20.0])
    rp, col, pl = _gpu_list(cuda_lib, q, box, 3.25, False)
    orp, ocol = oracle_lib.pairlist(q, box, 3.25, False, "brute")
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    assert 1 not in col[rp[0]:rp[1]]


def test_tiny_and_empty_systems(cuda_lib, oracle_lib):
    lj = cuda_lib
    box = np.array([10.0, 10.0, 10.0])
    for n in (0, 1, 2):
        q = np.zeros((n, 4))
        q[:, :3] = np.array([[1.0, 1.0, 1.0], [2.0, 1.0, 1.0]])[:n]
        rp, col, pl = _gpu_list(lj, q, box, 3.3, True)
        orp, ocol = oracle_lib.pairlist(q, box, 3.3, True, "brute")
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol)


def test_isolated_atoms_give_empty_rows(cuda_lib):
    q = np.zeros((3, 4))
    q[:, :3] = [[1, 1, 1], [8, 8, 8], [15, 15, 15]]
    rp, col, pl = _gpu_list(cuda_lib, q, np.array([24.0] * 3), 3.3, False)
    assert pl.nnz == 0 and np.all(rp == 0)


@pytest.mark.parametrize("half", [True, False])
def test_dense_cluster_overflows_the_row_slabs(cuda_lib, oracle_lib, half):
    """A gas with a dense cluster: the cluster's rows exceed the one-walk
    builder's slab (sized from the mean density), so the build finishes with
    the two-walk path; the list is still the oracle's."""
    rng = np.random.default_rng(9)
    box = np.array([15.0, 15.0, 15.0])
    gas = rng.random((1500, 3)) * box
    cluster = 7.0 + rng.random((600, 3)) * 2.2
    q = np.zeros((2100, 4))
    q[:, :3] = np.concatenate([gas, cluster])
    pl = _assert_same(cuda_lib, oracle_lib, q, box, 3.3, half)
    assert pl.max_row > 400


def test_errors(cuda_lib):
    lj = cuda_lib
    s = inputs.workload_small()
    q = to_dev(s.q)
    with pytest.raises(lj.LJError) as e:
        lj.lj_build_pairlist(q, [6.0, 6.0, 6.0], 3.3, True)
    assert e.value.status == lj.LJ_ERR_BOX
    bad = s.q.copy()
    bad[17, 1] = s.box[1] + 0.1
    with pytest.raises(lj.LJError) as e:
        lj.lj_build_pairlist(to_dev(bad), s.box, 3.3, True)
    assert e.value.status == lj.LJ_ERR_RANGE
    bad[17, 1] = float("nan")
    with pytest.raises(lj.LJError) as e:
        lj.lj_build_pairlist(to_dev(bad), s.box, 3.3, True)
    assert e.value.status == lj.LJ_ERR_RANGE


def test_capacity_retry(cuda_lib, oracle_lib):
    """A too-small column buffer reports the size needed; the binding regrows it."""
    s = inputs.workload_small()
    pl = cuda_lib.lj_build_pairlist(to_dev(s.q), s.box, 3.3, True, col_capacity=1000)
    orp, ocol = oracle_lib.pairlist(s.q, s.box, 3.3, True)
    assert pl.nnz == ocol.size
    assert np.array_equal(pl.col_view.cpu().numpy(), ocol)


@pytest.mark.parametrize("order", ["random", "cell"])
def test_paper_size_bit_exact(cuda_lib, oracle_lib, order):
    """N = 119,164 (the paper's benchmark size), the bench's half list."""
    s = inputs.workload_paper(order=order)
    _assert_same(cuda_lib, oracle_lib, s.q, s.box, s.rs, True)


@pytest.mark.slow
def test_million_atoms_bit_exact(cuda_lib, oracle_lib):
    s = inputs.workload_million()
    pl = _assert_same(cuda_lib, oracle_lib, s.q, s.box, s.rs, True)
    mean = pl.nnz / s.n
    assert abs(mean - 0.5 * 4 / 3 * math.pi * 3.3 ** 3) < 6


def test_build_on_a_side_stream_then_force_on_it(cuda_lib, oracle_lib):
    """The builder returns before its row sort ends; on the caller's own
    (non-default) stream the list is complete in stream order: a force call
    queued right behind it on that stream sees the finished list."""
    lj = cuda_lib
    s = inputs.workload_paper(order="random")
    q = to_dev(s.q)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        pl = lj.lj_build_pairlist(q, s.box, s.rs, True, stream=side)
        p = torch.zeros_like(q)
        lj.lj_force(q, p, pl, 0.01, s.rc, s.box, stream=side)
        rp_dev = pl.row_ptr.clone()
        col_dev = pl.col_view.clone()
    side.synchronize()
    orp, ocol = oracle_lib.pairlist(s.q, s.box, s.rs, True)
    assert np.array_equal(rp_dev.cpu().numpy(), orp)
    assert np.array_equal(col_dev.cpu().numpy(), ocol)
    ref = torch.zeros_like(q)
    lj.lj_force(q, ref, lj.lj_build_pairlist(q, s.box, s.rs, True), 0.01, s.rc, s.box)
    torch.cuda.synchronize()
    assert float((p - ref).abs().max()) <= 1e-13 * float(ref.abs().max())
