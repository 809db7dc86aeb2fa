"""Batched persistent launch (lj_force_batched) vs the oracle per system,
vs per-system launches, under CUDA-graph replay, and after autotuning."""
import numpy as np
import pytest
import torch

from paper_1806_05713_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-5


def _oracle_dp(oracle_lib, s, dt, half):
    rp, col = oracle_lib.pairlist(s.q, s.box, s.rs, half)
    return oracle_lib.force(s.q, np.zeros((s.n, 3)), rp, col, half, dt, s.rc, s.box)


def _per_system(b, p):
    out = p.cpu().numpy()
    return [out[int(o):int(o) + s.n, :3] for o, s in zip(b.atom_offset, b.systems)]


@pytest.fixture(scope="module")
def systems():
    return inputs.batched_systems(nsys=24, seed=5, n_min=500, n_max=6000)


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL), (2, FP64_TOL)])
@pytest.mark.parametrize("half", [True, False])
def test_batched_matches_oracle_per_system(cuda_lib, oracle_lib, systems, precision, tol, half):
    from paper_1806_05713_gb300.batch import Batch
    b = Batch(systems, 0.01, precision, half, tpi=8, rows_per_item=32)
    b.force()
    torch.cuda.synchronize()
    for s, got in zip(systems, _per_system(b, b.p4)):
        want = _oracle_dp(oracle_lib, s, 0.01, half)
        assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


@pytest.mark.parametrize("half", [True, False])
@pytest.mark.parametrize("rows", [8, 64])
def test_batched_stream_walk_matches_oracle(cuda_lib, oracle_lib, systems, half, rows):
    """FP64 batch with each work item's rows walked as one stream of entries
    (tpi = LJ_SCHED_STREAM) against the oracle, per system."""
    from paper_1806_05713_gb300.batch import Batch
    lj = cuda_lib
    b = Batch(systems, 0.01, lj.LJ_FP64, half, tpi=lj.LJ_SCHED_STREAM, rows_per_item=rows,
              plan_rows_min=8)
    b.force()
    torch.cuda.synchronize()
    for s, got in zip(systems, _per_system(b, b.p4)):
        want = _oracle_dp(oracle_lib, s, 0.01, half)
        assert np.max(np.abs(got - want)) <= FP64_TOL * np.max(np.abs(want))


def test_batched_stream_walk_refused_for_other_forms(cuda_lib, systems):
    from paper_1806_05713_gb300.batch import Batch
    lj = cuda_lib
    for prec in (lj.LJ_MIXED, lj.LJ_DFLOAT):
        with pytest.raises(lj.LJError):
            Batch(systems, 0.01, prec, True, tpi=lj.LJ_SCHED_STREAM, rows_per_item=16)


def test_batched_equals_per_system_launches_full_list(cuda_lib, systems):
    """Full lists are deterministic: the persistent launch gives the same bits
    as one lj_force call per system with the same row arithmetic (8 lanes
    per row, exact fixed-point displacement)."""
    from paper_1806_05713_gb300.batch import Batch
    b = Batch(systems, 0.01, 0, False, tpi=8, rows_per_item=16)
    p_a = torch.zeros_like(b.p4)
    p_b = torch.zeros_like(b.p4)
    b.force(p_a)
    b.force_per_system(p_b, tpi=cuda_lib.LJ_SCHED_FIXED | 8)
    torch.cuda.synchronize()
    assert torch.equal(p_a, p_b)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_graph_replay(cuda_lib, systems, precision):
    from paper_1806_05713_gb300.batch import Batch
    b = Batch(systems, 0.01, precision, False, tpi=4, rows_per_item=64)
    once = torch.zeros_like(b.p4)
    b.force(once)
    p = torch.zeros_like(b.p4)
    g = b.capture_graph(p)   # capture runs no kernels; the warm-up call adds one update
    torch.cuda.synchronize()
    p.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert torch.allclose(p, 2 * once, rtol=0, atol=1e-14 * float(once.abs().max()))


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_per_system_graph_equals_per_system_calls(cuda_lib, systems, precision):
    """The CUDA graph of the per-system lj_force calls replays exactly the
    calls it captured: on full lists (deterministic) its update is
    bit-identical to the same calls issued from the host."""
    from paper_1806_05713_gb300.batch import Batch
    b = Batch(systems, 0.01, precision, False, tpi=8, rows_per_item=32)
    direct = torch.zeros_like(b.p4)
    b.force_per_system(direct)
    p = torch.zeros_like(b.p4)
    g = b.capture_per_system_graph(p)
    torch.cuda.synchronize()
    p.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(p, direct)


def test_batched_dfloat_equals_per_system_launches_full_list(cuda_lib, systems):
    """The double-float row walk is the same in the persistent launch and in
    lj_force (two entries per lane, 8 lanes per row): same bits."""
    from paper_1806_05713_gb300.batch import Batch
    b = Batch(systems, 0.01, 2, False, tpi=8, rows_per_item=16)
    p_a = torch.zeros_like(b.p4)
    p_b = torch.zeros_like(b.p4)
    b.force(p_a)
    b.force_per_system(p_b, tpi=cuda_lib.LJ_SCHED_SWP2 | 8)
    torch.cuda.synchronize()
    assert torch.equal(p_a, p_b)


def test_batched_dfloat_noncubic_boxes(cuda_lib, oracle_lib):
    """Systems in stretched boxes take the per-axis scaled displacement."""
    from paper_1806_05713_gb300.batch import Batch
    systems = inputs.batched_systems(nsys=6, seed=8, n_min=500, n_max=3000)
    for k, s in enumerate(systems):
        if k % 2:
            st = np.array([1.0, 1.15, 1.3])
            s.q[:, :3] *= st
            s.box = s.box * st
    for half in (True, False):
        b = Batch(systems, 0.01, 2, half, tpi=8, rows_per_item=32)
        assert b.c_batch.flags == 0
        b.force()
        torch.cuda.synchronize()
        for s, got in zip(systems, _per_system(b, b.p4)):
            want = _oracle_dp(oracle_lib, s, 0.01, half)
            assert np.max(np.abs(got - want)) <= FP64_TOL * np.max(np.abs(want))


def test_autotune_picks_a_valid_schedule(cuda_lib, oracle_lib, systems):
    from paper_1806_05713_gb300.batch import Batch
    b = Batch(systems, 0.01, 0, True, tpi=8, rows_per_item=64, plan_rows_min=16)
    tpi, rows, ms = b.autotune(tpis=(4, 8, 16), rows=(16, 64), reps=3)
    assert tpi in (4, 8, 16) and rows in (16, 64) and 0 < ms < 1e3
    b.p4.zero_()
    b.force()
    torch.cuda.synchronize()
    s = systems[3]
    got = _per_system(b, b.p4)[3]
    want = _oracle_dp(oracle_lib, s, 0.01, True)
    assert np.max(np.abs(got - want)) <= FP64_TOL * np.max(np.abs(want))


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_autotune_picks_the_list_layout(cuda_lib, oracle_lib, systems, precision):
    """With both layouts offered the tuner times the half list (p_j atomics)
    and the full list and keeps the faster; the batch then gives the
    oracle's momenta with the kept layout."""
    from paper_1806_05713_gb300.batch import Batch
    b = Batch(systems, 0.01, precision, True, tpi=8, rows_per_item=64, plan_rows_min=16)
    tpi, rows, ms = b.autotune(tpis=(4, 8), rows=(16, 64), reps=2, layouts=(True, False))
    assert tpi in (4, 8) and rows in (16, 64) and 0 < ms < 1e3
    assert b.pairs == (int(b.nnz.sum()) if b.half else int(b.nnz.sum()) // 2)
    b.p4.zero_()
    b.force()
    torch.cuda.synchronize()
    tol = FP64_TOL if precision != 1 else MIXED_TOL
    for k in (0, 3):
        got = _per_system(b, b.p4)[k]
        want = _oracle_dp(oracle_lib, systems[k], 0.01, True)
        assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


def test_autotune_force_single_system(cuda_lib):
    lj = cuda_lib
    s = inputs.workload_small()
    q = torch.from_numpy(s.q).cuda()
    pl = lj.lj_build_pairlist(q, s.box, s.rs, True)
    best, ms, table = lj.lj_autotune_force(q, pl, 0.01, s.rc, s.box, reps=3)
    assert best in table and ms == min(table.values()) and np.isfinite(ms)


@pytest.mark.slow
def test_full_batch_sampled_systems(cuda_lib, oracle_lib):
    """512 systems (N log-uniform 500..32000): the bench's batch, checked on
    sampled systems against the oracle."""
    from paper_1806_05713_gb300.batch import Batch
    lj = cuda_lib
    systems = inputs.batched_systems(nsys=512, seed=0)
    want = {k: _oracle_dp(oracle_lib, systems[k], 0.01, True) for k in (0, 1, 97, 255, 300, 511)}
    # 8 lanes per row, and the autotuner's pick there: 64-row items walked in
    # per-lane chunks (lj_batch.tpi = LJ_SCHED_STREAM)
    for tpi in (8, lj.LJ_SCHED_STREAM):
        b = Batch(systems, 0.01, 0, True, tpi=tpi, rows_per_item=64)
        b.force()
        torch.cuda.synchronize()
        got = _per_system(b, b.p4)
        for k, w in want.items():
            assert np.max(np.abs(got[k] - w)) <= FP64_TOL * np.max(np.abs(w)), (tpi, k)
