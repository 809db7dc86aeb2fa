"""GPU force kernels vs the oracle (Algorithm 3 with Algorithm 1).

FP64: every schedule, half and full lists, within 1e-12 of max|dp|.
MIXED: within the stated error bound (max |dp error| <= 1e-5 max|dp|, RMS <= 2.5e-6)."""
import numpy as np
import pytest
import torch

from paper_1806_05713_gb300 import inputs
from conftest import to_dev

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-5
SCHEDULES = [1, 2, 4, 8, 16, 32, 132, 136, 144, 520, 644, 648, 656, 1028, 1032, 1040, 1156, 1160,
             1168, 1544, 1672, 2052, 2056, 2064, 2568, 10244, 10248, 10256, 10272, 17416, 18440]
# t lanes per row; 128|t two entries per lane (software-pipelined); 512|...
# length-sorted rows; 1024|... image-selected displacement; 2048|... exact
# fixed-point displacement (the default); 8192|2048|r the fixed-point rows,
# r rows per warp cut into one chunk of entries per lane; 16384|... rows in
# space-filling (cell) order


def _run(lj, s, half, precision, tpi, dt=0.01, eps=1.0, sigma=1.0, p0=None, rc=None, pl=None):
    rc = s.rc if rc is None else rc
    q = to_dev(s.q)
    if pl is None:
        pl = lj.lj_build_pairlist(q, s.box, s.rs, half)
    p = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda") if p0 is None else to_dev(p0)
    lj.lj_force(q, p, pl, dt, rc, s.box, eps, sigma, precision, tpi)
    torch.cuda.synchronize()
    return p.cpu().numpy()[:, :3], pl


def _oracle(oracle_lib, s, half, dt=0.01, eps=1.0, sigma=1.0, p0=None, rc=None):
    rc = s.rc if rc is None else rc
    rp, col = oracle_lib.pairlist(s.q, s.box, s.rs, half)
    p = np.zeros((s.n, 3)) if p0 is None else p0[:, :3]
    return oracle_lib.force(s.q, p, rp, col, half, dt, rc, s.box, eps, sigma)


def _relerr(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.fixture(scope="module")
def small():
    return inputs.workload_small()


@pytest.mark.parametrize("tpi", SCHEDULES)
@pytest.mark.parametrize("half", [True, False])
def test_fp64_small_all_schedules(cuda_lib, oracle_lib, small, tpi, half):
    got, _ = _run(cuda_lib, small, half, cuda_lib.LJ_FP64, tpi)
    want = _oracle(oracle_lib, small, half)
    assert _relerr(got, want) <= FP64_TOL


@pytest.mark.parametrize("tpi", [1, 4, 8, 32, 516, 520, 132, 136, 144, 648, 16392, 16516, 16520])
@pytest.mark.parametrize("half", [True, False])
def test_mixed_small(cuda_lib, oracle_lib, small, tpi, half):
    got, _ = _run(cuda_lib, small, half, cuda_lib.LJ_MIXED, tpi)
    want = _oracle(oracle_lib, small, half)
    assert _relerr(got, want) <= MIXED_TOL


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_eps_sigma_dt_and_existing_momenta(cuda_lib, oracle_lib, precision, tol):
    s = inputs.fcc_system(8, 0.9, 0.05, seed=3)
    p0 = np.random.default_rng(2).normal(size=(s.n, 4))
    kw = dict(dt=0.005, eps=1.3, sigma=1.1, rc=3.0)
    for half in (True, False):
        for tpi in ((8, 136, 1160, 2056, 2568) if precision == 0 else (8,)):
            got, _ = _run(cuda_lib, s, half, precision, tpi, p0=p0, **kw)
            want = _oracle(oracle_lib, s, half, p0=p0, **kw)
            assert _relerr(got - p0[:, :3], want - p0[:, :3]) <= tol


@pytest.mark.parametrize("precision", [0, 1])
def test_two_body_closed_form(cuda_lib, precision):
    """r = 1: dp = -+ 24 dt along d; r = 2^(1/6): dp ~ 0 (Algorithm 1)."""
    lj = cuda_lib
    dt = 0.01
    for r, want in [(1.0, 24 * dt), (2.0 ** (1 / 6), 0.0)]:
        q = np.zeros((2, 4))
        q[:, :3] = 5.0
        q[1, 0] += r
        s = inputs.LJSystem(q=q, box=np.array([20.0] * 3), rho=0.0)
        for half in (True, False):
            for tpi in (1, 32) + ((2056, 10244, 10272) if precision == 0 else ()):
                got, _ = _run(lj, s, half, precision, tpi, dt=dt)
                tol = 1e-15 if precision == 0 else 1e-6
                assert abs(got[1, 0] - want) <= tol * 24 * dt + 1e-14 * 48 * dt
                assert abs(got[0, 0] + want) <= tol * 24 * dt + 1e-14 * 48 * dt
                assert np.all(got[:, 1:] == 0.0)


@pytest.mark.parametrize("half", [True, False])
def test_fp64_stream_sparse_rows(cuda_lib, oracle_lib, half):
    """A dilute gas (rho = 0.002, 1,000 atoms): most rows are empty and whole
    windows of 4-32 rows hold no entry, the last window is ragged (1,000 is
    no multiple of 32 or 16); the stream walks against the oracle."""
    lj = cuda_lib
    g = np.random.default_rng(31)
    n, L = 1000, (1000 / 0.002) ** (1 / 3)
    q = np.zeros((n, 4))
    q[:, :3] = g.uniform(0.0, L, size=(n, 3))
    s = inputs.LJSystem(q=q, box=np.array([L] * 3), rho=0.002)
    want = _oracle(oracle_lib, s, half)
    assert np.count_nonzero(np.any(want != 0.0, axis=1)) < n // 2
    for tpi in (10244, 10248, 10256, 10272, 2056):
        got, _ = _run(lj, s, half, 0, tpi)
        assert _relerr(got, want) <= FP64_TOL, tpi


@pytest.mark.parametrize("precision,tpi", [(0, 2056), (0, 1032), (1, 8), (1, 132), (2, 136)])
def test_cell_order_full_list_bitwise(cuda_lib, precision, tpi):
    """LJ_SCHED_CELLS only changes which warp walks which row: on a full list
    (each row's sum kept by its own group, no atomics) the momenta are
    bit-identical with and without it (N = 119,164, random order)."""
    lj = cuda_lib
    s = inputs.workload_paper()
    q = to_dev(s.q)
    pl = lj.lj_build_pairlist(q, s.box, s.rs, False)
    out = []
    for t in (tpi, lj.LJ_SCHED_CELLS | tpi):
        p = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
        lj.lj_force(q, p, pl, 0.01, s.rc, s.box, precision=precision, tpi=t)
        torch.cuda.synchronize()
        out.append(p.cpu().numpy())
    assert np.array_equal(out[0], out[1])


def test_wrap_across_boundary(cuda_lib):
    lj = cuda_lib
    q = np.zeros((2, 4))
    q[0, :3] = [0.3, 5.0, 5.0]
    q[1, :3] = [9.3, 5.0, 5.0]
    s = inputs.LJSystem(q=q, box=np.array([10.0] * 3), rho=0.0)
    for precision in (0, 1):
        for half in (True, False):
            got, _ = _run(lj, s, half, precision, 8)
            assert abs(got[0, 0] - 0.24) < 1e-6 and abs(got[1, 0] + 0.24) < 1e-6


def test_small_box_mixed_image_choice(cuda_lib, oracle_lib):
    """L = 6.8 (2-3 cells): the mixed form picks the minimum image."""
    s = inputs.fcc_system(4, 0.8, 0.1, seed=9)   # L = 6.84
    s.rc, s.margin = 3.0, 0.3
    for half in (True, False):
        got, _ = _run(cuda_lib, s, half, 1, 8)
        want = _oracle(oracle_lib, s, half)
        assert _relerr(got, want) <= MIXED_TOL


@pytest.mark.parametrize("tpi", [1032, 2056, 2568, 10248])
def test_fp64_pairs_on_the_cutoff(cuda_lib, oracle_lib, tpi):
    """Pairs at r_c and one ulp either side, along an axis and a diagonal:
    the FP64 schedules interact exactly the oracle's pairs."""
    xs = []
    for k, d in enumerate([3.0, np.nextafter(3.0, 0.0), np.nextafter(3.0, 4.0),
                           3.0 - 1e-15, 3.0 + 2e-15, 3.0 - 1e-12]):
        y = 2.0 + 4.0 * k
        xs += [[10.0, y, 5.0], [10.0 + d, y, 5.0]]
    h = 3.0 / np.sqrt(3.0)
    xs += [[20.0, 30.0, 20.0], [20.0 + h, 30.0 + h, 20.0 + h]]
    xs += [[39.0, 35.0, 35.0], [np.nextafter(2.0, 0.0), 35.0, 35.0]]   # across the boundary
    q = np.zeros((len(xs), 4))
    q[:, :3] = xs
    s = inputs.LJSystem(q=q, box=np.array([40.0] * 3), rho=0.0)
    for half in (True, False):
        got, _ = _run(cuda_lib, s, half, 0, tpi)
        want = _oracle(oracle_lib, s, half)
        assert np.array_equal(np.any(want != 0.0, axis=1), np.any(got != 0.0, axis=1))
        assert _relerr(got, want) <= FP64_TOL


@pytest.mark.parametrize("scale", [0.3, 1.0, 25.0])
def test_fp64_fixed_point_box_sizes(cuda_lib, oracle_lib, scale):
    """The fixed-point shift k follows the box: tiny, unit and large boxes
    (sigma, r_c scaled with them), non-cubic, with momenta already set."""
    s = inputs.fcc_system(7, 0.9, 0.05, seed=4)
    st = np.array([1.0, 1.07, 1.15]) * scale
    s.q[:, :3] *= st
    s.box = s.box * st
    # momenta already set, at the scale of one impulse (a larger p0 would
    # hide the impulse's last digits in the rounding of p0 + dp)
    p0 = np.random.default_rng(6).normal(size=(s.n, 4)) * 1e-3 / scale
    kw = dict(dt=0.004, eps=0.8, sigma=1.05 * scale, rc=3.0 * scale)
    s.rc, s.margin = 3.0 * scale, 0.3 * scale
    for half in (True, False):
        want = _oracle(oracle_lib, s, half, p0=p0, **kw)
        for tpi in (2056, 1032):
            got, _ = _run(cuda_lib, s, half, 0, tpi, p0=p0, **kw)
            assert _relerr(got - p0[:, :3], want - p0[:, :3]) <= FP64_TOL


@pytest.mark.parametrize("tpi", [2052, 2056, 2064, 10244, 10256])
def test_fp64_long_rows(cuda_lib, oracle_lib, tpi):
    """r_c = 4, full list: ~330 entries a row, many strides of every group
    size of the fixed-point schedule."""
    s = inputs.fcc_system(10, 1.0, 0.05, seed=8)
    s.rc, s.margin = 4.0, 0.3
    for half in (True, False):
        got, _ = _run(cuda_lib, s, half, 0, tpi, rc=4.0)
        want = _oracle(oracle_lib, s, half, rc=4.0)
        assert _relerr(got, want) <= FP64_TOL


def test_fp64_box_wider_than_1024_cutoffs(cuda_lib, oracle_lib):
    """L = 4000 > 1024 r_c: the default FP64 schedule, the force+energy pass,
    the adjoint and the batched launch take image selection (the fixed point
    would resolve only 2^-41), and agree with the oracle; an explicit
    fixed-point schedule is refused."""
    from paper_1806_05713_gb300.batch import Batch
    lj = cuda_lib
    rng = np.random.default_rng(11)
    centres = np.array([[1.0, 2000.0, 3999.0], [3998.6, 1.2, 0.4], [2000.0, 2000.0, 2000.0]])
    pts = []
    for c in centres:
        for _ in range(6):
            pts.append(np.mod(c + rng.uniform(-1.2, 1.2, 3), 4000.0))
    q = np.zeros((len(pts), 4))
    q[:, :3] = pts
    s = inputs.LJSystem(q=q, box=np.array([4000.0] * 3), rho=0.0)
    qd = to_dev(s.q)
    for half in (True, False):
        want = _oracle(oracle_lib, s, half)
        got, pl = _run(lj, s, half, 0, 0)
        assert _relerr(got, want) <= FP64_TOL
        p = torch.zeros_like(qd)
        e = lj.lj_force_energy(qd, p, pl, 0.01, 3.0, s.box).item()
        rp, col = oracle_lib.pairlist(s.q, s.box, s.rs, half)
        assert abs(e - oracle_lib.energy(s.q, rp, col, half, 3.0, s.box)) <= 1e-12 * abs(e)
        assert _relerr(p.cpu().numpy()[:, :3], want) <= FP64_TOL
        with pytest.raises(lj.LJError):
            lj.lj_force(qd, torch.zeros_like(qd), pl, 0.01, 3.0, s.box, tpi=lj.LJ_SCHED_FIXED | 8)
    b = Batch([s, s], 0.01, 0, True, tpi=8, rows_per_item=8, plan_rows_min=8)
    b.force()
    torch.cuda.synchronize()
    want = _oracle(oracle_lib, s, True)
    out = b.p4.cpu().numpy()
    for k in range(2):
        assert _relerr(out[k * s.n:(k + 1) * s.n, :3], want) <= FP64_TOL


@pytest.mark.parametrize("half", [True, False])
@pytest.mark.parametrize("tpi", [2056, 2052, 2064, 10244, 10256])
def test_fp64_rare_lanes(cuda_lib, oracle_lib, half, tpi):
    """The fixed-point row's rare lanes: an extra atom 1e-11 from atom 0 (a
    squared distance far below the branch-free conversion's range, so the
    general conversion serves that pair), in a box of 8 sigma whose other
    entries fall on both sides of the conversion's two paths.  The close
    pair's impulse (~1e142) is checked on its two atoms, every other atom
    against its own scale."""
    lj = cuda_lib
    s = inputs.fcc_system(5, 1.0, 0.05, seed=21)      # L = 7.94, 500 atoms
    q = np.vstack([s.q, s.q[:1]])
    q[-1, 0] += 1e-11
    c = inputs.LJSystem(q=q, box=s.box, rho=s.rho)
    got, _ = _run(lj, c, half, 0, tpi)
    want = _oracle(oracle_lib, c, half)
    pair = [0, c.n - 1]
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got[pair] - want[pair])) <= FP64_TOL * np.max(np.abs(want[pair]))
    rest = np.ones(c.n, dtype=bool)
    rest[pair] = False
    assert _relerr(got[rest], want[rest]) <= FP64_TOL


@pytest.mark.parametrize("half", [True, False])
@pytest.mark.parametrize("tpi", [2056, 10256])
def test_fp64_scaled_system_divides(cuda_lib, oracle_lib, half, tpi):
    """Every length (positions, box, r_c, r_s, sigma) times 2^-64: each r^2
    then lies below 2^-119, outside the integer reciprocal's range, so every
    pair takes the division path.  (The other end, r^2 >= 2^120, cannot
    occur: lj_force refuses r_c^2 > 1e30.)  Scaling by a power of two is
    exact in binary arithmetic, so the oracle runs on the scaled system
    unchanged."""
    lj = cuda_lib
    f = 2.0 ** -64
    s = inputs.fcc_system(6, 1.0, 0.05, seed=4)
    c = inputs.LJSystem(q=s.q * f, box=s.box * f, rho=s.rho, rc=s.rc * f, margin=s.margin * f)
    got, _ = _run(lj, c, half, 0, tpi, sigma=f)
    want = _oracle(oracle_lib, c, half, sigma=f)
    assert np.all(np.isfinite(got))
    assert _relerr(got, want) <= FP64_TOL
    # and it is the unscaled result, scaled
    base, _ = _run(lj, s, half, 0, tpi)
    assert _relerr(got * f, base) <= FP64_TOL


def test_newton_third_law_half_list(cuda_lib, small):
    got, _ = _run(cuda_lib, small, True, 0, 2056)
    assert np.max(np.abs(got.sum(axis=0))) < 1e-12 * np.abs(got).sum()


def test_pad_column_untouched(cuda_lib, small):
    lj = cuda_lib
    q = to_dev(small.q)
    pl = lj.lj_build_pairlist(q, small.box, small.rs, True)
    p = torch.full((small.n, 4), 7.0, dtype=torch.float64, device="cuda")
    for prec, tpi in ((0, 2056), (0, 8), (1, 8), (2, 136)):
        lj.lj_force(q, p, pl, 0.01, 3.0, small.box, precision=prec, tpi=tpi)
    torch.cuda.synchronize()
    assert torch.all(p[:, 3] == 7.0)


@pytest.mark.parametrize("order", ["random", "cell"])
@pytest.mark.parametrize("half", [True, False])
def test_fp64_paper_size(cuda_lib, oracle_lib, order, half):
    """N = 119,164, both orderings and list kinds, the bench schedules."""
    s = inputs.workload_paper(order=order)
    want = _oracle(oracle_lib, s, half)
    pl = None
    for tpi in (8, 32, 136, 648, 1032, 1160, 1672, 2052, 2056, 2064, 2568, 10244, 10248, 10256,
                10272, 18440):
        got, pl = _run(cuda_lib, s, half, 0, tpi, pl=pl)
        assert _relerr(got, want) <= FP64_TOL, tpi


@pytest.mark.parametrize("half", [True, False])
def test_mixed_paper_size(cuda_lib, oracle_lib, half):
    s = inputs.workload_paper(order="cell")
    want = _oracle(oracle_lib, s, half)
    pl = None
    for tpi in (8, 16, 136):
        got, pl = _run(cuda_lib, s, half, 1, tpi, pl=pl)
        err = got - want
        assert np.max(np.abs(err)) / np.max(np.abs(want)) <= MIXED_TOL, tpi
        assert np.sqrt(np.mean(err ** 2)) / np.sqrt(np.mean(want ** 2)) <= 2.5e-6, tpi


@pytest.fixture(scope="module")
def million(oracle_lib):
    """N = 1,048,576 (64^3 FCC): 384 sampled atoms and their momentum change
    from the definition (every other atom, no list)."""
    s = inputs.workload_million()
    g = np.random.default_rng(17)
    idx = np.concatenate([[0, s.n - 1], g.choice(s.n, 382, replace=False)])
    want = oracle_lib.force_atoms(s.q, idx, 0.01, s.rc, s.box)
    return s, idx, want


@pytest.mark.parametrize("half", [True, False])
def test_million_atoms_all_forms_sampled(cuda_lib, million, half):
    """The benchmark's workload and launch configurations (the FP64 default
    and the schedules the benchmark times for each form), on sampled atoms
    against the oracle's per-atom sums."""
    lj = cuda_lib
    s, idx, want = million
    q = to_dev(s.q)
    pl = lj.lj_build_pairlist(q, s.box, s.rs, half)
    scale = np.max(np.abs(want))
    for prec, tpis, tol in ((0, (0, 2056, 2052, 1032, 10248, 10256), FP64_TOL),
                            (1, (4, 8, 16, 136, 16516), MIXED_TOL),
                            (2, (132, 136, 144), FP64_TOL)):
        for tpi in tpis:
            p = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
            lj.lj_force(q, p, pl, 0.01, s.rc, s.box, precision=prec, tpi=tpi)
            torch.cuda.synchronize()
            got = p[torch.from_numpy(idx).cuda(), :3].cpu().numpy()
            assert np.max(np.abs(got - want)) <= tol * scale, (prec, tpi)


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL), (2, FP64_TOL)])
def test_autotune_layout(cuda_lib, oracle_lib, small, precision, tol):
    """The layout chosen by measurement (half or full list) and its schedule
    give the oracle's momenta."""
    lj = cuda_lib
    q = to_dev(small.q)
    pl, tpi, ms, table = lj.lj_autotune_layout(q, small.box, small.rs, 0.01, small.rc,
                                               precision=precision, reps=2)
    assert (pl.half, tpi) in table and ms == min(table.values())
    assert {h for h, _ in table} == {True, False}
    p = torch.zeros_like(q)
    lj.lj_force(q, p, pl, 0.01, small.rc, small.box, precision=precision, tpi=tpi)
    torch.cuda.synchronize()
    want = _oracle(oracle_lib, small, True)
    assert _relerr(p.cpu().numpy()[:, :3], want) <= tol
