"""The double-float form (LJ_DFLOAT) vs the oracle: the FP64 bar (1e-12 of
max|dp|), on the small and paper-size systems, half and full lists, with
eps/sigma/dt, a non-cubic box, pairs on the cutoff, a pair closer than the
double-float range, a wrap across the boundary, and bitwise determinism of
the full list."""
import numpy as np
import pytest
import torch

from paper_1806_05713_gb300 import inputs
from conftest import to_dev

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
DF = 2
TPIS = [4, 8, 16, 132, 136, 144, 516, 520, 528, 648, 16516]  # 16384: LJ_SCHED_CELLS
# 128|t: two entries per lane in packed f32x2 registers; 512|t: rows in order of
# decreasing length


def _run(lj, s, half, tpi=8, dt=0.01, eps=1.0, sigma=1.0, p0=None, rc=None, pl=None):
    rc = s.rc if rc is None else rc
    q = to_dev(s.q)
    if pl is None:
        pl = lj.lj_build_pairlist(q, s.box, s.rs, half)
    p = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda") if p0 is None else to_dev(p0)
    lj.lj_force(q, p, pl, dt, rc, s.box, eps, sigma, DF, tpi)
    torch.cuda.synchronize()
    return p.cpu().numpy(), pl


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


@pytest.mark.parametrize("tpi", TPIS)
@pytest.mark.parametrize("half", [True, False])
def test_small(cuda_lib, oracle_lib, small, tpi, half):
    got, _ = _run(cuda_lib, small, half, tpi)
    want = _oracle(oracle_lib, small, half)
    assert _relerr(got[:, :3], want) <= FP64_TOL


def test_eps_sigma_dt_existing_momenta_noncubic(cuda_lib, oracle_lib):
    """A stretched FCC crystal in a 1 : 1.1 : 1.2 box, eps/sigma/dt not 1,
    momenta already set (p is updated in place, pad column untouched)."""
    s = inputs.fcc_system(8, 0.9, 0.05, seed=3)
    stretch = np.array([1.0, 1.1, 1.2])
    s.q[:, :3] *= stretch
    s.box = s.box * stretch
    p0 = np.random.default_rng(2).normal(size=(s.n, 4))
    kw = dict(dt=0.005, eps=1.3, sigma=1.1, rc=3.0)
    for half, tpi in ((True, 8), (False, 8), (True, 136), (False, 136)):
        got, _ = _run(cuda_lib, s, half, tpi, p0=p0, **kw)
        want = _oracle(oracle_lib, s, half, p0=p0, **kw)
        assert _relerr(got[:, :3] - p0[:, :3], want - p0[:, :3]) <= FP64_TOL
        assert np.array_equal(got[:, 3], p0[:, 3])


def test_two_body_closed_form(cuda_lib):
    """r = 1: dp = -+ 24 dt along d; r = 2^(1/6): dp ~ 0 (Algorithm 1)."""
    dt = 0.01
    for r, want in [(1.0, 24 * dt), (2.0 ** (1 / 6), 0.0)]:
        q = np.zeros((2, 4))
        q[:, :3] = 5.0
        q[1, 0] += r
        s = inputs.LJSystem(q=q, box=np.array([20.0] * 3), rho=0.0)
        for half, tpi in ((True, 4), (False, 4), (True, 132), (False, 132)):
            got, _ = _run(cuda_lib, s, half, tpi, dt=dt)
            assert abs(got[1, 0] - want) <= 1e-13 * 24 * dt
            assert abs(got[0, 0] + want) <= 1e-13 * 24 * dt
            assert np.all(got[:, 1:3] == 0.0)


def test_wrap_across_boundary(cuda_lib, oracle_lib):
    q = np.zeros((4, 4))
    q[0, :3] = [0.3, 5.0, 5.0]
    q[1, :3] = [9.3, 5.0, 5.0]
    q[2, :3] = [5.0, 0.05, 9.9]
    q[3, :3] = [5.5, 9.6, 0.4]
    s = inputs.LJSystem(q=q, box=np.array([10.0] * 3), rho=0.0)
    for half, tpi in ((True, 8), (False, 8), (True, 136), (False, 136)):
        got, _ = _run(cuda_lib, s, half, tpi)
        want = _oracle(oracle_lib, s, half)
        assert _relerr(got[:, :3], want) <= FP64_TOL
        assert abs(got[0, 0] - 0.24) < 1e-13


def test_pairs_on_the_cutoff(cuda_lib, oracle_lib):
    """Pairs at r_c (excluded: r^2 < r_c^2 is strict) and one ulp either side
    take the FP64 decision: the interacting set equals the oracle's."""
    L = 40.0
    xs = []
    for k, d in enumerate([3.0, np.nextafter(3.0, 0.0), np.nextafter(3.0, 4.0),
                           3.0 - 1e-15, 3.0 + 2e-15, 3.0 - 1e-12]):
        y = 2.0 + 4.0 * k
        xs += [[10.0, y, 5.0], [10.0 + d, y, 5.0]]
    # a diagonal pair with r^2 rounding onto r_c^2 from below in FP64
    xs += [[20.0, 30.0, 20.0], [20.0 + 3.0 / np.sqrt(3.0), 30.0 + 3.0 / np.sqrt(3.0),
                                20.0 + 3.0 / np.sqrt(3.0)]]
    q = np.zeros((len(xs), 4))
    q[:, :3] = xs
    s = inputs.LJSystem(q=q, box=np.array([L] * 3), rho=0.0)
    for half, tpi in ((True, 8), (False, 8), (True, 136), (False, 136)):
        got, _ = _run(cuda_lib, s, half, tpi)
        want = _oracle(oracle_lib, s, half)
        nz_want = np.any(want != 0.0, axis=1)
        nz_got = np.any(got[:, :3] != 0.0, axis=1)
        assert np.array_equal(nz_want, nz_got)
        assert _relerr(got[:, :3], want) <= FP64_TOL


def test_close_pair_takes_fp64(cuda_lib, oracle_lib):
    """r = 0.01 sigma: (sigma/r)^14 = 1e28 is beyond the double-float range
    of the pair loop; the FP64 formula serves that pair, the others stay in
    double-float."""
    q = np.zeros((4, 4))
    q[0, :3] = [5.0, 5.0, 5.0]
    q[1, :3] = [5.01, 5.0, 5.0]
    q[2, :3] = [6.1, 5.3, 5.0]
    q[3, :3] = [5.0, 6.2, 5.9]
    s = inputs.LJSystem(q=q, box=np.array([20.0] * 3), rho=0.0)
    for half, tpi in ((True, 4), (False, 4), (True, 132), (False, 132)):
        got, _ = _run(cuda_lib, s, half, tpi)
        want = _oracle(oracle_lib, s, half)
        assert np.all(np.isfinite(got))
        assert _relerr(got[:, :3], want) <= FP64_TOL
        # the remaining pairs, without the close one's huge impulse
        assert np.max(np.abs(got[2:, :3] - want[2:])) <= 1e-12 * np.max(np.abs(want[2:]))


def test_full_list_is_deterministic(cuda_lib, small):
    lj = cuda_lib
    q = to_dev(small.q)
    pl = lj.lj_build_pairlist(q, small.box, small.rs, False)
    for tpi in (8, 136):
        out = []
        for _ in range(3):
            p = torch.zeros((small.n, 4), dtype=torch.float64, device="cuda")
            lj.lj_force(q, p, pl, 0.01, 3.0, small.box, precision=DF, tpi=tpi)
            out.append(p)
        torch.cuda.synchronize()
        assert torch.equal(out[0], out[1]) and torch.equal(out[0], out[2])


def test_agrees_with_the_fp64_kernel(cuda_lib, small):
    lj = cuda_lib
    q = to_dev(small.q)
    for half in (True, False):
        pl = lj.lj_build_pairlist(q, small.box, small.rs, half)
        pd = torch.zeros((small.n, 4), dtype=torch.float64, device="cuda")
        p64 = torch.zeros_like(pd)
        lj.lj_force(q, pd, pl, 0.01, 3.0, small.box, precision=DF, tpi=8)
        lj.lj_force(q, p64, pl, 0.01, 3.0, small.box, precision=lj.LJ_FP64)
        torch.cuda.synchronize()
        err = float((pd - p64).abs().max()) / float(p64.abs().max())
        assert err <= 1e-13, err


@pytest.mark.parametrize("order", ["random", "cell"])
@pytest.mark.parametrize("half", [True, False])
def test_paper_size(cuda_lib, oracle_lib, order, half):
    """N = 119,164, both orderings and list kinds, the bench schedules."""
    s = inputs.workload_paper(order=order)
    want = _oracle(oracle_lib, s, half)
    pl = None
    for tpi in (8, 136, 144, 520, 648):
        got, pl = _run(cuda_lib, s, half, tpi, pl=pl)
        assert _relerr(got[:, :3], want) <= FP64_TOL, tpi


@pytest.mark.slow
def test_million_atoms(cuda_lib, oracle_lib):
    s = inputs.workload_million()
    want = _oracle(oracle_lib, s, True)
    got, _ = _run(cuda_lib, s, True, 0)
    assert _relerr(got[:, :3], want) <= FP64_TOL
