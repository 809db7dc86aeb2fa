"""Adjoint kernel (lj_force_vjp) and the autograd wrapper vs the oracle's
gradient and central finite differences (h = 1e-6) of the force-matching
loss  L = mean over atoms and components of (F(q; eps, sigma) - F_target)^2."""
import numpy as np
import pytest
import torch

from paper_1806_05713_gb300 import inputs
from conftest import to_dev

pytestmark = pytest.mark.gpu

EPS_T, SIG_T = 1.0, 1.0      # target parameters
EPS_M, SIG_M = 1.1, 0.97     # model parameters


def _setup(lj, oracle_lib, s, half):
    q = to_dev(s.q)
    pl = lj.lj_build_pairlist(q, s.box, s.rs, half)
    rp, col = oracle_lib.pairlist(s.q, s.box, s.rs, half)
    Ft = oracle_lib.forces(s.q, rp, col, half, s.rc, s.box, EPS_T, SIG_T)
    return q, pl, rp, col, Ft


@pytest.mark.parametrize("half", [True, False])
def test_vjp_fp64_matches_oracle(cuda_lib, oracle_lib, half):
    lj = cuda_lib
    s = inputs.fcc_system(8, 1.0, 0.1, seed=4)
    q, pl, rp, col, _ = _setup(lj, oracle_lib, s, half)
    R = np.random.default_rng(3).normal(size=(s.n, 4))
    gq, ges = lj.lj_force_vjp(q, to_dev(R), pl, s.rc, s.box, EPS_M, SIG_M, lj.LJ_FP64)
    torch.cuda.synchronize()
    want_q, want_e, want_s = oracle_lib.force_vjp(s.q, R, rp, col, half, s.rc, s.box, EPS_M, SIG_M)
    got = gq.cpu().numpy()
    assert np.all(got[:, 3] == 0.0)
    assert np.max(np.abs(got[:, :3] - want_q)) <= 1e-11 * np.max(np.abs(want_q))
    e, sg = ges.cpu().numpy()
    assert abs(e - want_e) <= 1e-10 * max(1.0, abs(want_e))
    assert abs(sg - want_s) <= 1e-10 * max(1.0, abs(want_s))


@pytest.mark.parametrize("half", [True, False])
def test_vjp_fp64_box_wider_than_1024_cutoffs(cuda_lib, oracle_lib, half):
    """L = 4000: the FP64 adjoint takes image selection there."""
    lj = cuda_lib
    rng = np.random.default_rng(12)
    pts = [np.mod(c + rng.uniform(-1.2, 1.2, 3), 4000.0)
           for c in ([0.5, 2000.0, 3999.5], [3999.0, 1.0, 0.2]) for _ in range(7)]
    q4 = np.zeros((len(pts), 4))
    q4[:, :3] = pts
    s = inputs.LJSystem(q=q4, box=np.array([4000.0] * 3), rho=0.0)
    q, pl, rp, col, _ = _setup(lj, oracle_lib, s, half)
    R = np.random.default_rng(5).normal(size=(s.n, 4))
    gq, ges = lj.lj_force_vjp(q, to_dev(R), pl, s.rc, s.box, EPS_M, SIG_M, lj.LJ_FP64)
    torch.cuda.synchronize()
    want_q, want_e, want_s = oracle_lib.force_vjp(s.q, R, rp, col, half, s.rc, s.box, EPS_M, SIG_M)
    assert np.max(np.abs(gq.cpu().numpy()[:, :3] - want_q)) <= 1e-11 * np.max(np.abs(want_q))
    e, sg = ges.cpu().numpy()
    assert abs(e - want_e) <= 1e-10 * max(1.0, abs(want_e))
    assert abs(sg - want_s) <= 1e-10 * max(1.0, abs(want_s))


@pytest.mark.parametrize("half", [True, False])
def test_vjp_mixed_within_stated_error(cuda_lib, oracle_lib, half):
    lj = cuda_lib
    s = inputs.fcc_system(8, 1.0, 0.1, seed=4)
    q, pl, rp, col, _ = _setup(lj, oracle_lib, s, half)
    R = np.random.default_rng(3).normal(size=(s.n, 4))
    gq, ges = lj.lj_force_vjp(q, to_dev(R), pl, s.rc, s.box, EPS_M, SIG_M, lj.LJ_MIXED)
    want_q, want_e, want_s = oracle_lib.force_vjp(s.q, R, rp, col, half, s.rc, s.box, EPS_M, SIG_M)
    got = gq.cpu().numpy()[:, :3]
    assert np.max(np.abs(got - want_q)) <= 1e-4 * np.max(np.abs(want_q))
    e, sg = ges.cpu().numpy()
    assert abs(e - want_e) <= 1e-4 * abs(want_e)
    assert abs(sg - want_s) <= 1e-4 * abs(want_s)


def _loss_and_grads(lj, q, pl, s, Ft_dev, precision):
    from paper_1806_05713_gb300.autograd import lj_forces
    qq = q.clone().requires_grad_(True)
    eps = torch.tensor(EPS_M, dtype=torch.float64, device="cuda", requires_grad=True)
    sig = torch.tensor(SIG_M, dtype=torch.float64, device="cuda", requires_grad=True)
    F = lj_forces(qq, eps, sig, pl, s.rc, s.box, precision)
    loss = ((F[:, :3] - Ft_dev[:, :3]) ** 2).mean()
    loss.backward()
    return loss.item(), qq.grad[:, :3].cpu().numpy(), eps.grad.item(), sig.grad.item()


@pytest.mark.parametrize("half", [True, False])
def test_autograd_fp64_vs_oracle_and_central_differences(cuda_lib, oracle_lib, half):
    lj = cuda_lib
    s = inputs.fcc_system(16, 1.0, 0.1, seed=1)     # N = 16,384 (one replica of the config)
    q, pl, rp, col, Ft = _setup(lj, oracle_lib, s, half)
    Ft_dev = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
    Ft_dev[:, :3] = torch.from_numpy(Ft).cuda()
    loss, gq, ge, gs = _loss_and_grads(lj, q, pl, s, Ft_dev, lj.LJ_FP64)
    # oracle gradient of the same loss
    Fm = oracle_lib.forces(s.q, rp, col, half, s.rc, s.box, EPS_M, SIG_M)
    R = 2.0 * (Fm - Ft) / Fm.size
    oq, oe, os_ = oracle_lib.force_vjp(s.q, R, rp, col, half, s.rc, s.box, EPS_M, SIG_M)
    assert abs(loss - np.mean((Fm - Ft) ** 2)) <= 1e-12 * loss
    assert np.max(np.abs(gq - oq)) <= 1e-10 * np.max(np.abs(oq))
    assert abs(ge - oe) <= 1e-9 * abs(oe) and abs(gs - os_) <= 1e-9 * abs(os_)

    # central differences of the GPU forward, h = 1e-6
    h = 1e-6

    def L(qd=q, e=EPS_M, sg=SIG_M):
        F = torch.zeros_like(qd)
        lj.lj_force(qd, F, pl, 1.0, s.rc, s.box, e, sg, lj.LJ_FP64)
        return ((F[:, :3] - Ft_dev[:, :3]) ** 2).mean().item()

    fe = (L(e=EPS_M + h) - L(e=EPS_M - h)) / (2 * h)
    fs = (L(sg=SIG_M + h) - L(sg=SIG_M - h)) / (2 * h)
    assert abs(fe - ge) <= 1e-6 * abs(ge), (fe, ge)
    assert abs(fs - gs) <= 1e-6 * abs(gs), (fs, gs)
    rng = np.random.default_rng(0)
    scale = np.max(np.abs(gq))
    for _ in range(6):
        i, a = int(rng.integers(s.n)), int(rng.integers(3))
        qp, qm = q.clone(), q.clone()
        qp[i, a] += h
        qm[i, a] -= h
        fd = (L(qd=qp) - L(qd=qm)) / (2 * h)
        assert abs(fd - gq[i, a]) <= 1e-5 * scale, (i, a, fd, gq[i, a])


def test_autograd_mixed_vs_oracle(cuda_lib, oracle_lib):
    lj = cuda_lib
    s = inputs.fcc_system(16, 1.0, 0.1, seed=1)
    q, pl, rp, col, Ft = _setup(lj, oracle_lib, s, False)
    Ft_dev = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
    Ft_dev[:, :3] = torch.from_numpy(Ft).cuda()
    loss, gq, ge, gs = _loss_and_grads(lj, q, pl, s, Ft_dev, lj.LJ_MIXED)
    Fm = oracle_lib.forces(s.q, rp, col, False, s.rc, s.box, EPS_M, SIG_M)
    R = 2.0 * (Fm - Ft) / Fm.size
    oq, oe, os_ = oracle_lib.force_vjp(s.q, R, rp, col, False, s.rc, s.box, EPS_M, SIG_M)
    assert np.max(np.abs(gq - oq)) <= 1e-4 * np.max(np.abs(oq))
    assert abs(ge - oe) <= 1e-4 * abs(oe) and abs(gs - os_) <= 1e-4 * abs(os_)


# --------------------------------------------------------------------------
# The double-float form, held to the FP64 tolerances
# --------------------------------------------------------------------------

@pytest.mark.parametrize("half", [True, False])
@pytest.mark.parametrize("stretch", [(1.0, 1.0, 1.0), (1.0, 1.1, 1.2)])
def test_vjp_dfloat_matches_oracle(cuda_lib, oracle_lib, half, stretch):
    lj = cuda_lib
    s = inputs.fcc_system(8, 1.0, 0.1, seed=4)
    st = np.array(stretch)
    s.q[:, :3] *= st
    s.box = s.box * st
    q, pl, rp, col, _ = _setup(lj, oracle_lib, s, half)
    R = np.random.default_rng(3).normal(size=(s.n, 4))
    gq, ges = lj.lj_force_vjp(q, to_dev(R), pl, s.rc, s.box, EPS_M, SIG_M, lj.LJ_DFLOAT)
    torch.cuda.synchronize()
    want_q, want_e, want_s = oracle_lib.force_vjp(s.q, R, rp, col, half, s.rc, s.box, EPS_M, SIG_M)
    got = gq.cpu().numpy()
    assert np.all(got[:, 3] == 0.0)
    assert np.max(np.abs(got[:, :3] - want_q)) <= 1e-11 * np.max(np.abs(want_q))
    e, sg = ges.cpu().numpy()
    assert abs(e - want_e) <= 1e-10 * max(1.0, abs(want_e))
    assert abs(sg - want_s) <= 1e-10 * max(1.0, abs(want_s))


def test_vjp_dfloat_close_pair_takes_fp64(cuda_lib, oracle_lib):
    """A pair at 0.02 sigma (u^8 beyond the double-float range) and pairs on
    the cutoff take the FP64 formulas."""
    lj = cuda_lib
    q4 = np.zeros((6, 4))
    q4[:, :3] = [[5.0, 5.0, 5.0], [5.02, 5.0, 5.0], [6.1, 5.3, 5.0], [5.0, 6.2, 5.9],
                 [12.0, 12.0, 12.0], [15.0, 12.0, 12.0]]
    s = inputs.LJSystem(q=q4, box=np.array([20.0] * 3), rho=0.0)
    for half in (True, False):
        q, pl, rp, col, _ = _setup(lj, oracle_lib, s, half)
        R = np.random.default_rng(8).normal(size=(s.n, 4))
        gq, ges = lj.lj_force_vjp(q, to_dev(R), pl, s.rc, s.box, EPS_M, SIG_M, lj.LJ_DFLOAT)
        want_q, want_e, want_s = oracle_lib.force_vjp(s.q, R, rp, col, half, s.rc, s.box,
                                                      EPS_M, SIG_M)
        got = gq.cpu().numpy()[:, :3]
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want_q)) <= 1e-11 * np.max(np.abs(want_q))
        e, sg = ges.cpu().numpy()
        assert abs(e - want_e) <= 1e-10 * max(1.0, abs(want_e))
        assert abs(sg - want_s) <= 1e-10 * max(1.0, abs(want_s))


def test_autograd_dfloat_vs_oracle(cuda_lib, oracle_lib):
    lj = cuda_lib
    s = inputs.fcc_system(16, 1.0, 0.1, seed=1)
    q, pl, rp, col, Ft = _setup(lj, oracle_lib, s, False)
    Ft_dev = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
    Ft_dev[:, :3] = torch.from_numpy(Ft).cuda()
    loss, gq, ge, gs = _loss_and_grads(lj, q, pl, s, Ft_dev, lj.LJ_DFLOAT)
    Fm = oracle_lib.forces(s.q, rp, col, False, s.rc, s.box, EPS_M, SIG_M)
    R = 2.0 * (Fm - Ft) / Fm.size
    oq, oe, os_ = oracle_lib.force_vjp(s.q, R, rp, col, False, s.rc, s.box, EPS_M, SIG_M)
    assert abs(loss - np.mean((Fm - Ft) ** 2)) <= 1e-11 * loss
    assert np.max(np.abs(gq - oq)) <= 1e-10 * np.max(np.abs(oq))
    assert abs(ge - oe) <= 1e-9 * abs(oe) and abs(gs - os_) <= 1e-9 * abs(os_)


def test_vjp_fp64_million_half_list_sampled(cuda_lib, oracle_lib):
    """N = 1,048,576 on a half list, the adjoint benchmark's size and layout
    (large half lists take the walk with one chunk of entries per lane):
    dLoss/dq on sampled atoms against the oracle's per-atom sums (each atom's
    full row from the oracle's list, processed alone), and dLoss/deps against
    the identity dL/deps = sum_i R_i . F_i(q; eps, sigma) / eps, with F from
    lj_force (itself checked against the oracle)."""
    lj = cuda_lib
    s = inputs.workload_million()
    q = to_dev(s.q)
    pl = lj.lj_build_pairlist(q, s.box, s.rs, True)
    g = np.random.default_rng(21)
    R = g.normal(size=(s.n, 4))
    R[:, 3] = 0.0
    gq, ges = lj.lj_force_vjp(q, to_dev(R), pl, s.rc, s.box, EPS_M, SIG_M, lj.LJ_FP64)
    F = torch.zeros_like(q)
    lj.lj_force(q, F, pl, 1.0, s.rc, s.box, EPS_M, SIG_M, lj.LJ_FP64)
    torch.cuda.synchronize()
    got = gq.cpu().numpy()[:, :3]
    assert np.all(np.isfinite(got))
    idx = np.concatenate([[0, s.n - 1], g.choice(s.n, 126, replace=False)])
    want = np.empty((idx.size, 3))
    for m, a in enumerate(idx):
        rp_a, col_a = oracle_lib.pairlist_rows(s.q, s.box, s.rs, False, int(a), int(a) + 1)
        row_ptr = np.zeros(s.n + 1, dtype=np.int32)
        row_ptr[a + 1:] = col_a.size
        wq, _, _ = oracle_lib.force_vjp(s.q, R, row_ptr, col_a, True, s.rc, s.box, EPS_M, SIG_M)
        want[m] = wq[a]
    assert np.max(np.abs(got[idx] - want)) <= 1e-11 * np.max(np.abs(want))
    e = float(ges.cpu().numpy()[0])
    want_e = float(np.sum(R[:, :3] * F.cpu().numpy()[:, :3])) / EPS_M
    assert abs(e - want_e) <= 1e-10 * abs(want_e)
