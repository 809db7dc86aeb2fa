"""Drift kernel and velocity-Verlet driver with the bookkeeping rebuild rule."""
import numpy as np
import pytest
import torch

from paper_1806_05713_gb300 import inputs
from conftest import to_dev

pytestmark = pytest.mark.gpu


def _np_drift(q, p, dt, L):
    """The definition: x = q + dt p (separately rounded), one periodic wrap."""
    out = q.copy()
    d2 = np.zeros(q.shape[0])
    for a in range(3):
        dq = dt * p[:, a]
        x = q[:, a] + dq
        x = np.where(x >= L[a], x - L[a], np.where(x < 0.0, x + L[a], x))
        x = np.where(x < L[a], x, 0.0)
        out[:, a] = x
        d2 = d2 + dq * dq
    return out, float(d2.max())


def test_drift_bit_exact(cuda_lib):
    lj = cuda_lib
    rng = np.random.default_rng(0)
    L = np.array([10.0, 12.5, 7.25])
    q = np.zeros((5000, 4))
    q[:, :3] = rng.random((5000, 3)) * L
    q[:3, 0] = [0.0, np.nextafter(L[0], 0), 5.0]
    p = rng.normal(size=(5000, 4)) * 3.0
    want, want_d2 = _np_drift(q, p, 0.013, L)
    qd = to_dev(q)
    m = lj.lj_drift(qd, to_dev(p), 0.013, L)
    got = qd.cpu().numpy()
    assert np.array_equal(got[:, :3], want[:, :3])
    assert np.array_equal(got[:, 3], q[:, 3])
    assert m.item() == want_d2
    assert np.all((got[:, :3] >= 0) & (got[:, :3] < L))


@pytest.mark.parametrize("precision", [0, 2])
def test_verlet_matches_oracle_integrator(cuda_lib, oracle_lib, precision):
    """FP64 and double-float forces: the same trajectory as the oracle's."""
    from paper_1806_05713_gb300.md import VelocityVerlet
    lj = cuda_lib
    s = inputs.fcc_system(10, 1.0, 0.05, seed=3)
    dt, steps = 0.005, 20
    p0 = np.random.default_rng(1).normal(size=(s.n, 4)) * 0.5
    p0[:, 3] = 0.0
    q, p = to_dev(s.q), to_dev(p0)
    vv = VelocityVerlet(q, p, s.box, s.rc, s.margin, dt, precision=precision)
    vv.run(steps)
    torch.cuda.synchronize()
    # reference: the same leapfrog with the oracle's list and force, fresh list every step
    qr, pr = s.q.copy(), p0[:, :3].copy()

    def kick(h):
        rp, col = oracle_lib.pairlist(qr, s.box, s.rs, True)
        return oracle_lib.force(qr, pr, rp, col, True, h, s.rc, s.box)
    pr = kick(0.5 * dt)
    for k in range(steps):
        qn, _ = _np_drift(qr, np.concatenate([pr, np.zeros((s.n, 1))], 1), dt, s.box)
        qr = qn
        pr = kick(0.5 * dt if k == steps - 1 else dt)
    dq = q.cpu().numpy()[:, :3] - qr[:, :3]
    dq -= s.box * np.round(dq / s.box)
    assert np.max(np.abs(dq)) < 1e-11
    assert np.max(np.abs(p.cpu().numpy()[:, :3] - pr)) < 1e-9 * np.max(np.abs(pr))


def test_energy_conservation_and_bookkeeping(cuda_lib):
    from paper_1806_05713_gb300.md import VelocityVerlet
    lj = cuda_lib
    s = inputs.fcc_system(10, 0.8, 0.05, seed=2)
    p0 = np.random.default_rng(5).normal(size=(s.n, 4)) * 1.2   # hot: atoms move, lists rebuild
    p0[:, 3] = 0.0
    p0[:, :3] -= p0[:, :3].mean(axis=0)
    q, p = to_dev(s.q), to_dev(p0)
    vv = VelocityVerlet(q, p, s.box, s.rc, s.margin, 0.002)
    e0 = vv.kinetic_energy() + vv.potential_energy(shifted=True)
    vv.run(400)
    e1 = vv.kinetic_energy() + vv.potential_energy(shifted=True)
    assert vv.rebuilds >= 3
    assert abs(e1 - e0) < 2e-3 * abs(e0), (e0, e1)
    # the list in use still holds every pair within r_c: same forces as a fresh list
    F_old = torch.zeros_like(q)
    lj.lj_force(q, F_old, vv.plist, 1.0, s.rc, s.box)
    fresh = lj.lj_build_pairlist(q, s.box, s.rs, True)
    F_new = torch.zeros_like(q)
    lj.lj_force(q, F_new, fresh, 1.0, s.rc, s.box)
    assert float((F_old - F_new).abs().max()) <= 1e-12 * float(F_new.abs().max())
    # total momentum stays zero (Newton's third law, half-list atomics)
    assert float(p[:, :3].sum(0).abs().max()) < 1e-9


def test_energies_from_the_force_pass(cuda_lib):
    """run(energies=...) records U(q(t_k)) from lj_force_energy; the last one
    equals a separate lj_energy pass on the final positions."""
    from paper_1806_05713_gb300.md import VelocityVerlet
    lj = cuda_lib
    s = inputs.fcc_system(8, 1.0, 0.05, seed=4)
    q = to_dev(s.q)
    p = torch.zeros_like(q)
    vv = VelocityVerlet(q, p, s.box, s.rc, s.margin, 0.005)
    U = torch.zeros(30, dtype=torch.float64, device="cuda")
    vv.run(30, energies=U)
    u_last = float(U[-1])
    assert abs(u_last - vv.potential_energy(shifted=True)) <= 1e-12 * abs(u_last)
    assert torch.all(U < 0)


def _hot_system(seed=2):
    s = inputs.fcc_system(10, 0.8, 0.05, seed=seed)
    p0 = np.random.default_rng(5).normal(size=(s.n, 4)) * 1.2
    p0[:, 3] = 0.0
    p0[:, :3] -= p0[:, :3].mean(axis=0)
    return s, p0


def test_device_driver_energies_and_displacement_criterion(cuda_lib):
    """Per-step energies through lj_md_steps equal the host-checked loop's
    (full list: bit for bit); the displacement criterion rebuilds no more
    often than the fastest-atom bound, keeps every pair within r_c in the
    list, and follows the same trajectory to rounding."""
    from paper_1806_05713_gb300.md import VelocityVerlet
    lj = cuda_lib
    s, p0 = _hot_system(seed=11)
    res = {}
    for name, driver, crit in (("host", "host", "fastest_atom"), ("device", "device", "fastest_atom"),
                               ("disp", "device", "displacement")):
        q, p = to_dev(s.q), to_dev(p0)
        vv = VelocityVerlet(q, p, s.box, s.rc, s.margin, 0.002, half=False, driver=driver,
                            criterion=crit)
        U = torch.zeros(90, dtype=torch.float64, device="cuda")
        vv.run(90, energies=U)
        torch.cuda.synchronize()
        res[name] = (q, p, U, vv)
    qh, ph, Uh, vh = res["host"]
    qd, pd, Ud, vd = res["device"]
    assert vd.rebuilds == vh.rebuilds >= 2
    assert torch.equal(Ud, Uh) and torch.equal(qd, qh) and torch.equal(pd, ph)
    qx, px, Ux, vx = res["disp"]
    assert vx.rebuilds <= vh.rebuilds
    dq = qx.cpu().numpy()[:, :3] - qh.cpu().numpy()[:, :3]
    dq -= s.box * np.round(dq / s.box)
    assert np.max(np.abs(dq)) < 1e-10
    assert float((Ux - Uh).abs().max()) <= 1e-10 * float(Uh.abs().max())
    F_old = torch.zeros_like(qx)
    lj.lj_force(qx, F_old, vx.plist, 1.0, s.rc, s.box)
    fresh = lj.lj_build_pairlist(qx, s.box, s.rs, False)
    F_new = torch.zeros_like(qx)
    lj.lj_force(qx, F_new, fresh, 1.0, s.rc, s.box)
    assert float((F_old - F_new).abs().max()) <= 1e-12 * float(F_new.abs().max())


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_device_driver_equals_host_driver(cuda_lib, precision):
    """lj_md_steps (the validity test on the device, steps queued in batches)
    against the host-checked loop: with the full list (no atomics, so every
    kernel is deterministic) the trajectories agree bit for bit and the list
    is rebuilt at the same steps."""
    from paper_1806_05713_gb300.md import VelocityVerlet
    s, p0 = _hot_system()
    out = {}
    for driver in ("device", "host"):
        q, p = to_dev(s.q), to_dev(p0)
        vv = VelocityVerlet(q, p, s.box, s.rc, s.margin, 0.002, precision=precision, half=False,
                            driver=driver)
        vv.run(150)
        vv.run(60)
        torch.cuda.synchronize()
        out[driver] = (q.cpu().numpy(), p.cpu().numpy(), vv.rebuilds)
    qd, pd, rd = out["device"]
    qh, ph, rh = out["host"]
    assert rd == rh and rd >= 3
    assert np.array_equal(qd, qh)
    assert np.array_equal(pd, ph)


def test_device_driver_half_list(cuda_lib):
    """Half list (FP64 atomics, so sums in any order): the two drivers agree
    to rounding and the list in use still holds every pair within r_c."""
    from paper_1806_05713_gb300.md import VelocityVerlet
    lj = cuda_lib
    s, p0 = _hot_system(seed=7)
    res = {}
    for driver in ("device", "host"):
        q, p = to_dev(s.q), to_dev(p0)
        vv = VelocityVerlet(q, p, s.box, s.rc, s.margin, 0.002, driver=driver)
        vv.run(120)
        torch.cuda.synchronize()
        res[driver] = (q, p, vv)
    q, p, vv = res["device"]
    assert vv.rebuilds >= 3
    dq = q.cpu().numpy()[:, :3] - res["host"][0].cpu().numpy()[:, :3]
    dq -= s.box * np.round(dq / s.box)
    assert np.max(np.abs(dq)) < 1e-10
    F_old = torch.zeros_like(q)
    lj.lj_force(q, F_old, vv.plist, 1.0, s.rc, s.box)
    fresh = lj.lj_build_pairlist(q, s.box, s.rs, True)
    F_new = torch.zeros_like(q)
    lj.lj_force(q, F_new, fresh, 1.0, s.rc, s.box)
    assert float((F_old - F_new).abs().max()) <= 1e-12 * float(F_new.abs().max())


def test_md_steps_stale_state_does_nothing(cuda_lib):
    """A state already marked stale: no drift, no kick, the list's rows
    emptied; a margin used up inside the call stops the steps after it."""
    lj = cuda_lib
    s, p0 = _hot_system()
    q, p = to_dev(s.q), to_dev(p0)
    pl = lj.lj_build_pairlist(q, s.box, s.rs, True)
    state = lj.lj_md_state_new(q.device)
    ints = state.view(torch.int32)
    ints[8] = 1                                   # stale
    q0, p0d = q.clone(), p.clone()
    lj.lj_md_steps(q, p, pl, 5, 0.002, s.rc, s.rs, s.box, state=state)
    torch.cuda.synchronize()
    assert torch.equal(q, q0) and torch.equal(p, p0d)
    assert int(pl.row_ptr.abs().sum()) == 0
    st = lj.lj_md_state_read(state)
    assert st["stale"] == 1 and st["steps"] == 0
    # a tiny margin: the first drift uses it up; only that drift happens
    pl = lj.lj_build_pairlist(q, s.box, s.rs, True)
    state = lj.lj_md_state_new(q.device)
    lj.lj_md_steps(q, p, pl, 4, 0.002, s.rc, s.rc + 1e-6, s.box, state=state)
    st = lj.lj_md_state_read(state)
    assert st["stale"] == 1 and st["steps"] == 0
    want, want_d2 = _np_drift(q0.cpu().numpy(), p0d.cpu().numpy(), 0.002, s.box)
    assert np.array_equal(q.cpu().numpy(), want)
    assert torch.equal(p, p0d)
    assert st["last_disp2"] == want_d2
    assert st["moved"] == np.sqrt(want_d2)


def test_pressure(cuda_lib, oracle_lib):
    """VelocityVerlet.pressure: (2 K + W) / 3V with the oracle's virial; a
    dilute gas is close to the ideal-gas value 2 K / 3V."""
    from paper_1806_05713_gb300.md import VelocityVerlet
    s, p0 = _hot_system()
    q, p = to_dev(s.q), to_dev(p0)
    vv = VelocityVerlet(q, p, s.box, s.rc, s.margin, 0.002)
    P = vv.pressure()
    K = vv.kinetic_energy()
    V = float(np.prod(s.box))
    rp, col = oracle_lib.pairlist(s.q, s.box, s.rs, True)
    W = oracle_lib.virial(s.q, rp, col, True, s.rc, s.box)
    want = (2 * K + W) / (3 * V)
    assert abs(P - want) <= 1e-12 * abs(want)
    # no pair within r_c (a jittered lattice of spacing 8): the ideal-gas value exactly
    rng = np.random.default_rng(4)
    g = (np.arange(7) + 0.5) * 8.0
    L = 56.0
    gas = np.zeros((343, 4))
    gas[:, :3] = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    gas[:, :3] += rng.uniform(-0.5, 0.5, (343, 3))
    pg = np.zeros((343, 4))
    pg[:, :3] = rng.normal(size=(343, 3))
    vg = VelocityVerlet(to_dev(gas), to_dev(pg), [L, L, L], 3.0, 0.3, 0.002)
    assert vg.pressure() == 2 * vg.kinetic_energy() / (3 * L ** 3)
