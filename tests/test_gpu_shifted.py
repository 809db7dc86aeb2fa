"""The force-shifted truncation (lj_force_shifted) vs the oracle's force_fs
and energy_fs, and its effect on energy conservation in velocity Verlet."""
import numpy as np
import pytest
import torch

from paper_1806_05713_gb300 import inputs
from conftest import to_dev

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _case(lj, oracle_lib, s, half, dt=0.01, eps=1.0, sigma=1.0, p0=None):
    q = to_dev(s.q)
    pl = lj.lj_build_pairlist(q, s.box, s.rs, half)
    p = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda") if p0 is None else to_dev(p0)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    lj.lj_force_shifted(q, p, pl, dt, s.rc, s.box, eps, sigma, out=e)
    p2 = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda") if p0 is None else to_dev(p0)
    lj.lj_force_shifted(q, p2, pl, dt, s.rc, s.box, eps, sigma)
    torch.cuda.synchronize()
    rp, col = oracle_lib.pairlist(s.q, s.box, s.rs, half)
    base = np.zeros((s.n, 3)) if p0 is None else p0[:, :3]
    want = oracle_lib.force_fs(s.q, base, rp, col, half, dt, s.rc, s.box, eps, sigma)
    want_e = oracle_lib.energy_fs(s.q, rp, col, half, s.rc, s.box, eps, sigma)
    got = p.cpu().numpy()[:, :3]
    scale = np.max(np.abs(want - base))
    assert np.max(np.abs(got - want)) <= FP64_TOL * scale
    assert abs(float(e.item()) - want_e) <= 1e-12 * abs(want_e)
    if not half:   # full lists are deterministic: the energy pass changes no bit
        assert torch.equal(p, p2)
    else:
        assert float((p - p2).abs().max()) <= 1e-13 * scale


@pytest.mark.parametrize("half", [True, False])
def test_small(cuda_lib, oracle_lib, half):
    _case(cuda_lib, oracle_lib, inputs.workload_small(), half)


@pytest.mark.parametrize("half", [True, False])
def test_eps_sigma_dt_existing_momenta(cuda_lib, oracle_lib, half):
    s = inputs.fcc_system(8, 0.9, 0.05, seed=13)
    p0 = np.random.default_rng(4).normal(size=(s.n, 4)) * 1e-3
    _case(cuda_lib, oracle_lib, s, half, dt=0.004, eps=1.2, sigma=0.93, p0=p0)


@pytest.mark.parametrize("half", [True, False])
def test_paper_size(cuda_lib, oracle_lib, half):
    _case(cuda_lib, oracle_lib, inputs.workload_paper(), half)


def test_pair_at_the_cutoff_gets_no_impulse(cuda_lib):
    lj = cuda_lib
    q = np.zeros((2, 4))
    q[:, :3] = 10.0
    q[1, 0] += np.nextafter(3.0, 0.0)   # just inside r_c: the shifted force is ~0
    s = inputs.LJSystem(q=q, box=np.array([20.0] * 3), rho=0.0)
    qd = to_dev(s.q)
    pl = lj.lj_build_pairlist(qd, s.box, s.rs, True)
    p = torch.zeros_like(qd)
    lj.lj_force_shifted(qd, p, pl, 1.0, 3.0, s.box)
    torch.cuda.synchronize()
    assert float(p.abs().max()) < 1e-12


def test_wide_box_is_refused(cuda_lib):
    lj = cuda_lib
    q = np.zeros((2, 4))
    q[:, :3] = 10.0
    q[1, 0] += 1.0
    qd = to_dev(q)
    pl = lj.lj_build_pairlist(qd, [4000.0] * 3, 3.3, True)
    with pytest.raises(lj.LJError):
        lj.lj_force_shifted(qd, torch.zeros_like(qd), pl, 0.01, 3.0, [4000.0] * 3)


def test_force_shifted_md_conserves_energy(cuda_lib):
    """Velocity Verlet on a hot FCC melt with the force-shifted truncation:
    its total energy (kinetic + force-shifted potential) is conserved as
    well as the plain cut's over 400 steps (both at the integrator's
    O(dt^2) level here)."""
    from paper_1806_05713_gb300.md import VelocityVerlet
    drift = {}
    for trunc in ("plain", "force_shifted"):
        s = inputs.fcc_system(10, 0.8, 0.05, seed=2)
        p0 = np.random.default_rng(5).normal(size=(s.n, 4)) * 1.2
        p0[:, 3] = 0.0
        p0[:, :3] -= p0[:, :3].mean(axis=0)
        q, p = to_dev(s.q), to_dev(p0)
        vv = VelocityVerlet(q, p, s.box, s.rc, s.margin, 0.002, truncation=trunc)
        e0 = vv.kinetic_energy() + vv.potential_energy()
        vv.run(400)
        e1 = vv.kinetic_energy() + vv.potential_energy()
        drift[trunc] = abs(e1 - e0) / abs(e0)
    assert drift["force_shifted"] < 1e-4 and drift["plain"] < 1e-4, drift
    assert drift["force_shifted"] < 3.0 * drift["plain"] + 1e-6, drift
