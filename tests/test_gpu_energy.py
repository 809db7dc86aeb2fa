"""GPU energy (Eq. 1, truncated, optionally shifted) vs the oracle."""
import numpy as np
import pytest
import torch

from paper_1806_05713_gb300 import inputs
from conftest import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("half", [True, False])
@pytest.mark.parametrize("shifted", [False, True])
def test_energy_matches_oracle(cuda_lib, oracle_lib, half, shifted):
    lj = cuda_lib
    s = inputs.workload_small()
    q = to_dev(s.q)
    pl = lj.lj_build_pairlist(q, s.box, s.rs, half)
    e = lj.lj_energy(q, pl, 3.0, s.box, 1.2, 0.95, shifted).item()
    rp, col = oracle_lib.pairlist(s.q, s.box, s.rs, half)
    want = oracle_lib.energy(s.q, rp, col, half, 3.0, s.box, 1.2, 0.95, shifted)
    assert abs(e - want) <= 1e-12 * abs(want)


def test_energy_closed_form_and_determinism(cuda_lib):
    lj = cuda_lib
    q = np.zeros((2, 4))
    q[:, :3] = 5.0
    q[1, 2] += 2.0 ** (1 / 6)
    pl = lj.lj_build_pairlist(to_dev(q), [20.0] * 3, 3.3, True)
    assert abs(lj.lj_energy(to_dev(q), pl, 3.0, [20.0] * 3).item() + 1.0) < 1e-15
    s = inputs.workload_paper()
    qd = to_dev(s.q)
    pl = lj.lj_build_pairlist(qd, s.box, s.rs, True)
    a = lj.lj_energy(qd, pl, 3.0, s.box).item()
    b = lj.lj_energy(qd, pl, 3.0, s.box).item()
    assert a == b


@pytest.mark.parametrize("half", [True, False])
@pytest.mark.parametrize("shifted", [False, True])
def test_force_energy_one_pass(cuda_lib, oracle_lib, half, shifted):
    """lj_force_energy: the same momenta as lj_force and the oracle's energy."""
    lj = cuda_lib
    s = inputs.fcc_system(12, 0.95, 0.05, seed=6)
    q = to_dev(s.q)
    pl = lj.lj_build_pairlist(q, s.box, s.rs, half)
    p1 = torch.zeros_like(q)
    e = lj.lj_force_energy(q, p1, pl, 0.01, 3.0, s.box, 1.1, 0.97, shifted).item()
    p2 = torch.zeros_like(q)
    lj.lj_force(q, p2, pl, 0.01, 3.0, s.box, 1.1, 0.97, tpi=lj.LJ_SCHED_FIXED | 8)
    torch.cuda.synchronize()
    if half:
        assert float((p1 - p2).abs().max()) <= 1e-13 * float(p2.abs().max())
    else:
        assert torch.equal(p1, p2)
    rp, col = oracle_lib.pairlist(s.q, s.box, s.rs, half)
    want = oracle_lib.energy(s.q, rp, col, half, 3.0, s.box, 1.1, 0.97, shifted)
    assert abs(e - want) <= 1e-12 * abs(want)
    again = lj.lj_force_energy(q, torch.zeros_like(q), pl, 0.01, 3.0, s.box, 1.1, 0.97, shifted).item()
    assert again == e


@pytest.mark.parametrize("half", [True, False])
@pytest.mark.parametrize("wide", [False, True])
def test_force_energy_virial(cuda_lib, oracle_lib, half, wide):
    """lj_force_energy_virial: the oracle's pair virial (and energy, and the
    momenta of lj_force_energy), deterministic; `wide` takes a box wider
    than 1024 r_c, where the pass runs the image-selected rows."""
    lj = cuda_lib
    s = inputs.fcc_system(10, 0.95, 0.06, seed=9)
    box = np.asarray(s.box, dtype=np.float64)
    q_np = s.q.copy()
    rc = 3.0
    if wide:
        # the same atoms in a box 2000 r_c wide along x (no image reaches across)
        box = box.copy()
        box[0] = 2000.0 * rc
    q = to_dev(q_np)
    pl = lj.lj_build_pairlist(q, box, s.rs, half)
    p1 = torch.zeros_like(q)
    ew = lj.lj_force_energy_virial(q, p1, pl, 0.01, rc, box, 1.1, 0.97, True).cpu().numpy()
    p2 = torch.zeros_like(q)
    e2 = lj.lj_force_energy(q, p2, pl, 0.01, rc, box, 1.1, 0.97, True).item()
    torch.cuda.synchronize()
    assert ew[0] == e2
    if half:
        assert float((p1 - p2).abs().max()) <= 1e-13 * float(p2.abs().max())
    else:
        assert torch.equal(p1, p2)
    rp, col = oracle_lib.pairlist(q_np, box, s.rs, half)
    want_w = oracle_lib.virial(q_np, rp, col, half, rc, box, 1.1, 0.97)
    want_e = oracle_lib.energy(q_np, rp, col, half, rc, box, 1.1, 0.97, True)
    assert abs(ew[1] - want_w) <= 1e-12 * abs(want_w)
    assert abs(ew[0] - want_e) <= 1e-12 * abs(want_e)
    again = lj.lj_force_energy_virial(q, torch.zeros_like(q), pl, 0.01, rc, box, 1.1, 0.97,
                                      True).cpu().numpy()
    assert np.array_equal(again, ew)
