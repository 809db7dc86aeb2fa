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
