"""The FP64 force in AoS4, AoS8 (q and p in one 64-byte record) and SoA
layouts (lj_force_strided): same arithmetic, so full lists give identical
bits across layouts, and every layout matches the oracle."""
import numpy as np
import pytest
import torch

from paper_1806_05713_gb300 import inputs

pytestmark = pytest.mark.gpu


def _layouts(lj, s, pl, half, lanes=8):
    n = s.n
    q4 = torch.from_numpy(s.q).cuda()
    out = {}
    # AoS4 through lj_force (image-selected schedule with the same lanes)
    p = torch.zeros_like(q4)
    lj.lj_force(q4, p, pl, 0.01, s.rc, s.box, tpi=lj.LJ_SCHED_IMAGES | lanes)
    out["lj_force"] = p[:, :3].cpu().numpy()
    # AoS4 through the strided entry
    p = torch.zeros_like(q4)
    lj.lj_force_strided(q4, p, n, 4, 1, pl, 0.01, s.rc, s.box, lanes_per_row=lanes)
    out["aos4"] = p[:, :3].cpu().numpy()
    # AoS8: {qx, qy, qz, 0, px, py, pz, 0} per atom
    rec = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
    rec[:, :3] = q4[:, :3]
    lj.lj_force_strided(rec, rec, n, 8, 1, pl, 0.01, s.rc, s.box, lanes_per_row=lanes, p_offset=4)
    out["aos8"] = rec[:, 4:7].cpu().numpy()
    assert torch.equal(rec[:, :3], q4[:, :3]) and torch.all(rec[:, 3] == 0) and torch.all(rec[:, 7] == 0)
    # SoA: x[], y[], z[] back to back
    qs = q4[:, :3].t().contiguous()
    ps = torch.zeros_like(qs)
    lj.lj_force_strided(qs, ps, n, 1, n, pl, 0.01, s.rc, s.box, lanes_per_row=lanes)
    out["soa"] = ps.t().cpu().numpy()
    return out


@pytest.mark.parametrize("half", [True, False])
def test_layouts_agree_and_match_oracle(cuda_lib, oracle_lib, half):
    lj = cuda_lib
    s = inputs.workload_small()
    pl = lj.lj_build_pairlist(torch.from_numpy(s.q).cuda(), s.box, s.rs, half)
    out = _layouts(lj, s, pl, half)
    rp, col = oracle_lib.pairlist(s.q, s.box, s.rs, half)
    want = oracle_lib.force(s.q, np.zeros((s.n, 3)), rp, col, half, 0.01, s.rc, s.box)
    scale = np.max(np.abs(want))
    for name, got in out.items():
        assert np.max(np.abs(got - want)) <= 1e-12 * scale, name
    if not half:  # deterministic: identical bits in every layout
        for name in ("aos4", "aos8", "soa"):
            assert np.array_equal(out[name], out["lj_force"]), name


def test_strided_argument_checks(cuda_lib):
    lj = cuda_lib
    s = inputs.workload_small()
    q4 = torch.from_numpy(s.q).cuda()
    pl = lj.lj_build_pairlist(q4, s.box, s.rs, True)
    p = torch.zeros_like(q4)
    with pytest.raises(lj.LJError):
        lj.lj_force_strided(q4, p, s.n, 0, 1, pl, 0.01, s.rc, s.box)
    with pytest.raises(lj.LJError):
        lj.lj_force_strided(q4, p, s.n, 4, 1, pl, 0.01, s.rc, s.box, lanes_per_row=3)
