"""The velocity-Verlet drivers' step bookkeeping, on the CPU: the library
calls are replaced by a stand-in that keeps their contract (lj_drift moves
and reports the step's largest displacement; lj_md_steps drifts, tests the
bound, empties the list once the margin is used up and kicks unless the
list is empty; lj_force kicks) and logs what the driver asked for.  The
host-checked driver and the device driver must issue the same drifts,
builds and kicks, in the same order, for any run split."""
import math

import numpy as np
import pytest
import torch

from paper_1806_05713_gb300 import lj as real_lj
from paper_1806_05713_gb300 import md


class _List:
    def __init__(self, half):
        self.half, self.empty, self.nnz = half, False, 1


class FakeLJ:
    """The calls md.VelocityVerlet makes, with the library's semantics on a
    scripted sequence of per-step largest displacements."""
    LJ_FP64, LJ_MIXED, LJ_DFLOAT, LJ_TPI_AUTO = 0, 1, 2, 0

    def __init__(self, disp):
        self.disp, self.n_drift, self.log = list(disp), 0, []

    # plumbing
    def _workspace(self, nbytes, device):
        return torch.empty(max(int(nbytes), 1), dtype=torch.uint8)

    def lj_force_workspace_bytes(self, n, box, precision):
        return 16

    def lj_force_energy_workspace_bytes(self, n):
        return 16

    lj_md_state_new = staticmethod(lambda device: torch.zeros(6, dtype=torch.float64))
    lj_md_state_read = staticmethod(real_lj.lj_md_state_read)

    # the path
    def lj_build_pairlist(self, q4, box, rs, half, reuse=None):
        self.log.append("build")
        return _List(half)

    def lj_force(self, q4, p4, plist, h, *args, **kw):
        if not plist.empty:
            self.log.append(("kick", h))

    def _next_disp(self):
        d = self.disp[self.n_drift]
        self.n_drift += 1
        self.log.append("drift")
        return d

    def lj_drift(self, q4, p4, dt, box, max_disp2):
        d = self._next_disp()
        max_disp2[0] = d * d
        return max_disp2

    def lj_md_steps(self, q4, p4, plist, k, dt, r_cut, r_search, box, eps, sigma, precision, tpi,
                    state, workspace, last_half_kick=False, q_build=None, energies=None):
        a = state.numpy()
        ints = a.view(np.int32)
        margin = r_search - r_cut
        for s in range(k):
            if not ints[8]:
                d = self._next_disp()
                a[0] = a[0] + math.sqrt(d * d)
                a[2] = d * d
                if 2.0 * a[0] >= margin:
                    ints[8] = 1
                    plist.empty = True
                else:
                    ints[9] += 1
            self.lj_force(q4, p4, plist, 0.5 * dt if (s == k - 1 and last_half_kick) else dt)
        return state


def _run(monkeypatch, disp, driver, splits, max_batch=64):
    fake = FakeLJ(disp)
    monkeypatch.setattr(md, "lj", fake)
    q = torch.zeros((4, 4), dtype=torch.float64)
    vv = md.VelocityVerlet(q, torch.zeros_like(q), [10.0, 10.0, 10.0], 3.0, 0.3, 0.01,
                           driver=driver)
    vv.max_batch = max_batch
    for n in splits:
        vv.run(n)
    return fake.log, vv.rebuilds


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("splits", [(50,), (1, 1, 30, 7), (13, 40), (2,) * 20])
def test_drivers_issue_the_same_steps(monkeypatch, seed, splits):
    rng = np.random.default_rng(seed)
    # per-step fastest-atom displacement: smooth, bursty or with long quiet spells
    kind = seed % 3
    n = sum(splits) + 5
    if kind == 0:
        disp = rng.uniform(0.005, 0.03, n)
    elif kind == 1:
        disp = np.where(rng.random(n) < 0.2, 0.2, 0.004)
    else:
        disp = np.where(np.arange(n) % 17 < 3, 0.05, 0.0)
    host, rb_host = _run(monkeypatch, disp, "host", splits)
    for max_batch in (1, 3, 64):
        dev, rb_dev = _run(monkeypatch, disp, "device", splits, max_batch)
        assert dev == host
        assert rb_dev == rb_host


def test_every_run_ends_with_a_half_kick(monkeypatch):
    disp = np.full(40, 0.01)
    log, _ = _run(monkeypatch, disp, "device", (10, 10))
    kicks = [e[1] for e in log if isinstance(e, tuple)]
    # opening half kick, 9 full kicks, closing half kick; twice
    assert kicks == [0.005] + [0.01] * 9 + [0.005] + [0.005] + [0.01] * 9 + [0.005]
    assert log.count("drift") == 20


def test_a_step_larger_than_the_margin_rebuilds_every_step(monkeypatch):
    disp = np.full(12, 0.5)          # 2 * 0.5 >= 0.3 at every step
    log, rebuilds = _run(monkeypatch, disp, "device", (6,))
    assert rebuilds == 1 + 6
    # each drift is followed by a build before its kick
    body = log[2:]                   # the first build and the opening half kick
    for s in range(6):
        assert body[3 * s: 3 * s + 3] == ["drift", "build", ("kick", 0.01 if s < 5 else 0.005)]
