"""Molecular dynamics around the force kernel: velocity Verlet (unit mass)
with the bookkeeping method of the paper's section "Verlet List and
Bookkeeping Method".

The list is built with search length r_s = r_c + margin and reused while
twice a bound on the largest displacement since the build stays below the
margin; then it is rebuilt.  The bound is the paper's fastest-atom one
(the sum over steps of the largest |dt p|) or, optionally, the largest
displacement |q - q_build| itself.  The kick and drift of consecutive
steps are merged (leapfrog form of velocity Verlet), so each step is one
drift and one force call -- the force kernel applies the kick directly
(Algorithm 1 updates the momenta with dt).

Two drivers.  The device driver (the plain truncation) runs the steps
through ``lj_md_steps``: batches of steps enqueued at once, the validity
test taken on the device (a list whose margin is used up is emptied there,
so the steps queued after it do nothing), and one read of the bookkeeping
state per batch; the batch length is predicted from the last step's
displacement so that few queued steps go unused.  The host driver (and the
force-shifted truncation) takes one ``lj_drift`` and one force call per
step with the test on the host.  Host-side orchestration only: every step
of the computation runs in the library's kernels.
"""
from __future__ import annotations

import math

import torch

from . import lj


class VelocityVerlet:
    """Integrates q4, p4 (device, AoS4, updated in place)."""

    def __init__(self, q4: torch.Tensor, p4: torch.Tensor, box, r_cut: float, margin: float,
                 dt: float, eps: float = 1.0, sigma: float = 1.0, precision: int = lj.LJ_FP64,
                 tpi: int = lj.LJ_TPI_AUTO, half: bool = True, truncation: str = "plain",
                 driver: str = "device", criterion: str = "fastest_atom"):
        """truncation: "plain" (Eq. (1) cut at r_c, the paper's choice) or
        "force_shifted" (the pair force taken to zero at r_c; FP64 only).
        driver: "device" (steps queued in batches through lj_md_steps; the
        plain truncation) or "host" (the validity test on the host after
        every drift).  criterion: "fastest_atom" (the paper's: the sum over
        steps of the fastest atom's step) or "displacement" (the largest
        displacement of any atom since the build, a tighter bound; device
        driver only)."""
        if truncation not in ("plain", "force_shifted"):
            raise ValueError("truncation must be 'plain' or 'force_shifted'")
        if driver not in ("device", "host"):
            raise ValueError("driver must be 'device' or 'host'")
        if criterion not in ("fastest_atom", "displacement"):
            raise ValueError("criterion must be 'fastest_atom' or 'displacement'")
        if truncation == "force_shifted":
            driver = "host"
        if criterion == "displacement" and driver != "device":
            raise ValueError("the displacement criterion needs the device driver and the plain "
                             "truncation")
        self.driver, self.criterion = driver, criterion
        if truncation == "force_shifted" and precision != lj.LJ_FP64:
            raise ValueError("the force-shifted truncation is FP64 only")
        self.truncation = truncation
        self.q4, self.p4 = q4, p4
        self.box = [float(x) for x in box]
        self.r_cut, self.dt = float(r_cut), float(dt)
        self.r_search = self.r_cut + float(margin)
        self.margin = self.r_search - self.r_cut   # the margin the built list has
        self.eps, self.sigma = float(eps), float(sigma)
        self.precision, self.tpi, self.half = int(precision), int(tpi), bool(half)
        self.plist = None
        self.rebuilds = 0
        self.moved = 0.0          # fastest-atom displacement bound since the last build
        self.max_disp2 = torch.zeros(1, dtype=torch.float64, device=q4.device)
        self.ws = lj._workspace(lj.lj_force_workspace_bytes(q4.shape[0], self.box, self.precision),
                                q4.device)
        self._fsws = (lj._workspace(lj.lj_force_shifted_workspace_bytes(q4.shape[0]), q4.device)
                      if truncation == "force_shifted" else None)
        self._half_kicked = False
        self._md_state = lj.lj_md_state_new(q4.device)
        self._q_build = q4.clone() if criterion == "displacement" else None
        self._mdws = None         # lj_md_steps workspace with per-step energies
        self.max_batch = 64       # steps enqueued per read of the device state, at most
        self._rebuild()

    def _rebuild(self):
        self.plist = lj.lj_build_pairlist(self.q4, self.box, self.r_search, self.half,
                                          reuse=self.plist)
        self.rebuilds += 1
        self.moved = 0.0
        self._md_state.zero_()
        if self._q_build is not None:
            self._q_build.copy_(self.q4)

    def _kick(self, h: float, energy_out: torch.Tensor | None = None):
        if self.truncation == "force_shifted":
            lj.lj_force_shifted(self.q4, self.p4, self.plist, h, self.r_cut, self.box, self.eps,
                                self.sigma, out=energy_out, workspace=self._fsws)
        elif energy_out is not None:
            # the FP64 force pass that also returns U(q) (shifted potential)
            lj.lj_force_energy(self.q4, self.p4, self.plist, h, self.r_cut, self.box, self.eps,
                               self.sigma, True, out=energy_out, workspace=self._ews)
        else:
            lj.lj_force(self.q4, self.p4, self.plist, h, self.r_cut, self.box, self.eps,
                        self.sigma, self.precision, self.tpi, workspace=self.ws)

    def run(self, steps: int, energies: torch.Tensor | None = None):
        """Advance `steps` steps; p4 ends at the same time as q4.  If
        `energies` (a device tensor of `steps` doubles) is given, the force
        passes also write the potential energy U(q(t_k)) of each new position
        into it (FP64 form; shifted, or force-shifted with that truncation)."""
        if steps <= 0:
            return
        if energies is not None:
            self._ews = lj._workspace(lj.lj_force_energy_workspace_bytes(self.q4.shape[0]),
                                      self.q4.device)
        if not self._half_kicked:
            self._kick(0.5 * self.dt)              # p(t + dt/2)
        if self.driver == "device":
            self._run_on_device(steps, energies)
        else:
            self._run_host_checked(steps, energies)
        self._half_kicked = False

    def _run_on_device(self, steps: int, energies: torch.Tensor | None):
        """`steps` leapfrog steps through lj_md_steps, the last with a half kick."""
        # the device state continues the host's bound across run() calls
        self._md_state.zero_()
        self._md_state[0] = self.moved
        prec, tpi, ws = self.precision, self.tpi, self.ws
        if energies is not None:                # the FP64 force-and-energy pass, as _kick's
            prec, tpi = lj.LJ_FP64, lj.LJ_TPI_AUTO
            if self._mdws is None:
                n = self.q4.shape[0]
                self._mdws = lj._workspace(max(lj.lj_force_workspace_bytes(n, self.box, prec),
                                               lj.lj_force_energy_workspace_bytes(n)),
                                           self.q4.device)
            ws = self._mdws
        done, base, batch = 0, 0, 8
        while done < steps:
            k = min(batch, steps - done)
            lj.lj_md_steps(self.q4, self.p4, self.plist, k, self.dt, self.r_cut, self.r_search,
                           self.box, self.eps, self.sigma, prec, tpi, state=self._md_state,
                           workspace=ws, last_half_kick=done + k == steps, q_build=self._q_build,
                           energies=None if energies is None else energies[done:done + k])
            st = lj.lj_md_state_read(self._md_state)
            done += st["steps"] - base
            base = st["steps"]
            if st["stale"]:
                # positions one drift ahead: rebuild, then the kick that step owes
                self._rebuild()
                self._kick(0.5 * self.dt if done + 1 == steps else self.dt,
                           None if energies is None else energies[done:done + 1])
                done += 1
                base = 0
                self.moved = 0.0
            else:
                self.moved = st["moved"]
            # steps until the margin is used up at the last step's pace, plus one
            step = math.sqrt(st["last_disp2"])
            left = 0.5 * self.margin - self.moved
            batch = self.max_batch if step == 0.0 else int(min(self.max_batch, left / step + 2))
            batch = max(1, batch)

    def _run_host_checked(self, steps: int, energies: torch.Tensor | None):
        for s in range(steps):
            lj.lj_drift(self.q4, self.p4, self.dt, self.box, self.max_disp2)
            self.moved += math.sqrt(float(self.max_disp2.item()))
            if 2.0 * self.moved >= self.margin:
                self._rebuild()
            last = s == steps - 1
            self._kick(0.5 * self.dt if last else self.dt,
                       None if energies is None else energies[s:s + 1])

    def kinetic_energy(self) -> float:
        return 0.5 * float((self.p4[:, :3] ** 2).sum())

    def pressure(self) -> float:
        """(2 K + W) / (3 V) with the pair virial W of the plain truncation
        (one FP64 force-and-energy pass with dt = 0 on scratch momenta)."""
        out = lj.lj_force_energy_virial(self.q4, torch.zeros_like(self.p4), self.plist, 0.0,
                                        self.r_cut, self.box, self.eps, self.sigma)
        W = float(out[1].item())
        V = self.box[0] * self.box[1] * self.box[2]
        return (2.0 * self.kinetic_energy() + W) / (3.0 * V)

    def potential_energy(self, shifted: bool = True) -> float:
        """The truncated potential energy (shifted by V(r_c) or not); with the
        force-shifted truncation, its energy (a force pass with dt = 0)."""
        if self.truncation == "force_shifted":
            out = torch.empty(1, dtype=torch.float64, device=self.q4.device)
            lj.lj_force_shifted(self.q4, torch.zeros_like(self.p4), self.plist, 0.0, self.r_cut,
                                self.box, self.eps, self.sigma, out=out, workspace=self._fsws)
            return float(out.item())
        return float(lj.lj_energy(self.q4, self.plist, self.r_cut, self.box, self.eps, self.sigma,
                                  shifted).item())
