"""Plain double-precision CPU oracle for the truncated LJ force over a Verlet list.

TEST INFRASTRUCTURE ONLY.  The CUDA library never imports, links or runs
anything here; only the tests, the smoke check and the benchmark's CPU
baseline do.  See ``lj_oracle.c`` for the passages of the paper each function
follows and the readings taken where the paper is silent.

Parity status of each function (what pins it, in ``tests/test_oracle_*.py``;
``test_oracle_properties.py`` repeats the list, force, momentum, translation
and force-shifted pins on random gases in random boxes with hypothesis):

* pairlist (brute, cells): pinned -- the two independent routes agree as
  sets; mean row length against the closed-form sphere volume; the paper's
  55-80 neighbours per atom.
* force: pinned -- sympy's symbolic derivative of Eq. (1); two-body closed
  forms (zero at 2^(1/6) sigma, 24 dt at r = sigma); Newton's third law;
  F = -grad E by central differences; half list == full list; invariance
  under permutation and translation; the eps/sigma scaling law.
* energy: pinned -- V(2^(1/6) sigma) = -eps, V(sigma) = 0, the shift.
* virial: pinned -- minus the derivative of the energy under a uniform
  scaling of coordinates and box (central differences); two-body closed
  forms (zero at 2^(1/6) sigma, 24 eps at r = sigma).
* force_vjp: pinned -- central finite differences of the loss (h = 1e-6)
  built from ``forces`` alone.
* force_fs, energy_fs (force-shifted truncation): pinned -- sympy's
  derivative of V(r) - V(r_c) - (r - r_c) V'(r_c) for two-body pairs; force
  and energy vanish at r_c (linearly, quadratically); F = -grad E_fs by
  central differences; Newton's third law; half list == full list.
* pairlist_rows, force_rows (a block of rows, for the bounded CPU timing
  sample): pinned -- the rows equal those of the O(N^2) definition; the
  momentum changes of a partition of the rows add up to the whole call.
* force_atoms (per-atom sum over every other atom, no list; for sampled
  checks of systems too large to list on the CPU): pinned -- equals the
  list-based call on sampled atoms (half and full lists); the two-body
  closed form at r = sigma; atoms beyond r_c contribute nothing.
"""
from .oracle import (build, energy, energy_fs, force, force_atoms, force_fs,  # noqa: F401
                     force_rows, force_vjp, forces, pairlist, pairlist_rows, virial)
