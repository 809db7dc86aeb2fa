"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these compares the oracle with itself: each check comes from a
closed form of Eq. (1), a symbolic derivative, an independent route to the
same result, an invariant, or a number printed in the paper.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1806_05713_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _two_body(r, L=20.0, axis=0):
    q = np.zeros((2, 4))
    q[0, :3] = 5.0
    q[1, :3] = 5.0
    q[1, axis] += r
    return q, np.array([L, L, L])


def _impulse(oracle_lib, q, box, rs, rc, dt, half=True, eps=1.0, sigma=1.0):
    rp, col = oracle_lib.pairlist(q, box, rs, half)
    p = np.zeros((q.shape[0], 3))
    return oracle_lib.force(q, p, rp, col, half, dt, rc, box, eps, sigma), (rp, col)


# --------------------------------------------------------------------------
# Pair list
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k,rho,rs,half", [
    (2, 1.0, 3.3, True),    # L = 3.17 < 2 r_s is not allowed; use smaller r_s below
    (3, 1.0, 2.2, True),    # L = 4.76, 2 cells per axis
    (3, 1.0, 1.5, False),   # 3 cells per axis
    (4, 0.8, 2.6, True),    # 2 cells
    (5, 1.0, 3.3, False),   # L = 7.94: 2 cells at r_s = 3.3
    (6, 1.2, 1.3, True),    # 6 cells
])
def test_pairlist_cells_equals_brute(oracle_lib, k, rho, rs, half):
    s = inputs.fcc_system(k, rho, 0.07, seed=11 + k)
    L = s.box[0]
    if L < 2 * rs:
        rs = 0.45 * L
    a = oracle_lib.pairlist(s.q, s.box, rs, half, "brute")
    b = oracle_lib.pairlist(s.q, s.box, rs, half, "cells")
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    assert a[1].size > 0


def test_pairlist_single_cell_and_nonuniform_box(oracle_lib):
    rng = np.random.default_rng(3)
    box = np.array([6.7, 9.1, 13.4])
    q = np.zeros((300, 4))
    q[:, :3] = rng.random((300, 3)) * box
    for half in (True, False):
        a = oracle_lib.pairlist(q, box, 3.3, half, "brute")
        b = oracle_lib.pairlist(q, box, 3.3, half, "cells")
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_full_list_is_half_list_and_its_transpose(oracle_lib):
    s = inputs.fcc_system(5, 1.0, 0.05, seed=2)
    rph, ch = oracle_lib.pairlist(s.q, s.box, 3.3, True)
    rpf, cf = oracle_lib.pairlist(s.q, s.box, 3.3, False)
    ih = np.repeat(np.arange(s.n), np.diff(rph))
    half_pairs = set(zip(ih.tolist(), ch.tolist()))
    assert all(i < j for i, j in half_pairs)
    sym = half_pairs | {(j, i) for i, j in half_pairs}
    iF = np.repeat(np.arange(s.n), np.diff(rpf))
    assert sym == set(zip(iF.tolist(), cf.tolist()))
    assert cf.size == 2 * ch.size
    for i in range(s.n):  # rows ascending
        row = cf[rpf[i]:rpf[i + 1]]
        assert np.all(np.diff(row) > 0)


def test_mean_row_length_matches_sphere_volume(oracle_lib):
    """Uniform random positions: mean full row = (N-1)/V * (4/3) pi r_s^3."""
    rng = np.random.default_rng(5)
    n, L = 4000, 4000.0 ** (1.0 / 3.0)
    q = np.zeros((n, 4))
    q[:, :3] = rng.random((n, 3)) * L
    rp, col = oracle_lib.pairlist(q, np.array([L, L, L]), 3.3, False)
    expect = (n - 1) / L ** 3 * 4.0 / 3.0 * math.pi * 3.3 ** 3
    assert abs(col.size / n - expect) / expect < 0.01


def test_perfect_lattice_rows_equal_lattice_vector_count(oracle_lib):
    """Unjittered FCC: every full row holds exactly the number of FCC lattice
    vectors shorter than r_s, counted here by enumerating integer triples
    (in units of a/2) with an even sum."""
    s = inputs.fcc_system(8, 1.0, 0.0, seed=0, order="lattice")
    a = inputs.lattice_constant(1.0)
    rs = 3.3
    m = int(np.ceil(2 * rs / a)) + 1
    g = np.arange(-m, m + 1)
    v = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    v = v[(v.sum(1) % 2 == 0) & (np.abs(v).sum(1) > 0)]
    count = int(np.sum(np.sum((v * a / 2) ** 2, 1) < rs * rs))
    rp, col = oracle_lib.pairlist(s.q, s.box, rs, False)
    assert np.all(np.diff(rp) == count)
    rph, colh = oracle_lib.pairlist(s.q, s.box, rs, True)
    assert colh.size * 2 == count * s.n


def test_neighbour_count_in_paper_band(oracle_lib):
    """'approximately 55 to 80' j-atoms per i-atom (section Remainder Loop
    Elimination) at the benchmark density and cutoff: the half list holds
    about 56 in-cutoff and 75 in-search-range partners per atom."""
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    lo, hi = g["j_per_i_low"]["value"], g["j_per_i_high"]["value"]
    s = inputs.workload_small()
    rp, col = oracle_lib.pairlist(s.q, s.box, 3.3, True)
    rpc, colc = oracle_lib.pairlist(s.q, s.box, 3.0, True)
    assert lo <= colc.size / s.n <= hi
    assert lo <= col.size / s.n <= hi


def test_benchmark_workload_matches_paper(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    s = inputs.workload_paper()
    assert s.n == g["benchmark_n_atoms"]["value"]
    assert abs(s.n / np.prod(s.box) - g["benchmark_number_density"]["value"]) < 1e-12
    assert s.rc == g["benchmark_cutoff_sigma"]["value"]


# --------------------------------------------------------------------------
# Force: closed forms and the symbolic derivative of Eq. (1)
# --------------------------------------------------------------------------

def test_force_zero_at_potential_minimum(oracle_lib):
    dt = 0.01
    q, box = _two_body(2.0 ** (1.0 / 6.0))
    p, _ = _impulse(oracle_lib, q, box, 3.3, 3.0, dt)
    # |df r| at the minimum is 0 up to the rounding of (48 - 24 r^6).
    assert np.max(np.abs(p)) < 1e-13 * 48 * dt


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_force_at_sigma_is_24_dt_repulsive(oracle_lib, axis):
    """Algorithm 1 at r = 1: df = (48 - 24) dt = 24 dt, pushing the pair apart."""
    dt = 0.01
    q, box = _two_body(1.0, axis=axis)
    p, _ = _impulse(oracle_lib, q, box, 3.3, 3.0, dt)
    expect = np.zeros(3)
    expect[axis] = 24 * dt
    assert np.allclose(p[1], expect, rtol=1e-15, atol=1e-17)
    assert np.allclose(p[0], -expect, rtol=1e-15, atol=1e-17)


def test_force_matches_symbolic_derivative(oracle_lib):
    sp = pytest.importorskip("sympy")
    r, e, s = sp.symbols("r epsilon sigma", positive=True)
    V = 4 * e * ((s / r) ** 12 - (s / r) ** 6)          # Eq. (1)
    F = sp.lambdify((r, e, s), -sp.diff(V, r), "mpmath")  # radial force on j
    rng = np.random.default_rng(7)
    for _ in range(40):
        rr = float(rng.uniform(0.85, 2.95))
        ee = float(rng.uniform(0.5, 2.0))
        ss = float(rng.uniform(0.8, 1.2))
        dt = 0.01
        q, box = _two_body(rr, axis=int(rng.integers(3)))
        p, _ = _impulse(oracle_lib, q, box, 3.4, 3.0, dt, eps=ee, sigma=ss)
        got = np.linalg.norm(p[1]) * np.sign(p[1].sum())
        want = float(F(rr, ee, ss)) * dt
        assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (rr, ee, ss, got, want)


def test_minimum_image_across_boundary(oracle_lib):
    """A pair split by the periodic boundary interacts through the short image."""
    dt = 0.01
    L = 10.0
    q = np.zeros((2, 4))
    q[0, :3] = [0.3, 5.0, 5.0]
    q[1, :3] = [L - 0.7, 5.0, 5.0]   # image distance 1.0 along -x from atom 0
    p, _ = _impulse(oracle_lib, q, np.array([L, L, L]), 3.3, 3.0, dt)
    assert np.allclose(p[0], [24 * dt, 0, 0], rtol=1e-14)
    assert np.allclose(p[1], [-24 * dt, 0, 0], rtol=1e-14)


def test_margin_pairs_are_excluded(oracle_lib):
    """Pairs in the list beyond r_c contribute nothing (bookkeeping margin)."""
    q, box = _two_body(3.1)
    p, (rp, col) = _impulse(oracle_lib, q, box, 3.3, 3.0, 0.01)
    assert col.size == 1 and np.all(p == 0.0)


def test_search_margin_does_not_change_forces(oracle_lib):
    s = inputs.fcc_system(6, 1.0, 0.05, seed=5)
    p1, _ = _impulse(oracle_lib, s.q, s.box, 3.3, 3.0, 0.01)
    p0, _ = _impulse(oracle_lib, s.q, s.box, 3.0, 3.0, 0.01)
    assert np.allclose(p1, p0, rtol=0, atol=1e-14 * np.max(np.abs(p0)))


# --------------------------------------------------------------------------
# Force: invariants and independent routes
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small(oracle_lib):
    s = inputs.workload_small()
    rph, ch = oracle_lib.pairlist(s.q, s.box, 3.3, True)
    rpf, cf = oracle_lib.pairlist(s.q, s.box, 3.3, False)
    return s, (rph, ch), (rpf, cf)


def test_newton_third_law(oracle_lib, small):
    s, (rp, col), _ = small
    p = oracle_lib.force(s.q, np.zeros((s.n, 3)), rp, col, True, 0.01, 3.0, s.box)
    assert np.max(np.abs(p.sum(axis=0))) < 1e-13 * np.abs(p).sum()
    assert np.max(np.abs(p)) > 0.05


def test_half_list_equals_full_list(oracle_lib, small):
    s, (rph, ch), (rpf, cf) = small
    ph = oracle_lib.force(s.q, np.zeros((s.n, 3)), rph, ch, True, 0.01, 3.0, s.box)
    pf = oracle_lib.force(s.q, np.zeros((s.n, 3)), rpf, cf, False, 0.01, 3.0, s.box)
    assert np.max(np.abs(ph - pf)) < 1e-13 * np.max(np.abs(ph))


def test_force_accumulates_onto_existing_momenta(oracle_lib, small):
    s, (rp, col), _ = small
    p0 = np.random.default_rng(1).normal(size=(s.n, 3))
    a = oracle_lib.force(s.q, p0, rp, col, True, 0.01, 3.0, s.box)
    b = oracle_lib.force(s.q, np.zeros((s.n, 3)), rp, col, True, 0.01, 3.0, s.box)
    assert np.allclose(a, p0 + b, rtol=0, atol=1e-14)


def test_permutation_invariance(oracle_lib, small):
    s, (rp, col), _ = small
    perm = np.random.default_rng(9).permutation(s.n)
    q2 = s.q[perm]
    rp2, col2 = oracle_lib.pairlist(q2, s.box, 3.3, True)
    a = oracle_lib.force(s.q, np.zeros((s.n, 3)), rp, col, True, 0.01, 3.0, s.box)
    b = oracle_lib.force(q2, np.zeros((s.n, 3)), rp2, col2, True, 0.01, 3.0, s.box)
    assert np.max(np.abs(a[perm] - b)) < 1e-13 * np.max(np.abs(a))


def test_translation_invariance(oracle_lib, small):
    s, (rp, col), _ = small
    shift = np.array([3.7, -11.2, 0.9])
    q2 = s.q.copy()
    q2[:, :3] = inputs.wrap(q2[:, :3] + shift, s.box[0])
    rp2, col2 = oracle_lib.pairlist(q2, s.box, 3.3, True)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    a = oracle_lib.force(s.q, np.zeros((s.n, 3)), rp, col, True, 0.01, 3.0, s.box)
    b = oracle_lib.force(q2, np.zeros((s.n, 3)), rp2, col2, True, 0.01, 3.0, s.box)
    assert np.max(np.abs(a - b)) < 1e-10 * np.max(np.abs(a))


def test_eps_sigma_scaling_law(oracle_lib):
    """F(q; eps, sigma) in a box L with cutoff rc equals (eps/sigma) times the
    reduced-unit force at q/sigma, box L/sigma, cutoff rc/sigma."""
    s = inputs.fcc_system(5, 1.0, 0.05, seed=4)
    eps, sig = 1.7, 1.3
    qs = s.q.copy()
    qs[:, :3] *= sig
    box = s.box * sig
    rp, col = oracle_lib.pairlist(qs, box, 3.3 * sig, True)
    a = oracle_lib.forces(qs, rp, col, True, 3.0 * sig, box, eps, sig)
    rp1, col1 = oracle_lib.pairlist(s.q, s.box, 3.3, True)
    b = oracle_lib.forces(s.q, rp1, col1, True, 3.0, s.box)
    assert np.max(np.abs(a - eps / sig * b)) < 1e-12 * np.max(np.abs(a))


# --------------------------------------------------------------------------
# Energy
# --------------------------------------------------------------------------

def test_energy_closed_forms(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    for r, want in [(2.0 ** (1.0 / 6.0), g["lj_well_depth_at_minimum"]["value"]), (1.0, 0.0)]:
        q, box = _two_body(r)
        rp, col = oracle_lib.pairlist(q, box, 3.3, True)
        assert abs(oracle_lib.energy(q, rp, col, True, 3.0, box) - want) < 1e-15
    q, box = _two_body(1.5)
    rp, col = oracle_lib.pairlist(q, box, 3.3, True)
    v3 = 4.0 * (3.0 ** -12 - 3.0 ** -6)
    v15 = 4.0 * (1.5 ** -12 - 1.5 ** -6)
    assert abs(oracle_lib.energy(q, rp, col, True, 3.0, box, shifted=True) - (v15 - v3)) < 1e-15
    # eps, sigma: V(2^(1/6) sigma) = -eps
    sig, eps = 1.3, 2.5
    q, box = _two_body(2.0 ** (1.0 / 6.0) * sig)
    rp, col = oracle_lib.pairlist(q, box, 3.3 * sig, True)
    assert abs(oracle_lib.energy(q, rp, col, True, 3.0 * sig, box, eps, sig) + eps) < 1e-14


def test_energy_half_equals_full(oracle_lib, small):
    s, (rph, ch), (rpf, cf) = small
    a = oracle_lib.energy(s.q, rph, ch, True, 3.0, s.box)
    b = oracle_lib.energy(s.q, rpf, cf, False, 3.0, s.box)
    assert abs(a - b) < 1e-12 * abs(a)
    # energy per atom of an FCC LJ solid at rho = 1 lies near -7 (cohesive energy)
    assert -8.0 < a / s.n < -6.0


def test_force_is_minus_gradient_of_energy(oracle_lib):
    s = inputs.fcc_system(5, 1.0, 0.08, seed=21)
    rp, col = oracle_lib.pairlist(s.q, s.box, 3.3, True)
    F = oracle_lib.forces(s.q, rp, col, True, 3.0, s.box)
    h = 1e-5
    rng = np.random.default_rng(0)
    for _ in range(12):
        i, a = int(rng.integers(s.n)), int(rng.integers(3))
        qp, qm = s.q.copy(), s.q.copy()
        qp[i, a] += h
        qm[i, a] -= h
        ep = oracle_lib.energy(qp, rp, col, True, 3.0, s.box)
        em = oracle_lib.energy(qm, rp, col, True, 3.0, s.box)
        fd = -(ep - em) / (2 * h)
        assert abs(fd - F[i, a]) < 1e-6 * max(1.0, abs(F[i, a])), (i, a, fd, F[i, a])


@pytest.mark.parametrize("half", [True, False])
def test_virial_is_minus_scaling_derivative_of_energy(oracle_lib, half):
    """W = sum r F(r) = -dU/dlambda at lambda = 1 when every coordinate and
    the box are scaled by lambda (central differences of the shifted energy,
    whose pair set and shift stay fixed for small h)."""
    s = inputs.fcc_system(5, 0.9, 0.08, seed=23)
    rp, col = oracle_lib.pairlist(s.q, s.box, 3.3, half)
    W = oracle_lib.virial(s.q, rp, col, half, 3.0, s.box, 1.1, 0.95)
    h = 1e-6

    def U(lam):
        q = s.q.copy()
        q[:, :3] *= lam
        return oracle_lib.energy(q, rp, col, half, 3.0, np.asarray(s.box) * lam, 1.1, 0.95,
                                 shifted=True)
    fd = -(U(1 + h) - U(1 - h)) / (2 * h)
    assert abs(fd - W) < 1e-6 * abs(W), (fd, W)


def test_virial_closed_forms(oracle_lib):
    """One pair: r F(r) is zero at the potential minimum 2^(1/6) sigma and
    24 eps at r = sigma; beyond r_c it is not counted."""
    for r, want in ((2 ** (1 / 6), 0.0), (1.0, 24.0), (0.9, 24.0 * (2 * 0.9 ** -12 - 0.9 ** -6)),
                    (3.05, 0.0)):
        q, box = _two_body(r)
        rp, col = oracle_lib.pairlist(q, box, 3.3, True)
        W = oracle_lib.virial(q, rp, col, True, 3.0, box)
        assert abs(W - want) < 1e-12 * max(1.0, abs(want)), (r, W, want)


# --------------------------------------------------------------------------
# Adjoint
# --------------------------------------------------------------------------

def _loss(oracle_lib, q, rp, col, half, box, eps, sig, F_target):
    F = oracle_lib.forces(q, rp, col, half, 3.0, box, eps, sig)
    return np.mean((F - F_target) ** 2)


@pytest.mark.parametrize("half", [True, False])
def test_vjp_matches_central_differences(oracle_lib, half):
    s = inputs.fcc_system(4, 1.0, 0.1, seed=8)   # N = 256, L = 6.35
    rp, col = oracle_lib.pairlist(s.q, s.box, 3.1, half)
    Ft = oracle_lib.forces(s.q, rp, col, half, 3.0, s.box, 1.0, 1.0)
    eps, sig = 1.1, 0.97
    F = oracle_lib.forces(s.q, rp, col, half, 3.0, s.box, eps, sig)
    R = 2.0 * (F - Ft) / F.size
    gq, ge, gs = oracle_lib.force_vjp(s.q, R, rp, col, half, 3.0, s.box, eps, sig)
    h = 1e-6
    L = lambda q=s.q, e=eps, g=sig: _loss(oracle_lib, q, rp, col, half, s.box, e, g, Ft)
    fe = (L(e=eps + h) - L(e=eps - h)) / (2 * h)
    fs = (L(g=sig + h) - L(g=sig - h)) / (2 * h)
    assert abs(fe - ge) < 1e-6 * max(abs(fe), 1e-3), (fe, ge)
    assert abs(fs - gs) < 1e-6 * max(abs(fs), 1e-3), (fs, gs)
    rng = np.random.default_rng(1)
    scale = np.max(np.abs(gq))
    for _ in range(10):
        i, a = int(rng.integers(s.n)), int(rng.integers(3))
        qp, qm = s.q.copy(), s.q.copy()
        qp[i, a] += h
        qm[i, a] -= h
        fd = (L(q=qp) - L(q=qm)) / (2 * h)
        assert abs(fd - gq[i, a]) < 1e-5 * scale, (i, a, fd, gq[i, a])


# --------------------------------------------------------------------------
# Force-shifted truncation
# --------------------------------------------------------------------------

def _pair_at(r):
    q = np.zeros((2, 4))
    q[:, :3] = 10.0
    q[1, 0] += r
    return q


def test_fs_matches_symbolic_definition(oracle_lib):
    """V_fs(r) = V(r) - V(r_c) - (r - r_c) V'(r_c), differentiated by sympy:
    the impulse on the second atom of a pair along x is -V_fs'(r) dt, and
    the pair energy is V_fs(r)."""
    sympy = pytest.importorskip("sympy")
    r, rc, e, s = sympy.symbols("r r_c epsilon sigma", positive=True)
    V = 4 * e * ((s / r) ** 12 - (s / r) ** 6)
    Vfs = V - V.subs(r, rc) - (r - rc) * sympy.diff(V, r).subs(r, rc)
    F = sympy.lambdify((r, rc, e, s), -sympy.diff(Vfs, r))
    E = sympy.lambdify((r, rc, e, s), Vfs)
    box = np.array([20.0] * 3)
    for rv, rcv, ev, sv in [(1.0, 3.0, 1.0, 1.0), (1.3, 2.5, 1.2, 0.9), (2.9, 3.0, 1.0, 1.0),
                            (0.95, 4.0, 0.7, 1.1)]:
        q = _pair_at(rv)
        rp, col = oracle_lib.pairlist(q, box, rcv + 0.3, True)
        p = oracle_lib.force_fs(q, np.zeros((2, 3)), rp, col, True, 0.01, rcv, box, ev, sv)
        want = float(F(rv, rcv, ev, sv)) * 0.01
        assert abs(p[1, 0] - want) <= 1e-12 * max(1.0, abs(want))
        assert abs(p[0, 0] + want) <= 1e-12 * max(1.0, abs(want))
        got_e = oracle_lib.energy_fs(q, rp, col, True, rcv, box, ev, sv)
        assert abs(got_e - float(E(rv, rcv, ev, sv))) <= 1e-12 * max(1.0, abs(got_e))


def test_fs_force_and_energy_vanish_at_the_cutoff(oracle_lib):
    """The shifted force goes to zero linearly and the shifted energy
    quadratically as r -> r_c; the plain truncation jumps."""
    box = np.array([20.0] * 3)
    f, en, fp = [], [], []
    for d in (1e-2, 1e-3, 1e-4):
        q = _pair_at(3.0 - d)
        rp, col = oracle_lib.pairlist(q, box, 3.3, True)
        f.append(abs(oracle_lib.force_fs(q, np.zeros((2, 3)), rp, col, True, 1.0, 3.0, box)[1, 0]))
        fp.append(abs(oracle_lib.force(q, np.zeros((2, 3)), rp, col, True, 1.0, 3.0, box)[1, 0]))
        en.append(abs(oracle_lib.energy_fs(q, rp, col, True, 3.0, box)))
    assert 8 < f[0] / f[1] < 12 and 8 < f[1] / f[2] < 12
    assert 80 < en[0] / en[1] < 120 and 80 < en[1] / en[2] < 120
    assert min(fp) > 1e-3   # the plain force does not vanish at r_c
    q = _pair_at(3.0)      # at r_c exactly: excluded
    rp, col = oracle_lib.pairlist(q, box, 3.3, True)
    assert oracle_lib.energy_fs(q, rp, col, True, 3.0, box) == 0.0


def test_fs_force_is_minus_gradient_of_fs_energy(oracle_lib):
    s = inputs.fcc_system(5, 1.0, 0.08, seed=22)
    rp, col = oracle_lib.pairlist(s.q, s.box, 3.3, True)
    F = oracle_lib.force_fs(s.q, np.zeros((s.n, 3)), rp, col, True, 1.0, 3.0, s.box)
    h = 1e-5
    rng = np.random.default_rng(1)
    for _ in range(12):
        i, a = int(rng.integers(s.n)), int(rng.integers(3))
        qp, qm = s.q.copy(), s.q.copy()
        qp[i, a] += h
        qm[i, a] -= h
        fd = -(oracle_lib.energy_fs(qp, rp, col, True, 3.0, s.box) -
               oracle_lib.energy_fs(qm, rp, col, True, 3.0, s.box)) / (2 * h)
        assert abs(fd - F[i, a]) < 1e-6 * max(1.0, abs(F[i, a])), (i, a, fd, F[i, a])


def test_fs_newton_and_half_equals_full(oracle_lib, small):
    s, (rp, col), (rpf, colf) = small
    ph = oracle_lib.force_fs(s.q, np.zeros((s.n, 3)), rp, col, True, 0.01, 3.0, s.box)
    pf = oracle_lib.force_fs(s.q, np.zeros((s.n, 3)), rpf, colf, False, 0.01, 3.0, s.box)
    assert np.max(np.abs(ph.sum(axis=0))) < 1e-12 * np.abs(ph).sum()
    assert np.max(np.abs(ph - pf)) <= 1e-13 * np.max(np.abs(ph))
    eh = oracle_lib.energy_fs(s.q, rp, col, True, 3.0, s.box)
    ef = oracle_lib.energy_fs(s.q, rpf, colf, False, 3.0, s.box)
    assert abs(eh - ef) <= 1e-12 * abs(eh)


# --------------------------------------------------------------------------
# Row blocks and per-atom sums (the bounded CPU sample and the sampled
# parity checks at full size)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("half", [True, False])
def test_pairlist_rows_equal_brute_force_rows(oracle_lib, small, half):
    """A block of rows from the cell method equals the same rows of the
    O(N^2) definition; blocks of a partition concatenate to the whole list."""
    s = small[0]
    brute_rp, brute_col = oracle_lib.pairlist(s.q, s.box, 3.3, half, "brute")
    cuts = [0, 1, 997, 1500, 3999, s.n]
    cols = []
    for i0, i1 in zip(cuts[:-1], cuts[1:]):
        rp, col = oracle_lib.pairlist_rows(s.q, s.box, 3.3, half, i0, i1)
        want_rp = brute_rp[i0:i1 + 1] - brute_rp[i0]
        assert np.array_equal(rp, want_rp)
        assert np.array_equal(col, brute_col[brute_rp[i0]:brute_rp[i1]])
        cols.append(col)
    assert np.array_equal(np.concatenate(cols), brute_col)
    empty_rp, empty_col = oracle_lib.pairlist_rows(s.q, s.box, 3.3, half, 17, 17)
    assert empty_rp.tolist() == [0] and empty_col.size == 0


@pytest.mark.parametrize("half", [True, False])
def test_force_over_row_blocks_sums_to_whole_call(oracle_lib, small, half):
    """The momentum changes of a partition of the rows, each from zero, add up
    to the change of one call over the whole list (momentum changes add)."""
    s, lh, lf = small
    rp_all, col_all = lh if half else lf
    whole = oracle_lib.force(s.q, np.zeros((s.n, 3)), rp_all, col_all, half, 0.01, 3.0, s.box)
    total = np.zeros((s.n, 3))
    cuts = [0, 640, 2222, 3001, s.n]
    for i0, i1 in zip(cuts[:-1], cuts[1:]):
        rp, col = oracle_lib.pairlist_rows(s.q, s.box, 3.3, half, i0, i1)
        part = oracle_lib.force_rows(s.q, np.zeros((s.n, 3)), rp, col, half, 0.01, 3.0, s.box,
                                     i0, i1)
        if not half:   # a full-list block changes only its own rows
            outside = np.ones(s.n, dtype=bool)
            outside[i0:i1] = False
            assert not part[outside].any()
        total += part
    assert np.max(np.abs(total - whole)) <= 1e-13 * np.max(np.abs(whole))


def test_force_atoms_equals_list_force(oracle_lib, small):
    """The per-atom sum over all atoms equals the list-based call (half and
    full lists) on sampled atoms: two routes to the same definition."""
    s, (rph, ch), (rpf, cf) = small
    ph = oracle_lib.force(s.q, np.zeros((s.n, 3)), rph, ch, True, 0.01, 3.0, s.box)
    pf = oracle_lib.force(s.q, np.zeros((s.n, 3)), rpf, cf, False, 0.01, 3.0, s.box)
    idx = np.array([0, 1, 2, 1234, 2999, s.n - 1] +
                   list(np.random.default_rng(4).choice(s.n, 40, replace=False)))
    got = oracle_lib.force_atoms(s.q, idx, 0.01, 3.0, s.box)
    scale = np.max(np.abs(ph))
    assert np.max(np.abs(got - ph[idx])) <= 1e-13 * scale
    assert np.max(np.abs(got - pf[idx])) <= 1e-13 * scale


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_force_atoms_two_body_closed_form(oracle_lib, axis):
    """At r = sigma the impulse on atom 0 is -24 dt eps / sigma along d
    (repulsive), and nothing beyond r_c contributes."""
    q, box = _two_body(1.0, axis=axis)
    far = np.zeros((1, 4))
    far[0, :3] = 5.0
    far[0, axis] = 5.0 + 4.5          # 4.5 and 3.5 from the pair: beyond r_c = 3
    q3 = np.vstack([q, far])
    got = oracle_lib.force_atoms(q3, [0, 1], 0.01, 3.0, box)
    want = np.zeros(3)
    want[axis] = -24.0 * 0.01
    assert np.allclose(got[0], want, rtol=1e-15, atol=0)
    assert np.allclose(got[1], -want, rtol=1e-15, atol=0)
