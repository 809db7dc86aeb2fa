"""Property-based pins of the CPU oracle (hypothesis): random small systems
in random boxes, each checked against a route that does not share the
oracle's code path -- brute force against the cell method, forces against
central differences of the energy, the virial against the derivative of
the energy under scaling, conservation of momentum, invariance under
translation across the periodic boundary."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

SETTINGS = dict(max_examples=25, deadline=None, derandomize=True)


@st.composite
def gas(draw, min_n=2, max_n=48):
    """n atoms uniform in a box whose sides are at least 2 r_s."""
    n = draw(st.integers(min_n, max_n))
    rs = draw(st.floats(1.2, 3.3))
    sides = [draw(st.floats(2.0 * rs + 0.01, 4.0 * rs)) for _ in range(3)]
    seed = draw(st.integers(0, 2 ** 31 - 1))
    rng = np.random.default_rng(seed)
    q = np.zeros((n, 4))
    q[:, :3] = rng.random((n, 3)) * np.array(sides)
    return q, np.array(sides), rs


@settings(**SETTINGS)
@given(gas(), st.booleans())
def test_cells_equal_brute_force(oracle_lib, g, half):
    q, box, rs = g
    a = oracle_lib.pairlist(q, box, rs, half, "cells")
    b = oracle_lib.pairlist(q, box, rs, half, "brute")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def _spread(q, box, dmin=0.75):
    """Drop atoms closer than dmin to an earlier one (keeps forces moderate)."""
    keep = []
    for i in range(q.shape[0]):
        ok = True
        for j in keep:
            d = q[i, :3] - q[j, :3]
            d -= box * np.round(d / box)
            if np.dot(d, d) < dmin * dmin:
                ok = False
                break
        if ok:
            keep.append(i)
    return q[keep]


@settings(**SETTINGS)
@given(gas(min_n=3, max_n=30), st.floats(0.85, 1.2), st.floats(0.8, 1.3))
def test_force_is_minus_energy_gradient(oracle_lib, g, eps, sigma):
    q, box, rs = g
    q = _spread(q, box, 0.75 * sigma)
    rc = 0.9 * rs
    rp, col = oracle_lib.pairlist(q, box, rs, True)
    F = oracle_lib.forces(q, rp, col, True, rc, box, eps, sigma)
    h = 1e-6
    for i in range(min(q.shape[0], 4)):
        for a in range(3):
            qp, qm = q.copy(), q.copy()
            qp[i, a] += h
            qm[i, a] -= h
            # a move of 1e-6 changes no list decision unless a pair sits within 1e-6 of r_c
            fd = -(oracle_lib.energy(qp, rp, col, True, rc, box, eps, sigma) -
                   oracle_lib.energy(qm, rp, col, True, rc, box, eps, sigma)) / (2 * h)
            assert abs(fd - F[i, a]) <= 1e-5 * max(1.0, np.max(np.abs(F))), (i, a)


@settings(**SETTINGS)
@given(gas(min_n=2, max_n=40), st.booleans())
def test_momentum_is_conserved(oracle_lib, g, half):
    q, box, rs = g
    q = _spread(q, box, 0.7)
    rp, col = oracle_lib.pairlist(q, box, rs, half)
    p0 = np.random.default_rng(1).normal(size=(q.shape[0], 3))
    p = oracle_lib.force(q, p0, rp, col, half, 0.01, 0.95 * rs, box)
    dp = p - p0
    assert np.max(np.abs(dp.sum(axis=0))) <= 1e-12 * max(1.0, np.abs(dp).sum())


@settings(**SETTINGS)
@given(gas(min_n=2, max_n=40), st.floats(0.0, 1.0), st.floats(0.0, 1.0), st.floats(0.0, 1.0))
def test_translation_across_the_boundary(oracle_lib, g, tx, ty, tz):
    q, box, rs = g
    q = _spread(q, box, 0.7)
    rp, col = oracle_lib.pairlist(q, box, rs, False)
    F = oracle_lib.forces(q, rp, col, False, 0.95 * rs, box)
    qs = q.copy()
    qs[:, :3] = np.mod(q[:, :3] + np.array([tx, ty, tz]) * box, box)
    qs[:, :3] = np.where(qs[:, :3] >= box, 0.0, qs[:, :3])
    rps, cols = oracle_lib.pairlist(qs, box, rs, False)
    Fs = oracle_lib.forces(qs, rps, cols, False, 0.95 * rs, box)
    assert np.max(np.abs(Fs - F)) <= 1e-9 * max(1.0, np.max(np.abs(F)))


@settings(**SETTINGS)
@given(gas(min_n=3, max_n=30))
def test_force_shifted_is_minus_its_energy_gradient(oracle_lib, g):
    q, box, rs = g
    q = _spread(q, box, 0.75)
    rc = 0.9 * rs
    rp, col = oracle_lib.pairlist(q, box, rs, True)
    F = oracle_lib.force_fs(q, np.zeros((q.shape[0], 3)), rp, col, True, 1.0, rc, box)
    h = 1e-6
    for i in range(min(q.shape[0], 3)):
        for a in range(3):
            qp, qm = q.copy(), q.copy()
            qp[i, a] += h
            qm[i, a] -= h
            fd = -(oracle_lib.energy_fs(qp, rp, col, True, rc, box) -
                   oracle_lib.energy_fs(qm, rp, col, True, rc, box)) / (2 * h)
            assert abs(fd - F[i, a]) <= 1e-5 * max(1.0, np.max(np.abs(F))), (i, a)


@settings(**SETTINGS)
@given(gas(min_n=3, max_n=30), st.floats(0.85, 1.2), st.floats(0.8, 1.3), st.booleans())
def test_virial_is_minus_scaling_derivative(oracle_lib, g, eps, sigma, half):
    """W = -dU/dlambda for coordinates and box scaled by lambda (the shifted
    energy, so that the pair set and the shift stay fixed for small h)."""
    q, box, rs = g
    q = _spread(q, box, 0.75 * sigma)
    rc = 0.9 * rs
    rp, col = oracle_lib.pairlist(q, box, rs, half)
    W = oracle_lib.virial(q, rp, col, half, rc, box, eps, sigma)
    h = 1e-7

    def U(lam):
        qs = q.copy()
        qs[:, :3] *= lam
        return oracle_lib.energy(qs, rp, col, half, rc, box * lam, eps, sigma, shifted=True)
    fd = -(U(1 + h) - U(1 - h)) / (2 * h)
    scale = max(1.0, abs(W))
    assert abs(fd - W) < 1e-5 * scale, (fd, W)
