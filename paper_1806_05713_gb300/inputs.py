"""Seeded synthetic LJ workloads.

This module only *places* particles: a face-centred-cubic (FCC) lattice, a
uniform jitter, a periodic wrap into [0, L) and a reordering of the particle
indices.  It contains none of the method's arithmetic (no pair list, no
distance, no force) and is the one module shared by the CUDA path's tests and
benchmark and by the CPU oracle's tests.

The benchmark condition of the paper (section "Benchmark Conditions") is an
FCC crystal of N = 119164 = 4*31^3 atoms at number density 1.0 with cutoff
3.0 sigma.  The same construction is used for every workload here: k^3 cubic
unit cells of side a = (4/rho)^(1/3), four basis sites per cell, box side
L = k*a, each coordinate jittered by an independent uniform draw on
[-delta, +delta].

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw k of stream s is mix64(key(seed, s) + (k+1)*gamma), with the
published increment gamma = 0x9E3779B97F4A7C15 and the published finaliser
constants.  A uniform double in [0, 1) takes the top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Named streams so that each kind of draw is independent of the others.
STREAM_JITTER = 1
STREAM_PERMUTE = 2
STREAM_SUBSAMPLE = 3
STREAM_SYSTEM_N = 4
STREAM_SYSTEM_RHO = 5
STREAM_SYSTEM_RC = 6
STREAM_SYSTEM_SEED = 7


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    base = np.uint64((int(seed) * 0x100000001B3 + int(stream) * 0x5851F42D4C957F2D) & 0xFFFFFFFFFFFFFFFF)
    return _mix64(np.array([base], dtype=np.uint64))[0]


def splitmix64_u64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Raw 64-bit draws offset .. offset+count-1 of (seed, stream)."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _key(seed, stream) + k * _GAMMA
    return _mix64(z)


def uniform01(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    u = splitmix64_u64(seed, stream, count, offset) >> np.uint64(11)
    return u.astype(np.float64) * (1.0 / 9007199254740992.0)


def lattice_constant(rho: float) -> float:
    """Side of the cubic FCC unit cell holding 4 atoms at number density rho."""
    return (4.0 / rho) ** (1.0 / 3.0)


def fcc_sites(k: int, a: float) -> np.ndarray:
    """The 4*k^3 FCC sites of a k x k x k block of cubic cells of side a.

    Site order: cell index x fastest, then y, then z; the four basis sites of
    one cell are consecutive.  This order is spatially coherent and is the
    "lattice" ordering.
    """
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    idx = np.arange(k, dtype=np.float64)
    cz, cy, cx = np.meshgrid(idx, idx, idx, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)  # x fastest
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    return sites * a


def wrap(x: np.ndarray, L: float) -> np.ndarray:
    """Periodic wrap into [0, L): x - L*floor(x/L), with L itself mapped to 0."""
    y = x - L * np.floor(x / L)
    y[y >= L] = 0.0
    y[y < 0.0] = 0.0
    return y


def _blocked_order(k: int, block: int) -> np.ndarray:
    """Particle order that walks the lattice in blocks of block^3 unit cells.

    Rows that are adjacent in this order are adjacent in space, which is what
    a cell-sorted particle order gives a force kernel (its j neighbours are
    shared between consecutive rows).
    """
    ncell = k * k * k
    c = np.arange(ncell)
    cx, cy, cz = c % k, (c // k) % k, c // (k * k)
    bx, by, bz = cx // block, cy // block, cz // block
    nb = (k + block - 1) // block
    bid = (bz * nb + by) * nb + bx
    inner = ((cz % block) * block + (cy % block)) * block + (cx % block)
    cell_order = np.lexsort((inner, bid))
    return (cell_order[:, None] * 4 + np.arange(4)[None, :]).ravel()


@dataclass
class LJSystem:
    """One periodic LJ configuration.

    q: (N, 4) float64, AoS4 {x, y, z, 0} positions wrapped into [0, L).
    box: (3,) float64 box sides.
    """
    q: np.ndarray
    box: np.ndarray
    rho: float
    rc: float = 3.0
    margin: float = 0.3
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.q.shape[0])

    @property
    def rs(self) -> float:
        return self.rc + self.margin


def _aos4(xyz: np.ndarray) -> np.ndarray:
    q = np.zeros((xyz.shape[0], 4), dtype=np.float64)
    q[:, :3] = xyz
    return q


def fcc_system(k: int, rho: float = 1.0, jitter: float = 0.05, seed: int = 0,
               order: str = "random", rc: float = 3.0, margin: float = 0.3) -> LJSystem:
    """k^3 FCC cells at density rho, jittered by U(-jitter, jitter), wrapped.

    order: "random" (a seeded random permutation of the particle indices),
    "cell" (blocks of 2^3 unit cells, spatially coherent) or "lattice"
    (generation order).
    """
    a = lattice_constant(rho)
    L = k * a
    xyz = fcc_sites(k, a)
    n = xyz.shape[0]
    if jitter:
        u = uniform01(seed, STREAM_JITTER, 3 * n).reshape(n, 3)
        xyz = xyz + jitter * (2.0 * u - 1.0)
    xyz = wrap(xyz, L)
    if order == "random":
        keys = splitmix64_u64(seed, STREAM_PERMUTE, n)
        perm = np.argsort(keys, kind="stable")
        xyz = xyz[perm]
    elif order == "cell":
        xyz = xyz[_blocked_order(k, 2)]
    elif order != "lattice":
        raise ValueError(f"unknown order {order!r}")
    return LJSystem(q=_aos4(xyz), box=np.array([L, L, L]), rho=rho, rc=rc, margin=margin,
                    meta={"k": k, "jitter": jitter, "seed": seed, "order": order})


def subsampled_system(n: int, rho: float, seed: int, jitter: float = 0.05,
                      rc: float = 3.0, margin: float = 0.3) -> LJSystem:
    """An FCC-derived system of exactly n atoms at density exactly rho.

    k = ceil((n/4)^(1/3)) cells per side, L = (n/rho)^(1/3), a = L/k; the
    4k^3 sites are jittered and wrapped, then n of them are kept, chosen
    without replacement by a seeded permutation.
    """
    k = max(1, math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-12))
    while 4 * k ** 3 < n:
        k += 1
    L = (n / rho) ** (1.0 / 3.0)
    a = L / k
    xyz = fcc_sites(k, a)
    m = xyz.shape[0]
    if jitter:
        u = uniform01(seed, STREAM_JITTER, 3 * m).reshape(m, 3)
        xyz = xyz + jitter * (2.0 * u - 1.0)
    xyz = wrap(xyz, L)
    keys = splitmix64_u64(seed, STREAM_SUBSAMPLE, m)
    keep = np.argsort(keys, kind="stable")[:n]
    xyz = xyz[keep]
    return LJSystem(q=_aos4(xyz), box=np.array([L, L, L]), rho=rho, rc=rc, margin=margin,
                    meta={"k": k, "jitter": jitter, "seed": seed, "order": "random"})


def batched_systems(nsys: int = 512, seed: int = 0, n_min: int = 500, n_max: int = 32000,
                    rho_lo: float = 0.8, rho_hi: float = 1.2, rcs=(2.5, 3.0),
                    margin: float = 0.3, jitter: float = 0.05) -> list[LJSystem]:
    """Many independent periodic systems of uneven size from one seed.

    N is log-uniform on [n_min, n_max] (rounded), rho uniform on
    [rho_lo, rho_hi], rc one of `rcs` with equal probability.
    """
    un = uniform01(seed, STREAM_SYSTEM_N, nsys)
    ur = uniform01(seed, STREAM_SYSTEM_RHO, nsys)
    uc = uniform01(seed, STREAM_SYSTEM_RC, nsys)
    sub = splitmix64_u64(seed, STREAM_SYSTEM_SEED, nsys)
    out = []
    for s in range(nsys):
        n = int(round(math.exp(math.log(n_min) + un[s] * (math.log(n_max) - math.log(n_min)))))
        rho = rho_lo + ur[s] * (rho_hi - rho_lo)
        rc = rcs[min(int(uc[s] * len(rcs)), len(rcs) - 1)]
        sysm = subsampled_system(n, rho, int(sub[s] & np.uint64(0x7FFFFFFF)), jitter=jitter,
                                 rc=rc, margin=margin)
        sysm.meta["index"] = s
        out.append(sysm)
    return out


# Named workloads (sizes as the paper's benchmark and its GB300 extensions).
def workload_small(seed: int = 0, order: str = "random") -> LJSystem:
    """N = 4,000: 10^3 FCC cells, rho = 1, jitter 0.05, rc 3.0, margin 0.3."""
    return fcc_system(10, 1.0, 0.05, seed, order)


def workload_paper(seed: int = 0, order: str = "random") -> LJSystem:
    """N = 119,164: 31^3 FCC cells, the paper's benchmark size, rho = 1."""
    return fcc_system(31, 1.0, 0.05, seed, order)


def workload_million(seed: int = 0, order: str = "random") -> LJSystem:
    """N = 1,048,576: 64^3 FCC cells at rho = 1."""
    return fcc_system(64, 1.0, 0.05, seed, order)


def workload_replicas(replicas: int = 64, k: int = 16, seed: int = 0) -> list[LJSystem]:
    """Independent replicas of 4*k^3 atoms at rho = 1 with jitter 0.1."""
    return [fcc_system(k, 1.0, 0.1, seed * 1000003 + r, "random") for r in range(replicas)]
