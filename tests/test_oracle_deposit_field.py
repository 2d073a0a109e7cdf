"""Pins of the oracle's cloud-in-cell deposit, E = -G phi and gather
(Alg. 2 E-field line; the deposit/interpolate steps of Fig. sc_workflow):

- CIC conserves charge and the first moment exactly (the linear weights
  reproduce the particle position), puts a particle at a cell centre wholly
  into that cell and one at a cell vertex 1/8 into each of eight cells;
- central differences with the quadratic ghosts are exact for quadratic
  potentials, and CIC interpolation reproduces the resulting linear field.
"""
import numpy as np
import pytest

import hierarchies
import oracle
from paper_1812_03689_gb300 import inputs


def test_deposit_conserves_charge_and_dipole():
    w = inputs.workload("c1_small")
    x, y, z, q = w.particles()
    H = oracle.OracleHierarchy(32, 1, particles=(x, y, z, q), boxes=w.boxes)
    rho = H.get(0, "rho")
    X, Y, Z = H.centres(0)
    V = H.h(0) ** 3
    assert abs(rho.sum() * V - q.sum()) <= 1e-13 * q.sum()
    for C, p in ((X, x), (Y, y), (Z, z)):
        assert abs((rho * C).sum() * V - (q * p).sum()) <= 1e-13 * q.sum()


def test_deposit_fine_level_for_interior_particles():
    H = oracle.OracleHierarchy(16, 1, boxes=hierarchies.centred(16))
    rng = np.random.default_rng(8)
    # particles whose 8 fine nodes are inside level 1 (fine cells 8..23)
    p = rng.uniform(10.0 / 32, 22.0 / 32, size=(50, 3))
    q = rng.uniform(0.5, 1.5, size=50)
    H.deposit(p[:, 0], p[:, 1], p[:, 2], q)
    rho = H.get(1, "rho")
    X, Y, Z = H.centres(1)
    V = H.h(1) ** 3
    assert abs(rho.sum() * V - q.sum()) <= 1e-13 * q.sum()
    for d, C in enumerate((X, Y, Z)):
        assert abs((rho * C).sum() * V - (q * p[:, d]).sum()) <= 1e-13 * q.sum()


def test_deposit_centre_and_vertex():
    H = oracle.OracleHierarchy(8, 0)
    h = H.h(0)
    H.deposit(np.array([2.5 * h]), np.array([3.5 * h]), np.array([4.5 * h]), np.array([1.0]))
    rho = H.get(0, "rho")
    assert rho[4, 3, 2] == pytest.approx(1.0 / h ** 3, rel=1e-15)
    assert np.count_nonzero(rho) == 1
    H.deposit(np.array([3 * h]), np.array([3 * h]), np.array([5 * h]), np.array([1.0]))
    rho = H.get(0, "rho")
    assert np.count_nonzero(rho) == 8
    assert np.allclose(rho[4:6, 2:4, 2:4], 0.125 / h ** 3, rtol=1e-15, atol=0)


def test_deposit_mirror():
    H = oracle.OracleHierarchy(16, 0)
    rng = np.random.default_rng(9)
    p = rng.uniform(0.1, 0.9, size=(200, 3))
    q = np.ones(200)
    H.deposit(p[:, 0], p[:, 1], p[:, 2], q)
    a = H.get(0, "rho")
    H.deposit(1.0 - p[:, 0], p[:, 1], p[:, 2], q)
    b = H.get(0, "rho")
    assert np.abs(a[:, :, ::-1] - b).max() <= 1e-12 * np.abs(a).max()


def _quadratic(rng):
    c = rng.normal(size=10)
    p = lambda X, Y, Z: (c[0] + c[1] * X + c[2] * Y + c[3] * Z + c[4] * X * X + c[5] * Y * Y + c[6] * Z * Z
                         + c[7] * X * Y + c[8] * Y * Z + c[9] * X * Z)
    grad = lambda X, Y, Z: (c[1] + 2 * c[4] * X + c[7] * Y + c[9] * Z,
                            c[2] + 2 * c[5] * Y + c[7] * X + c[8] * Z,
                            c[3] + 2 * c[6] * Z + c[8] * Y + c[9] * X)
    return p, grad


def _away_from_covered(m):
    """Cells of the level that are neither covered nor face-adjacent to a
    covered cell (average down replaces covered values by 8-child means,
    which equal the point value only for linear functions)."""
    c = m == 2
    near = c.copy()
    for ax in range(3):
        near |= np.roll(c, 1, axis=ax) | np.roll(c, -1, axis=ax)
    return (m > 0) & ~near


def _inner(H, l):
    n = H.n0 * 2 ** l
    X, Y, Z = H.centres(l)
    lo, hi = 1.0 / n, 1 - 1.0 / n
    return (X > lo) & (X < hi) & (Y > lo) & (Y < hi) & (Z > lo) & (Z < hi)


CASES = {"centred": (16, 1, hierarchies.centred(16)), "nested": (32, 2, hierarchies.nested_centred(32)),
         "notched": (24, 1, hierarchies.notched(24))}


@pytest.mark.parametrize("name", list(CASES))
def test_field_exact_for_quadratic_phi(name):
    n0, lmax, boxes = CASES[name]
    H = oracle.OracleHierarchy(n0, lmax, boxes=boxes)
    rng = np.random.default_rng(10)
    p, grad = _quadratic(rng)
    for l in range(H.nlevels):
        H.set(l, "phi", p(*H.centres(l)))
    H.average_down()
    H.efield()
    for l in range(H.nlevels):
        rows = _away_from_covered(H.mask(l)) & _inner(H, l)
        assert rows.sum() > 0
        g = grad(*H.centres(l))
        for d, f in enumerate(("ex", "ey", "ez")):
            assert np.abs(H.get(l, f)[rows] + g[d][rows]).max() < 1e-9, (l, f)


@pytest.mark.parametrize("name", list(CASES) + ["channel"])
def test_field_and_gather_exact_for_linear_phi(name):
    n0, lmax, boxes = CASES[name] if name in CASES else (24, 1, hierarchies.channel(24, 2))
    H = oracle.OracleHierarchy(n0, lmax, boxes=boxes)
    a = np.random.default_rng(14).normal(size=4)
    for l in range(H.nlevels):
        X, Y, Z = H.centres(l)
        H.set(l, "phi", a[0] + a[1] * X + a[2] * Y + a[3] * Z)
    H.average_down()
    H.efield()
    for l in range(H.nlevels):
        rows = (H.mask(l) > 0) & _inner(H, l)
        for d, f in enumerate(("ex", "ey", "ez")):
            assert np.abs(H.get(l, f)[rows] + a[1 + d]).max() < 1e-9, (l, f)
    pts = np.random.default_rng(15).uniform(2.0 / n0, 1 - 2.0 / n0, size=(2000, 3))
    ex, ey, ez, ph = H.gather(pts[:, 0], pts[:, 1], pts[:, 2], with_phi=True)
    for d, e in enumerate((ex, ey, ez)):
        assert np.abs(e + a[1 + d]).max() < 1e-9
    assert np.abs(ph - (a[0] + pts @ a[1:])).max() < 1e-12


def test_gather_exact_for_quadratic_phi_single_level():
    H = oracle.OracleHierarchy(16, 0)
    rng = np.random.default_rng(16)
    p, grad = _quadratic(rng)
    H.set(0, "phi", p(*H.centres(0)))
    H.efield()
    pts = rng.uniform(2.0 / 16, 1 - 2.0 / 16, size=(500, 3))
    ex, ey, ez = H.gather(pts[:, 0], pts[:, 1], pts[:, 2])
    g = grad(pts[:, 0], pts[:, 1], pts[:, 2])
    for e, gd in zip((ex, ey, ez), g):
        assert np.abs(e + gd).max() < 1e-9
