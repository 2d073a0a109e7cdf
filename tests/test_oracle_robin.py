"""Pins of the oracle's Robin faces, the paper's open-boundary approximation
d phi/dn + phi/d = 0 discretised by central difference (Eq. robin_bc),
against answers the oracle does not compute itself:

- d -> 0 turns the Robin face into the homogeneous Dirichlet face: the solve
  matches the type-II DST solve of the same rho;
- a manufactured solution of the continuous problem: with k tan(k/2) = 1/d,
  Phi = X(x) X(y) X(z), X(t) = cos(k (t - 1/2)), meets the Robin condition
  on every face of the unit cube and -Lap Phi = 3 k^2 Phi, so the one-level
  solve of rho = 3 k^2 Phi converges to Phi at second order, and its field
  E = -grad phi to -grad Phi;
- with refined levels, the V-cycles reach LAPACK's dense solve of the
  assembled composite system, and the level-0 operator stays symmetric
  positive definite;
- physics: for a uniformly charged sphere at the centre, Robin faces at the
  distance of the face centres (d = 1/2, where the free-space field meets
  d phi/dr + phi/r = 0) give a potential much closer to the free-space
  closed form than Dirichlet faces do.
"""
import numpy as np
import pytest
import scipy.optimize

import oracle
from test_oracle_solve import composite_system, dst_solve


def robin_k(d):
    """Smallest k > 0 with k tan(k/2) = 1/d."""
    return scipy.optimize.brentq(lambda k: k * np.tan(k / 2) - 1.0 / d, 1e-9, np.pi - 1e-9)


def test_small_distance_is_dirichlet():
    n0 = 16
    rho = np.random.default_rng(5).normal(size=(n0, n0, n0))
    H = oracle.OracleHierarchy(n0, 0, robin_d=1e-14)
    H.set(0, "rho", rho)
    H.solve(eps=1e-13, bottom_rtol=1e-15)
    want = dst_solve(rho, H.h(0))
    assert np.linalg.norm(H.get(0, "phi") - want) <= 1e-10 * np.linalg.norm(want)


@pytest.mark.parametrize("d", [0.5, 1.7])
def test_manufactured_solution_second_order(d):
    k = robin_k(d)
    errs = []
    for n0 in (8, 16, 32):
        H = oracle.OracleHierarchy(n0, 0, robin_d=d)
        X, Y, Z = H.centres(0)
        cx, cy, cz = (np.cos(k * (t - 0.5)) for t in (X, Y, Z))
        sx = np.sin(k * (X - 0.5))
        H.set(0, "rho", 3 * k * k * cx * cy * cz)
        it, rel = H.solve(eps=1e-12, bottom_rtol=1e-15)
        assert rel[0] <= 1e-12
        H.average_down()
        H.efield()
        errs.append((np.abs(H.get(0, "phi") - cx * cy * cz).max(),
                     np.abs(H.get(0, "ex") - k * sx * cy * cz).max()))
    for a, b in zip(errs, errs[1:]):
        assert a[0] / b[0] >= 3.8, errs      # potential: second order
        assert a[1] / b[1] >= 3.5, errs      # field: second order
    assert errs[-1][0] <= 1e-3


@pytest.mark.parametrize("boxes", [
    [(1, (4, 4, 4), (11, 11, 11))],
    [(1, (4, 4, 4), (11, 11, 11)), (2, (12, 12, 12), (19, 19, 19))],
])
def test_composite_solve_matches_dense_direct(boxes):
    lmax = max(b[0] for b in boxes)
    H = oracle.OracleHierarchy(8, lmax, boxes=boxes, robin_d=0.5)
    rng = np.random.default_rng(22)
    rhos = [rng.normal(size=H.shape(l)) * (H.mask(l) > 0) for l in range(H.nlevels)]
    for l in range(H.nlevels):
        H.set(l, "rho", rhos[l])
    A, keep, off = composite_system(H)
    b = np.concatenate([H.to_rows(l, rhos[l])[keep[l]] for l in range(H.nlevels)])
    want = np.linalg.solve(A, b)
    it, rel = H.solve(eps=1e-13, max_iter=200, bottom_rtol=1e-15)
    assert rel.max() <= 1e-13
    got = np.concatenate([H.to_rows(l, H.get(l, "phi"))[keep[l]] for l in range(H.nlevels)])
    assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want)


def test_level0_operator_symmetric_positive_definite():
    H = oracle.OracleHierarchy(6, 0, brick=4, robin_d=0.3)
    A = H.matrix(0, "A_nf").toarray()
    assert np.abs(A - A.T).max() == 0.0
    lam = np.linalg.eigvalsh(A)
    assert lam.min() > 0.0
    # a corner cell has three Robin faces, a face cell one, an inner cell none
    h = H.h(0)
    alpha = (2 * 0.3 - h) / (2 * 0.3 + h)
    diag = np.diag(A) * h * h
    assert np.isclose(diag.max(), 6.0)
    assert np.isclose(diag.min(), 3.0 + 3 * (1.0 - alpha))


def test_open_boundary_approximates_free_space():
    n0, R = 32, 0.2
    err = {}
    for d in (0.0, 0.5):
        H = oracle.OracleHierarchy(n0, 0, robin_d=d)
        X, Y, Z = H.centres(0)
        r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
        H.set(0, "rho", np.where(r < R, 3 / (4 * np.pi * R ** 3), 0.0))
        H.solve(eps=1e-12)
        exact = np.where(r > R, 1 / (4 * np.pi * r), (3 - r * r / (R * R)) / (8 * np.pi * R))
        err[d] = np.abs(H.get(0, "phi") - exact).max() / exact.max()
    assert err[0.5] * 2.5 <= err[0.0], err
