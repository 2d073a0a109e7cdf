"""Pins of the oracle's periodic faces (Sec. 5.2 lists periodic faces
beside Dirichlet and Robin) against answers it does not compute itself:

- one level: the periodic 7-point operator is diagonalised by the discrete
  Fourier transform, eigenvalues (4/h^2) sum_d sin^2(pi k_d / n); the
  numpy FFT solve of the neutralised rho (zero mode dropped) is the exact
  mean-free answer;
- a manufactured solution Phi = sin(2 pi x) sin(2 pi y) sin(2 pi z)
  (-Lap Phi = 12 pi^2 Phi, periodic on the unit cube) is reached at second
  order;
- with refined levels, LAPACK's least-squares solve of the assembled
  (singular) composite system agrees up to a constant, and A_nf^0 is
  symmetric with the constants in its null space.
"""
import numpy as np
import pytest

import oracle
from test_oracle_solve import composite_system


def fft_solve(rho, h):
    n = rho.shape
    k = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    lam = sum((4.0 / h ** 2) * np.sin(np.pi * kk / m) ** 2 for kk, m in zip(k, n))
    lam[0, 0, 0] = 1.0
    f = np.fft.fftn(rho - rho.mean()) / lam
    f[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(f))


@pytest.mark.parametrize("n0", [8, 16])
def test_single_level_matches_fft(n0):
    H = oracle.OracleHierarchy(n0, 0, periodic=True)
    rho = np.random.default_rng(n0).normal(size=(n0, n0, n0))
    H.set(0, "rho", rho)
    it, rel = H.solve(eps=1e-13, bottom_rtol=1e-15)
    assert rel[0] <= 1e-13
    want = fft_solve(rho, H.h(0))
    assert np.linalg.norm(H.get(0, "phi") - want) <= 1e-12 * np.linalg.norm(want)


def test_manufactured_second_order():
    errs = []
    for n0 in (8, 16, 32):
        H = oracle.OracleHierarchy(n0, 0, periodic=True)
        X, Y, Z = H.centres(0)
        P = np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(2 * np.pi * Z)
        H.set(0, "rho", 12 * np.pi ** 2 * P)
        H.solve(eps=1e-12, bottom_rtol=1e-15)
        errs.append(np.abs(H.get(0, "phi") - P).max())
    assert errs[0] / errs[1] >= 3.3 and errs[1] / errs[2] >= 3.8, errs   # ratio -> 4


@pytest.mark.parametrize("boxes", [
    [(1, (4, 4, 4), (11, 11, 11))],
    [(1, (4, 4, 4), (11, 11, 11)), (2, (12, 12, 12), (19, 19, 19))],
])
def test_composite_solve_matches_least_squares(boxes):
    lmax = max(b[0] for b in boxes)
    H = oracle.OracleHierarchy(8, lmax, boxes=boxes, periodic=True)
    rng = np.random.default_rng(23)
    rhos = [rng.normal(size=H.shape(l)) * (H.mask(l) > 0) for l in range(H.nlevels)]
    for l in range(H.nlevels):
        H.set(l, "rho", rhos[l])
    it, rel = H.solve(eps=1e-12, max_iter=200, bottom_rtol=1e-15)
    assert rel.max() <= 1e-12
    A, keep, off = composite_system(H)
    vol = np.concatenate([np.full(len(keep[l]), H.h(l) ** 3) for l in range(H.nlevels)])
    b = np.concatenate([H.to_rows(l, H.get(l, "rho"))[keep[l]] for l in range(H.nlevels)])
    assert abs(vol @ b) <= 1e-13 * np.abs(b).max()         # neutralised
    want = np.linalg.lstsq(A, b, rcond=None)[0]
    want -= vol @ want                                      # mean-free
    got = np.concatenate([H.to_rows(l, H.get(l, "phi"))[keep[l]] for l in range(H.nlevels)])
    assert abs(vol @ got) <= 1e-13 * np.abs(got).max()
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_level0_operator_null_space():
    H = oracle.OracleHierarchy(6, 0, brick=4, periodic=True)
    A = H.matrix(0, "A_nf").toarray()
    assert np.abs(A - A.T).max() == 0.0
    assert np.abs(A @ np.ones(A.shape[0])).max() <= 1e-12 * np.abs(A).max()
    lam = np.linalg.eigvalsh(A)
    assert abs(lam[0]) <= 1e-10 * lam[-1] and lam[1] > 0
