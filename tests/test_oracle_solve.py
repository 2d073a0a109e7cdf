"""Pins of the oracle's solver (Alg. 1-3) against answers it does not
compute itself:

- one level with homogeneous Dirichlet faces: the cell-centred 7-point
  operator with the -phi_0 ghost is diagonalised by the type-II discrete
  sine transform, eigenvalues (4/h^2) sum_d sin^2(pi k_d / (2 n)); the
  scipy DST solve of the same rho is the exact discrete answer;
- several levels: LAPACK's dense solve of the composite system L^comp phi =
  -rho on the uncovered cells (Sec. 5.3), assembled from the exported
  per-level blocks, is the exact discrete answer the V-cycles must reach.
"""
import numpy as np
import pytest
import scipy.fft
import scipy.sparse as sp

import hierarchies
import oracle


def dst_solve(rho, h):
    n = rho.shape
    k = [np.arange(1, m + 1) for m in n]
    lam = sum((4.0 / h ** 2) * np.sin(np.pi * kk / (2 * m)) ** 2
              for kk, m in zip(np.meshgrid(*k, indexing="ij"), n))
    return scipy.fft.idstn(scipy.fft.dstn(rho, type=2) / lam, type=2)


@pytest.mark.parametrize("n0", [8, 16, 24])
def test_single_level_matches_dst(n0):
    H = oracle.OracleHierarchy(n0, 0)
    rho = np.random.default_rng(n0).normal(size=(n0, n0, n0))
    H.set(0, "rho", rho)
    it, rel = H.solve(eps=1e-13, bottom_rtol=1e-15)
    want = dst_solve(rho, H.h(0))
    got = H.get(0, "phi")
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    assert rel[0] <= 1e-13


def composite_system(H):
    """Dense matrix of the composite system over the uncovered cells of
    every level (all cells of the finest level), rows in level order."""
    L = H.nlevels
    keep, off = [], [0]
    for l in range(L):
        m = H.to_rows(l, H.mask(l))
        keep.append(np.where(m == 1)[0] if l < L - 1 else np.arange(len(m)))
        off.append(off[-1] + len(keep[-1]))
    N = off[-1]
    A = np.zeros((N, N))
    for l in range(L):
        rows = keep[l]
        blocks = [(l, "A_comp" if l < L - 1 else "A_nf")]
        if l > 0:
            blocks.append((l - 1, "B_crse"))
        if l < L - 1:
            blocks.append((l + 1, "B_fine"))
        for lc, name in blocks:
            M = H.matrix(l, name).toarray()[rows]
            full_cols = M
            A[off[l]:off[l + 1], off[lc]:off[lc + 1]] = full_cols[:, keep[lc]]
            # nothing may couple to cells outside the composite domain
            dropped = np.setdiff1d(np.arange(M.shape[1]), keep[lc])
            assert np.abs(M[:, dropped]).max(initial=0.0) == 0.0, (l, name)
    return A, keep, off


@pytest.mark.parametrize("name", ["one_box", "two_levels", "notched", "channel"])
def test_composite_solve_matches_dense_direct(name):
    if name == "one_box":
        n0, lmax, boxes = 8, 1, [(1, (4, 4, 4), (11, 11, 11))]
    elif name == "two_levels":
        n0, lmax, boxes = 8, 2, [(1, (4, 4, 4), (11, 11, 11)), (2, (12, 12, 12), (19, 19, 19))]
    elif name == "notched":
        n0, lmax, boxes = 12, 1, hierarchies.notched(12)
    else:
        n0, lmax, boxes = 16, 1, hierarchies.channel(16, 2)
    H = oracle.OracleHierarchy(n0, lmax, boxes=boxes)
    rng = np.random.default_rng(21)
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


def test_vcycle_contracts():
    """Each V-cycle reduces the composite residual (a working multigrid
    cycle, not a divergent or stalled one)."""
    H = oracle.OracleHierarchy(32, 2, boxes=hierarchies.nested_centred(32))
    rng = np.random.default_rng(2)
    for l in range(H.nlevels):
        H.set(l, "rho", rng.normal(size=H.shape(l)))
    prev = H.residual().max()
    for k in range(4):
        it, rel = H.solve(eps=0.0, max_iter=1, warm=True)
        assert rel.max() < 0.5 * prev
        prev = rel.max()


def test_average_down_and_covered_values():
    """After the solve the covered cells hold the 8-cell averages of their
    children (Alg. 2 average down)."""
    H = oracle.OracleHierarchy(16, 1, boxes=hierarchies.centred(16))
    rng = np.random.default_rng(4)
    for l in range(2):
        H.set(l, "rho", rng.normal(size=H.shape(l)))
    H.solve(eps=1e-12)
    f = H.get(1, "phi")
    avg = f.reshape(f.shape[0] // 2, 2, f.shape[1] // 2, 2, f.shape[2] // 2, 2).mean(axis=(1, 3, 5))
    lo1 = H.level_box(1)[0] // 2
    c = H.get(0, "phi")[lo1[2]:lo1[2] + avg.shape[0], lo1[1]:lo1[1] + avg.shape[1], lo1[0]:lo1[0] + avg.shape[2]]
    assert np.abs(c - avg).max() < 1e-15 * np.abs(avg).max() * 10
