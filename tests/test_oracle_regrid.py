"""Pins of the oracle's regrid (Sec. 4.2, AMR policies: tags by charge
density, potential or electric field, grown by the buffer, marked as aligned
blocks of brick/2 cells, kept under proper nesting in the new coarser
level) against answers worked out by hand from the rules, and one invariant:

- a hierarchy tagged by density regrids onto itself by the same policy;
- lambda = 0 tags every cell, so level 1 is every block whose grown box
  stays two cells inside the domain: the central 16^3 fine cells of 16^3;
- a single potential peak (lambda = 0.9) and its buffer mark the blocks the
  3^3 neighbourhood touches;
- a single non-zero potential cell c makes |E_w| largest (= v / 2h) at the
  two face neighbours of c along w and zero at c, so lambda = 1 tags exactly
  those six cells.
"""
import numpy as np

import oracle
from paper_1812_03689_gb300 import inputs


def fine_mask_box(H, l=1):
    lo, hi, n = H.level_box(l)
    return tuple(lo), tuple(hi), n, bool((H.mask(l) > 0).all())


def test_density_regrid_is_a_fixed_point():
    w = inputs.workload("c1_small")
    parts = w.particles()
    H = oracle.OracleHierarchy(32, 2, particles=parts, tag_mode="rel", tag_lambda=0.1)
    assert H.nlevels == 3
    R = H.regrid("rel", 0.1, 2, particles=parts)
    assert R.nlevels == H.nlevels
    for l in range(H.nlevels):
        assert np.array_equal(R.mask(l), H.mask(l)), l
        assert np.array_equal(R.get(l, "rho"), H.get(l, "rho")), l


def test_lambda_zero_refines_every_nested_block():
    H = oracle.OracleHierarchy(16, 0)
    H.set(0, "phi", np.random.default_rng(1).normal(size=(16, 16, 16)))
    R = H.regrid("phi", 0.0, 1)
    assert R.nlevels == 2
    # blocks 1..2 of 0..3 per axis (4 coarse cells each) -> fine cells 8..23
    assert fine_mask_box(R) == ((8, 8, 8), (23, 23, 23), 16 ** 3, True)


def test_single_potential_peak():
    phi = np.zeros((16, 16, 16))
    phi[7, 6, 9] = 1.0          # cell (i, j, k) = (9, 6, 7)
    phi[3, 3, 3] = 0.5          # below 0.9 of the maximum
    for buffer, want in ((1, ((16, 8, 8), (23, 15, 23), 2 * 8 ** 3)), (0, ((16, 8, 8), (23, 15, 15), 8 ** 3))):
        H = oracle.OracleHierarchy(16, 0)
        H.set(0, "phi", phi)
        R = H.regrid("phi", 0.9, 1, buffer=buffer)
        lo, hi, n, full = fine_mask_box(R)
        assert (lo, hi, n) == want and full, (buffer, lo, hi, n)


def test_single_cell_field_policy():
    phi = np.zeros((16, 16, 16))
    phi[11, 4, 8] = 2.0         # cell c = (8, 4, 11)
    H = oracle.OracleHierarchy(16, 0)
    H.set(0, "phi", phi)
    H.average_down()
    H.efield()
    h = H.h(0)
    ex = H.get(0, "ex")
    assert np.isclose(np.abs(ex).max(), 2.0 / (2 * h)) and ex[11, 4, 8] == 0.0
    R = H.regrid("efield", 1.0, 1, buffer=0)
    # tagged: (7,4,11) -> block (1,1,2); (9,4,11), (8,5,11), (8,4,10) -> (2,1,2);
    # (8,3,11) -> (2,0,2) and (8,4,12) -> (2,1,3) are not nested (face blocks)
    m = R.mask(1) > 0
    lo, hi, n = R.level_box(1)
    assert (tuple(lo), tuple(hi), n) == ((8, 8, 16), (23, 15, 23), 2 * 8 ** 3) and m.all()


def _fine_blocks(R, l=1, bc=4):
    """Coarse blocks (bc^3 cells of level l-1) that level l of R covers."""
    lo, hi, _ = R.level_box(l)
    m = R.mask(l) > 0
    got = set()
    for k, j, i in zip(*np.nonzero(m)):
        c = (int(i + lo[0]) // 2, int(j + lo[1]) // 2, int(k + lo[2]) // 2)
        got.add(tuple(x // bc for x in c))
    return got


def test_density_threshold_hand_worked():
    # Eq. tag_charge (absolute: |rho| >= lambda) and the relative form of the
    # workloads (rho > lambda max rho, max over the signed values), on one
    # cell per nestable block of a 16^3 level 0 (blocks of 4 cells; only
    # blocks 1..2 per axis stay two cells inside the domain), buffer 0.
    lam = 0.5
    cells = {
        (5, 5, 5): 1.0,                          # the maximum          -> block (1, 1, 1)
        (9, 5, 5): 0.5,                          # exactly lambda * max -> block (2, 1, 1)
        (5, 9, 5): np.nextafter(0.5, 1.0),       # just above           -> block (1, 2, 1)
        (9, 9, 5): -2.0,                         # negative, |rho| = 2  -> block (2, 2, 1)
        (5, 5, 9): np.nextafter(0.5, 0.0),       # just below           -> block (1, 1, 2)
    }
    rho = np.zeros((16, 16, 16))
    for (i, j, k), v in cells.items():
        rho[k, j, i] = v
    want = {
        # relative: strict '>' (0.5 itself is not tagged), signed values (the
        # -2 cell is not tagged and does not set the maximum: were max|rho|
        # = 2 used, the threshold 1 would drop the just-above cell too)
        "rel": {(1, 1, 1), (1, 2, 1)},
        # absolute: '>=' on |rho| (0.5 and -2 are tagged, just below is not)
        "abs": {(1, 1, 1), (2, 1, 1), (1, 2, 1), (2, 2, 1)},
    }
    for policy, blocks in want.items():
        H = oracle.OracleHierarchy(16, 0)
        H.set(0, "rho", rho)
        R = H.regrid(policy, lam, 1, buffer=0)
        assert R.nlevels == 2, policy
        assert _fine_blocks(R) == blocks, (policy, _fine_blocks(R))
        lo, hi, n = R.level_box(1)
        assert n == len(blocks) * 8 ** 3, (policy, n)
