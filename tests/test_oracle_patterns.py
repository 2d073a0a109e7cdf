"""Pins of the oracle's ghost-interpolation pattern selection (Sec. 5.1,
Tab. bit_pattern, Tab. Lagrange_2d_linear, Eq. 2d_lagrange) against the
paper's printed tables and against polynomial reproduction."""
import numpy as np
import pytest

import hierarchies
import oracle
from conftest import golden_path


def _golden():
    rows = []
    for line in open(golden_path("bit_patterns.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        kind, case, bits, value = line.split()
        rows.append((kind, int(case), bits, int(value)))
    return rows


def test_printed_bit_strings_match_printed_values():
    # the table's two columns agree when the string is read MSB first
    for kind, case, bits, value in _golden():
        assert int(bits, 2) == value, (kind, case)


def test_oracle_tables_are_the_printed_ones():
    for kind, case, _bits, value in _golden():
        got = oracle.quad_pattern(case) if kind == "quad" else oracle.lin_pattern(case)
        assert got == value, (kind, case)


def _cells(value, w):
    return {(i, j) for j in range(w) for i in range(w) if value >> (i + w * j) & 1}


@pytest.mark.parametrize("kind,w,side,centre", [("quad", 5, 3, (2, 2)), ("lin", 3, 2, (1, 1))])
def test_patterns_are_full_blocks_through_the_centre(kind, w, side, centre):
    seen = set()
    for k, case, _bits, value in _golden():
        if k != kind:
            continue
        cells = _cells(value, w)
        i0 = min(i for i, _ in cells)
        j0 = min(j for _, j in cells)
        assert cells == {(i0 + a, j0 + b) for a in range(side) for b in range(side)}, case
        assert centre in cells, case
        seen.add((i0, j0))
    # the quadratic cases enumerate every 3x3 block position that holds the
    # centre; case 0 is the centred one (Fig. Lagrange_configurations)
    if kind == "quad":
        assert len(seen) == 9
        assert _cells(oracle.quad_pattern(0), 5) == {(i, j) for i in (1, 2, 3) for j in (1, 2, 3)}
    else:
        assert len(seen) == 4


def _notched():
    # a cube with an octant notched out: near its concave edges and corner
    # the transverse 5x5 surfaces meet covered cells, so shifted and corner
    # quadratic stencils are selected
    return oracle.OracleHierarchy(24, 1, boxes=hierarchies.notched(24))


def _in_plane_quadratic(rng):
    c = rng.normal(size=6)
    return lambda u, v: c[0] + c[1] * u + c[2] * v + c[3] * u * u + c[4] * u * v + c[5] * v * v


def test_ghost_step1_reproduces_quadratics_and_uses_shifted_cases():
    """Step 1 of the two-step interpolation is exact for any polynomial of
    degree <= 2 in the two transverse coordinates, whichever case is
    selected; the notched level exercises the shifted and corner cases."""
    H = _notched()
    rng = np.random.default_rng(3)
    cells0 = H.cells(0)
    h0 = H.h(0)
    h1 = H.h(1)
    m1 = H.mask(1)
    lo1 = H.level_box(1)[0]
    used_shapes = set()
    checked = 0
    for c in H.cells(1):
        for d in range(3):
            for s in (-1, 1):
                nb = c.copy()
                nb[d] += s
                rel = nb - lo1
                inside = np.all(rel >= 0) and np.all(rel < np.array(m1.shape[::-1]))
                if inside and m1[rel[2], rel[1], rel[0]] > 0:
                    continue
                cols, w, order = H.ghost_stencil(1, c, d, s)
                assert order == 2
                ax = [e for e in range(3) if e != d]
                p = _in_plane_quadratic(rng)
                xc = (cells0[cols] + 0.5) * h0
                target = (c + 0.5) * h1
                got = np.dot(w, p(xc[:, ax[0]], xc[:, ax[1]]))
                want = p(target[ax[0]], target[ax[1]])
                assert abs(got - want) < 1e-12 * (1 + abs(want)), (c, d, s)
                assert abs(w.sum() - 1.0) < 1e-14
                # which block of the 5x5 surface was used
                C = (c >> 1).copy()
                C[d] += s
                off = cells0[cols] - C
                used_shapes.add((int(off[:, ax[0]].min()), int(off[:, ax[1]].min())))
                checked += 1
    assert checked > 100
    assert (-1, -1) in used_shapes          # case 0
    assert (0, 0) in used_shapes            # a corner case (case 8)
    assert len(used_shapes) >= 4


def test_normal_step_weights_via_operator_rows():
    """Step 2 folds into A_nf: a fine cell with one coarse-fine face and its
    inward neighbour get A_nf entries (5 + 1/3)/h^2 and -(4/5)/h^2, and the
    coarse row part sums to -(8/15)/h^2 (the step-1 weights sum to one)."""
    H = oracle.OracleHierarchy(16, 1, boxes=[(1, (8, 8, 8), (23, 23, 23))])
    A = H.matrix(1, "A_nf").toarray()
    B = H.matrix(1, "B_crse").toarray()
    h2 = H.h(1) ** 2
    cells = H.cells(1)
    # a fine cell on the low-x face, away from edges
    r = int(np.where((cells[:, 0] == 8) & (cells[:, 1] == 15) & (cells[:, 2] == 15))[0][0])
    r1 = int(np.where((cells[:, 0] == 9) & (cells[:, 1] == 15) & (cells[:, 2] == 15))[0][0])
    assert A[r, r] * h2 == pytest.approx(5 + 1 / 3, abs=1e-13)
    assert A[r, r1] * h2 == pytest.approx(-4 / 5, abs=1e-13)
    assert B[r].sum() * h2 == pytest.approx(-8 / 15, abs=1e-13)


@pytest.mark.parametrize("width,order", [(2, 1), (1, 0)])
def test_channel_falls_back_in_table_order(width, order):
    """A channel two coarse cells wide leaves no 3x3 block of uncovered
    cells, so the linear table is used; one cell wide leaves no 2x2 block
    either, and the ghost falls back to the coarse value.  Linear stencils
    reproduce in-plane linear functions."""
    H = oracle.OracleHierarchy(24, 1, boxes=hierarchies.channel(24, width))
    st = H.ghost_stats()
    assert st["linear" if order == 1 else "constant"] > 0
    assert st["constant" if order == 1 else "linear"] == 0
    rng = np.random.default_rng(5)
    cells0 = H.cells(0)
    m1 = H.mask(1)
    lo1 = H.level_box(1)[0]
    seen = 0
    for c in H.cells(1):
        for d in range(3):
            for s in (-1, 1):
                nb = c.copy()
                nb[d] += s
                rel = nb - lo1
                inside = np.all(rel >= 0) and np.all(rel < np.array(m1.shape[::-1]))
                if inside and m1[rel[2], rel[1], rel[0]] > 0:
                    continue
                cols, w, o = H.ghost_stencil(1, c, d, s)
                if o != order:
                    continue
                seen += 1
                ax = [e for e in range(3) if e != d]
                a0, a1, a2 = rng.normal(size=3)
                xc = (cells0[cols] + 0.5) * H.h(0)
                t = (c + 0.5) * H.h(1)
                got = np.dot(w, a0 + a1 * xc[:, ax[0]] + a2 * xc[:, ax[1]])
                want = a0 + a1 * t[ax[0]] + a2 * t[ax[1]]
                if order == 1:
                    assert len(w) == 4
                    assert abs(got - want) < 1e-12 * (1 + abs(want))
                else:
                    assert len(w) == 1 and w[0] == 1.0
    assert seen > 0
