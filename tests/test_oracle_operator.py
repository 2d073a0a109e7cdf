"""Pins of the oracle's composite operator (Sec. 5.1 Eqs.
lap_flux_differencing, coarse_fluxes, flux_differencing, Eq. 2d_lagrange;
Sec. 5.3 matrices) against closed forms that do not restate it:

- polynomial exactness: the flux-differenced composite Laplacian applied to
  samples of a quadratic returns its constant Laplacian on every row whose
  stencil stays off the domain faces (the quadratic ghosts, the central
  fine-face fluxes and the averaged coarse-face flux are all exact there);
  with linear fall-back ghosts present, linear functions give zero;
- the discrete divergence theorem: the volume-weighted sum of L phi over the
  composite domain equals the flux through the domain faces, for any phi,
  because fine and coarse sides see the same interface fluxes.
"""
import numpy as np
import pytest

import hierarchies
import oracle


def _apply_L(H, values):
    """L phi on every level via Alg. 1 with rho = 0 (r = -A phi = L phi)."""
    for l in range(H.nlevels):
        H.set(l, "rho", 0.0)
        H.set(l, "phi", values[l])
    H.residual()
    return [H.get(l, "res") for l in range(H.nlevels)]


def _interior(H, l, margin):
    """Mask of cells at least `margin` cells (of level l) away from the
    domain faces."""
    lo, hi, _ = H.level_box(l)
    n = H.n0 * 2 ** l
    ax = [np.arange(lo[d], hi[d] + 1) for d in range(3)]
    ok = [(a >= margin) & (a <= n - 1 - margin) for a in ax]
    return ok[2][:, None, None] & ok[1][None, :, None] & ok[0][None, None, :]


def _quadratic(rng):
    c = rng.normal(size=10)

    def p(X, Y, Z):
        return (c[0] + c[1] * X + c[2] * Y + c[3] * Z + c[4] * X * X + c[5] * Y * Y + c[6] * Z * Z
                + c[7] * X * Y + c[8] * Y * Z + c[9] * X * Z)

    return p, 2.0 * (c[4] + c[5] + c[6])


CASES = {
    "centred": (32, 1, hierarchies.centred(32)),
    "nested": (32, 2, hierarchies.nested_centred(32)),
    "notched": (24, 1, hierarchies.notched(24)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_quadratic_exactness(name):
    n0, lmax, boxes = CASES[name]
    H = oracle.OracleHierarchy(n0, lmax, boxes=boxes)
    assert H.ghost_stats()["linear"] == 0 and H.ghost_stats()["constant"] == 0
    rng = np.random.default_rng(11)
    p, lap = _quadratic(rng)
    vals = [p(*H.centres(l)) for l in range(H.nlevels)]
    Lphi = _apply_L(H, vals)
    scale = max(np.abs(v).max() for v in vals) * (H.n0 * 2 ** lmax) ** 2
    for l in range(H.nlevels):
        m = H.mask(l)
        rows = (m == 1) if l < H.nlevels - 1 else (m > 0)
        rows &= _interior(H, l, 1 << l)
        assert rows.sum() > 0
        err = np.abs(Lphi[l][rows] - lap).max()
        assert err < 1e-11 * scale, (l, err)


@pytest.mark.parametrize("width", [2, 1])
def test_linear_exactness_with_fallbacks(width):
    H = oracle.OracleHierarchy(24, 1, boxes=hierarchies.channel(24, width))
    rng = np.random.default_rng(12)
    a = rng.normal(size=4)
    vals = [a[0] + a[1] * X + a[2] * Y + a[3] * Z for X, Y, Z in (H.centres(l) for l in range(H.nlevels))]
    Lphi = _apply_L(H, vals)
    for l in range(H.nlevels):
        m = H.mask(l)
        rows = ((m == 1) if l == 0 else (m > 0)) & _interior(H, l, 1 << l)
        # constant fall-back ghosts are exact only for constants
        if width == 1:
            vals_c = [np.full_like(v, a[0]) for v in vals]
            Lc = _apply_L(H, vals_c)
            assert np.abs(Lc[l][rows]).max() < 1e-9
        else:
            assert np.abs(Lphi[l][rows]).max() < 1e-9 * (H.n0 * 2 ** l) ** 2


@pytest.mark.parametrize("name", ["centred", "nested", "notched", "channel"])
def test_divergence_theorem(name):
    if name == "channel":
        n0, lmax, boxes = 24, 1, hierarchies.channel(24, 2)
    else:
        n0, lmax, boxes = CASES[name]
    H = oracle.OracleHierarchy(n0, lmax, boxes=boxes)
    rng = np.random.default_rng(13)
    vals = [rng.normal(size=H.shape(l)) for l in range(H.nlevels)]
    Lphi = _apply_L(H, vals)
    total = 0.0
    absum = 0.0
    for l in range(H.nlevels):
        m = H.mask(l)
        rows = (m == 1) if l < H.nlevels - 1 else (m > 0)
        v = H.h(l) ** 3 * Lphi[l][rows]
        total += v.sum()
        absum += np.abs(v).sum()
    # flux through the domain faces: homogeneous Dirichlet ghost -phi_0 gives
    # face flux -2 phi_0 / h on each boundary face of level 0
    phi0 = vals[0]
    h = H.h(0)
    bnd = 0.0
    for axis in range(3):
        for sl in (0, -1):
            face = np.take(phi0, sl, axis=axis)
            bnd += (h * h) * (-2.0 * face / h).sum()
    assert abs(total - bnd) < 1e-12 * absum


def test_level0_operator_is_symmetric_and_composite_rows_skip_covered_cells():
    H = oracle.OracleHierarchy(32, 2, boxes=hierarchies.nested_centred(32))
    A0 = H.matrix(0, "A_nf")
    assert abs(A0 - A0.T).max() < 1e-9
    for l in range(H.nlevels - 1):
        Ac = H.matrix(l, "A_comp").tocsc()
        covered = H.to_rows(l, H.mask(l)) == 2
        # no composite row reads a covered cell, and covered rows are empty
        assert abs(Ac[:, np.where(covered)[0]]).max() == 0
        assert abs(Ac.tocsr()[np.where(covered)[0]]).max() == 0
    for l in range(1, H.nlevels):
        Bc = H.matrix(l, "B_crse").tocsc()
        covered_c = H.to_rows(l - 1, H.mask(l - 1)) == 2
        assert abs(Bc[:, np.where(covered_c)[0]]).max() == 0
