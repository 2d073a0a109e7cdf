"""Physics pins of the oracle: the symmetry problem of Sec. 6.1 and the
charged sphere of Sec. 6.2 (closed-form potential), plus second-order
convergence to a smooth radial closed form."""
import math

import numpy as np
import pytest
from scipy.special import erf

import hierarchies
import oracle
from conftest import golden_path


def test_symmetry_problem():
    """Three centred levels, rho = 1, 1.5, 2 on levels 0, 1, 2 (Sec. 6.1):
    phi is mirror symmetric and E mirror antisymmetric about the centre."""
    H = oracle.OracleHierarchy(32, 2, boxes=hierarchies.nested_centred(32))
    for l, r in enumerate((1.0, 1.5, 2.0)):
        H.set(l, "rho", r * (H.mask(l) > 0))
    it, rel = H.solve(eps=1e-14, max_iter=100, bottom_rtol=1e-16)
    for l in range(H.nlevels):
        phi = H.get(l, "phi")
        scale = np.abs(phi).max()
        for ax in range(3):
            assert np.abs(phi - np.flip(phi, axis=2 - ax)).max() <= 1e-12 * scale
        for d, f in enumerate(("ex", "ey", "ez")):
            e = H.get(l, f)
            es = np.abs(e).max()
            assert np.abs(e + np.flip(e, axis=2 - d)).max() <= 1e-11 * es
            for ax in range(3):
                if ax != d:
                    assert np.abs(e - np.flip(e, axis=2 - ax)).max() <= 1e-11 * es


def _golden_sphere():
    vals = {}
    for line in open(golden_path("sphere_paper.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def sphere_phi(r, Q, R, eps0=1.0):
    """Potential of a uniformly charged sphere (closed form of Sec. 6.2)."""
    k = Q / (4 * math.pi * eps0)
    r = np.asarray(r, dtype=float)
    return np.where(r > R, k / np.maximum(r, 1e-300), k * (3 - (r / R) ** 2) / (2 * R))


def sphere_E(r, Q, R, eps0=1.0):
    k = Q / (4 * math.pi * eps0)
    r = np.asarray(r, dtype=float)
    return np.where(r > R, k / np.maximum(r, 1e-300) ** 2, k * r / R ** 3)


def test_sphere_closed_form_reproduces_paper_values():
    g = _golden_sphere()
    eps0 = 8.8541878128e-12
    R = g["radius_m"]
    Q = g["n_particles"] * 4 * math.pi * eps0 * R ** 2 * g["charge_factor"]
    assert sphere_E(R, Q, R, eps0) == pytest.approx(g["peak_field_V_per_m"], rel=1e-12)
    assert sphere_phi(0.0, Q, R, eps0) == pytest.approx(g["centre_potential_V"], rel=1e-12)
    # continuity at the surface
    assert sphere_phi(R * (1 - 1e-12), Q, R, eps0) == pytest.approx(sphere_phi(R * (1 + 1e-12), Q, R, eps0))


def fold_dirichlet(H, rho0, g):
    """Inhomogeneous Dirichlet data g on the faces of level 0, folded into
    the right-hand side: the ghost 2 g - phi_0 adds 2 g / h^2 per face."""
    b = rho0.copy()
    h = H.h(0)
    n = H.n0
    c = (np.arange(n) + 0.5) * h
    for axis in range(3):
        for side, xf in ((0, 0.0), (n - 1, 1.0)):
            idx = [slice(None)] * 3
            idx[2 - axis] = side
            others = [c, c]
            A, B = np.meshgrid(*others, indexing="ij")
            pts = [None, None, None]
            pts[axis] = np.full_like(A, xf)
            o = [a for a in range(3) if a != axis]
            # dense layout is [k, j, i]: the two remaining array axes in
            # order are (z or y) then (y or x)
            pts[o[1]], pts[o[0]] = A, B
            b[tuple(idx)] += 2.0 * g(*pts) / h ** 2
    return b


def _sphere_rho(H, l, R, Q, sub=8):
    """Volume-fraction density of the sphere on level l's cells."""
    X, Y, Z = H.centres(l)
    h = H.h(l)
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    frac = (r < R).astype(float)
    cut = np.abs(r - R) < h
    o = (np.arange(sub) + 0.5) / sub - 0.5
    ox, oy, oz = np.meshgrid(o, o, o, indexing="ij")
    xs, ys, zs = X[cut][:, None], Y[cut][:, None], Z[cut][:, None]
    rr = np.sqrt((xs + h * ox.ravel() - 0.5) ** 2 + (ys + h * oy.ravel() - 0.5) ** 2 +
                 (zs + h * oz.ravel() - 0.5) ** 2)
    frac[cut] = (rr < R).mean(axis=1)
    return frac * Q / (4.0 / 3.0 * math.pi * R ** 3)


def _solve_radial(n0, lmax, rho_fn, phi_fn):
    boxes = hierarchies.centred(n0) if lmax == 1 else None
    H = oracle.OracleHierarchy(n0, lmax, boxes=boxes)
    for l in range(H.nlevels):
        rho = rho_fn(H, l)
        if l == 0:
            rho = fold_dirichlet(H, rho, lambda x, y, z: phi_fn(np.sqrt((x - .5) ** 2 + (y - .5) ** 2 + (z - .5) ** 2)))
        H.set(l, "rho", rho * (H.mask(l) > 0))
    H.solve(eps=1e-12, max_iter=60, bottom_rtol=1e-14)
    err = 0.0
    for l in range(H.nlevels):
        X, Y, Z = H.centres(l)
        r = np.sqrt((X - .5) ** 2 + (Y - .5) ** 2 + (Z - .5) ** 2)
        m = H.mask(l) == 1 if l < H.nlevels - 1 else H.mask(l) > 0
        err = max(err, np.abs(H.get(l, "phi") - phi_fn(r))[m].max())
    return err


def test_smooth_radial_charge_second_order():
    """A Gaussian charge (closed-form potential Q erf(r / (sqrt 2 s)) /
    (4 pi r)) converges at second order in the max norm, on a single level
    and with a refined centre."""
    s, Q = 0.05, 1.0

    def rho_fn(H, l):
        X, Y, Z = H.centres(l)
        r2 = (X - .5) ** 2 + (Y - .5) ** 2 + (Z - .5) ** 2
        return Q * np.exp(-r2 / (2 * s * s)) / (2 * math.pi * s * s) ** 1.5

    def phi_fn(r):
        r = np.maximum(r, 1e-12)
        return Q * erf(r / (math.sqrt(2) * s)) / (4 * math.pi * r)

    e16, e32, e64 = (_solve_radial(n, 0, rho_fn, phi_fn) for n in (16, 32, 64))
    # sigma = 0.8 h at 16^3 is under-resolved; from 32^3 on the ratio is ~4
    assert e16 / e32 > 2.5 and e32 / e64 > 3.5
    # refining the centre of 32^3 once reaches the accuracy of uniform 64^3
    a = _solve_radial(32, 1, rho_fn, phi_fn)
    assert a < 1.1 * e64


def test_uniform_sphere_against_closed_form():
    """The Sec. 6.2 sphere (R = 0.2, Q = 1, centre 0.5) with the analytic
    potential as Dirichlet data: the error shrinks with resolution and the
    refined base 32^3 + 1 level is more accurate than the base alone."""
    R, Q = 0.2, 1.0
    rho_fn = lambda H, l: _sphere_rho(H, l, R, Q)
    phi_fn = lambda r: sphere_phi(r, Q, R)
    e32 = _solve_radial(32, 0, rho_fn, phi_fn)
    e64 = _solve_radial(64, 0, rho_fn, phi_fn)
    a = _solve_radial(32, 1, rho_fn, phi_fn)
    phi0 = sphere_phi(0.0, Q, R)
    assert e64 < 0.5 * e32
    assert a < 0.7 * e32
    assert a / phi0 < 2e-3
