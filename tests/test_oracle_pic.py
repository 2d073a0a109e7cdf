"""Pins of the oracle's particle side (oracle/pic.py) against closed forms:

- the domain transform puts the farthest particle exactly on the face of the
  central 1/(1 + delta) of the cube, and a bunch scaled by two about the
  centre maps to the same cube coordinates bit for bit with S doubled;
- through the whole oracle step (deposit, solve, E, rescale, gather) the
  field of the doubled bunch is exactly a quarter of the field of the
  original (Eq. efield_transform, E ~ s^-2 in three dimensions) and the
  potential exactly a half (Eq. potential_transform);
- the kick-drift push in a uniform field gives p_k = p_0 + k a dt and
  x_k = x_0 + k dt p_0 + a dt^2 k (k + 1) / 2;
- the moments of hand-made distributions: +-a gives sigma = a and xi = 1,
  the five points -2..2 give sigma^2 = 2 and xi = 6.8 / 4, and a large
  Gaussian sample gives xi near 3.
"""
import numpy as np

import oracle
from oracle import pic


def bunch(n=3000, seed=5):
    g = np.random.default_rng(seed)
    return [g.normal(0.0, s, n) + c for s, c in ((0.3, 1.0), (0.2, -2.0), (0.25, 0.5))]


def test_transform_extent_and_scale_invariance():
    x, y, z = bunch()
    c = (1.0, -2.0, 0.5)
    u, v, w, S = pic.domain_transform(x, y, z, c, 0.2)
    ext = max(np.abs(x - 1.0).max(), np.abs(y + 2.0).max(), np.abs(z - 0.5).max())
    assert np.isclose(S, 2.4 * ext)
    lim = 0.5 / 1.2
    got = max(np.abs(u - 0.5).max(), np.abs(v - 0.5).max(), np.abs(w - 0.5).max())
    assert np.isclose(got, lim, rtol=1e-15) and got <= lim * (1 + 1e-15)
    x2, y2, z2 = (2 * (a - cv) + cv for a, cv in zip((x, y, z), c))
    u2, v2, w2, S2 = pic.domain_transform(x2, y2, z2, c, 0.2)
    assert S2 == 2 * S
    assert np.array_equal(u2, u) and np.array_equal(v2, v) and np.array_equal(w2, w)


def step_fields(pos, q, c):
    u, v, w, S = pic.domain_transform(*pos, c, 0.2)
    H = oracle.OracleHierarchy(16, 1, particles=(u, v, w, q), tag_mode="rel", tag_lambda=0.1)
    H.solve(eps=1e-13, bottom_rtol=1e-15)
    H.average_down()
    H.efield()
    pic.rescale_fields(H, S)
    ex, ey, ez, ph = H.gather(u, v, w, with_phi=True)
    return np.stack([ex, ey, ez]), ph


def test_field_and_potential_scaling_law():
    x, y, z = bunch(2000)
    q = np.full(2000, 1.0 / 2000)
    c = (1.0, -2.0, 0.5)
    E1, P1 = step_fields([x, y, z], q, c)
    E2, P2 = step_fields([2 * (a - cv) + cv for a, cv in zip((x, y, z), c)], q, c)
    assert np.abs(E1).max() > 0
    assert np.array_equal(E2, E1 / 4)
    assert np.array_equal(P2, P1 / 2)


def test_push_uniform_field():
    g = np.random.default_rng(2)
    x0 = [g.uniform(-1, 1, 50) for _ in range(3)]
    p0 = [g.uniform(-1, 1, 50) for _ in range(3)]
    E = [np.full(50, 0.75), np.full(50, -0.5), np.full(50, 0.25)]
    qm, dt, K = 2.0, 1e-2, 25
    pos, mom = x0, p0
    for _ in range(K):
        pos, mom = pic.push(pos, mom, E, qm, dt)
    for d in range(3):
        a = qm * E[d]
        assert np.allclose(mom[d], p0[d] + K * a * dt, rtol=1e-13, atol=1e-14)
        assert np.allclose(pos[d], x0[d] + K * dt * p0[d] + a * dt * dt * K * (K + 1) / 2, rtol=1e-13, atol=1e-14)


def test_moments_closed_forms():
    a = np.array([3.0 - 0.5, 3.0 + 0.5] * 10)
    m = pic.moments(a, a * 2, a - 3.0)
    assert np.allclose(m["centroid"], [3.0, 6.0, 0.0]) and np.allclose(m["sigma"], [0.5, 1.0, 0.5])
    assert np.allclose(m["xi"], 1.0)
    b = np.arange(-2.0, 3.0) + 7.0
    m = pic.moments(b, b, b)
    assert np.allclose(m["sigma"] ** 2, 2.0) and np.allclose(m["xi"], 6.8 / 4)
    g = np.random.default_rng(9).normal(size=(3, 400000))
    m = pic.moments(*g)
    assert np.all(np.abs(m["xi"] - 3.0) < 0.05)
