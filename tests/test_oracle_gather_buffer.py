"""Pins of the oracle's gather buffer (buffer cells against the spurious
self-force near coarse-fine faces, which the paper corrects as in the work
it cites):

- buffer 0 is the plain rule (the finest level holding the 8 nodes);
- a buffer wider than every refined level interpolates every particle from
  level 0: equal to cloud-in-cell interpolation of the dense level-0 field,
  written out here in numpy;
- a single particle half a fine cell inside the refined box feels a
  self-force several times smaller with a buffer than without, while a
  particle deep inside the box is unaffected.
"""
import numpy as np

import oracle
from paper_1812_03689_gb300 import inputs


def cic_dense(field, lo, h, x, y, z):
    out = np.zeros(len(x))
    for p in range(len(x)):
        s = [x[p] / h - 0.5 - lo[0], y[p] / h - 0.5 - lo[1], z[p] / h - 0.5 - lo[2]]
        i = [int(np.floor(v)) for v in s]
        w = [v - np.floor(v) for v in s]
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    wt = (w[0] if a else 1 - w[0]) * (w[1] if b else 1 - w[1]) * (w[2] if c else 1 - w[2])
                    out[p] += wt * field[i[2] + c, i[1] + b, i[0] + a]
    return out


def test_buffer_zero_and_level0_limit():
    w = inputs.workload("c1_small")
    parts = w.particles()
    O = oracle.OracleHierarchy(w.n0, w.lmax, boxes=w.boxes, particles=parts)
    O.solve(eps=1e-12)
    plain = O.gather(*parts[:3])
    O.set_gather_buffer(0)
    assert all(np.array_equal(a, b) for a, b in zip(O.gather(*parts[:3]), plain))
    O.set_gather_buffer(40)
    far = O.gather(*parts[:3])
    lo, hi, _ = O.level_box(0)
    sel = slice(0, 300)
    for d, f in enumerate(("ex", "ey", "ez")):
        want = cic_dense(O.get(0, f), lo, O.h(0), parts[0][sel], parts[1][sel], parts[2][sel])
        assert np.allclose(far[d][sel], want, rtol=1e-13, atol=1e-13 * np.abs(want).max())
    assert any(not np.array_equal(a, b) for a, b in zip(far, plain))


def test_buffer_reduces_self_force_at_the_interface():
    n0, boxes = 32, [(1, (16, 16, 16), (47, 47, 47))]
    force = {}
    for xc in (8.5, 12.0):
        x, y, z, q = (np.array([v / n0]) for v in (xc, 16.3, 16.1, n0))
        q[:] = 1.0
        O = oracle.OracleHierarchy(n0, 1, boxes=boxes, particles=(x, y, z, q))
        O.solve(eps=1e-13, bottom_rtol=1e-15)
        for b in (0, 2):
            O.set_gather_buffer(b)
            force[xc, b] = np.linalg.norm([e[0] for e in O.gather(x, y, z)])
    assert force[8.5, 2] * 5 <= force[8.5, 0], force
    assert force[12.0, 2] == force[12.0, 0]
