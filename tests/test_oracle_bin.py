"""Pins of the oracle's particle binning: hand-worked keys for particles
placed in known bricks of a known hierarchy, the no-key case at the domain
face, and the counting sort against numpy's stable argsort."""
import numpy as np

import hierarchies
import oracle

NOKEY = 0xFFFFFFFF


def test_hand_worked_keys():
    # base 32^3 (h0 = 1/32, bricks 4 x 4 x 4 -> keys 0..63); level 1 = fine
    # cells 16..47 (h1 = 1/64, bricks 4 x 4 x 4 -> keys 64..127)
    O = oracle.OracleHierarchy(32, 1, boxes=hierarchies.centred(32))
    pts = {
        # centre: level 1, cell 32 -> brick (2,2,2) = 64 + 2 + 4 (2 + 4 * 2)
        (0.5, 0.5, 0.5): 64 + 2 + 4 * (2 + 4 * 2),
        # x = 0.26: level-1 nodes 16, 17 (valid), cell 16 -> brick x 0
        (0.26, 0.5, 0.5): 64 + 0 + 4 * (2 + 4 * 2),
        # x = 0.253: level-1 node 15 invalid -> level 0, cell 8 -> brick x 1
        (0.253, 0.5, 0.5): 0 + 1 + 4 * (2 + 4 * 2),
        # x = 0.1: level 0 only, cells 3 -> brick 0
        (0.1, 0.1, 0.1): 0,
        # x = 0.01: level-0 node -1 is outside the level -> no key
        (0.01, 0.5, 0.5): NOKEY,
        # last level-0 brick: x = 0.95 -> cell 30 -> brick 3
        (0.95, 0.95, 0.95): 3 + 4 * (3 + 4 * 3),
    }
    xs = np.array([p[0] for p in pts]), np.array([p[1] for p in pts]), np.array([p[2] for p in pts])
    keys, perm, nk = O.bin(*xs)
    assert nk == 128
    assert keys.tolist() == list(pts.values())


def test_counting_sort_is_stable_by_key():
    O = oracle.OracleHierarchy(32, 2, boxes=hierarchies.nested_centred(32))
    rng = np.random.default_rng(9)
    x, y, z = (rng.uniform(0.0, 1.0, 5000) for _ in range(3))
    keys, perm, nk = O.bin(x, y, z)
    assert np.array_equal(perm, np.argsort(keys.astype(np.uint64), kind="stable"))
    assert ((keys < nk) | (keys == NOKEY)).all()
    # particles near the faces (within half a base cell) have no key
    near = (np.minimum.reduce([x, y, z, 1 - x, 1 - y, 1 - z]) < 0.5 / 32)
    assert (keys[near] == NOKEY).all()
