"""Box-list hierarchies used by the oracle pins and the GPU parity tests.

Boxes are (level, lo, hi), inclusive, in that level's index space.  ``cbox``
takes the extent in the next-coarser level's index space (fine boxes must
cover whole coarse cells)."""


def cbox(level, lo, hi):
    return (level, tuple(2 * v for v in lo), tuple(2 * v + 1 for v in hi))


# one centred box (config-1 layout): every ghost uses the centred case 0
def centred(n0=32):
    q = n0 // 4
    return [cbox(1, (q, q, q), (3 * q - 1, 3 * q - 1, 3 * q - 1))]


# two nested centred boxes (the symmetry problem of Sec. 6.1)
def nested_centred(n0=32):
    q = n0 // 4
    l1 = centred(n0)
    lo2, hi2 = 2 * q + q, 2 * (3 * q) - q - 1          # level-1 cells, centred half
    return l1 + [cbox(2, (lo2, lo2, lo2), (hi2, hi2, hi2))]


# a cube with one octant notched out: shifted and corner quadratic cases
def notched(n0=24):
    a, m, b = n0 // 4, n0 // 2, 3 * n0 // 4 - 1
    return [cbox(1, (a, a, a), (b, b, m - 1)), cbox(1, (a, a, m), (m - 1, b, b)), cbox(1, (m, a, m), (b, m - 1, b))]


# a slab with two walls and a channel of the given width (in coarse cells)
# between them: width 2 forces linear ghosts, width 1 the constant fall-back
def channel(n0=24, width=2):
    a, b = n0 // 4, 3 * n0 // 4 - 1
    z0, z1 = a, a + 3
    w0 = a + 1
    return [cbox(1, (a, a, z0), (b, b, z1)), cbox(1, (a, a, z1 + 1), (w0, b, z1 + 4)),
            cbox(1, (w0 + width + 1, a, z1 + 1), (b, b, z1 + 4))]
