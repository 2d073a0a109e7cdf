"""The gather buffer on the GPU (amr_set_gather_buffer) against the
oracle's, on the config-1 step (32^3 + the central 16^3 coarse cells
refined, 1e4 Gaussian particles) for buffers 0..3, field 1e-9 relative; and
the GPU's self-force at the interface shrinking with the buffer."""
import numpy as np
import pytest

import oracle
from paper_1812_03689_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amrmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_03689_gb300 import build
    build.build()
    from paper_1812_03689_gb300 import amrmg as m
    return m


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_buffer_parity(amrmg):
    w = inputs.workload("c1_small")
    parts = w.particles()
    dev = [torch.from_numpy(a).cuda() for a in parts]
    G = amrmg.Hierarchy(w.n0, w.lmax, boxes=w.boxes, particles=dev)
    O = oracle.OracleHierarchy(w.n0, w.lmax, boxes=w.boxes, particles=parts)
    assert G.solve(eps=1e-13)["status"] == "AMR_OK"
    O.solve(eps=1e-13, bottom_rtol=1e-15)
    prev = None
    for b in (0, 1, 2, 3, 0):
        G.set_gather_buffer(b)
        O.set_gather_buffer(b)
        g = np.stack([t.cpu().numpy() for t in G.gather(*dev[:3])])
        o = np.stack(O.gather(*parts[:3]))
        assert relerr(g, o) <= 1e-9, b
        if prev is not None and b:
            assert not np.array_equal(g, prev)       # the buffer changes the interpolation
        prev = g
    with pytest.raises(amrmg.AmrError):
        G.set_gather_buffer(9)


def test_self_force_shrinks(amrmg):
    n0, boxes = 32, [(1, (16, 16, 16), (47, 47, 47))]
    p = [np.array([v / n0]) for v in (8.5, 16.3, 16.1)] + [np.array([1.0])]
    dev = [torch.from_numpy(a).cuda() for a in p]
    G = amrmg.Hierarchy(n0, 1, boxes=boxes, particles=dev)
    G.solve(eps=1e-13)
    f = {}
    for b in (0, 2):
        G.set_gather_buffer(b)
        f[b] = np.linalg.norm([t.cpu().numpy()[0] for t in G.gather(*dev[:3])])
    assert f[2] * 5 <= f[0], f
