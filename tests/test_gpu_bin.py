"""GPU particle binning (amr_bin) against the oracle: keys bit-exact on the
same particles (the level choice and the brick are integer decisions taken
from FP64 positions on both sides, power-of-two grids); the permutation is a
permutation of all particles that sorts the keys (the order of equal keys is
left open, so only what is unique is compared)."""
import numpy as np
import pytest

import hierarchies
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


def check(G, O, x, y, z):
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x, y, z)]
    keys, perm, nk = G.bin(*dev)
    torch.cuda.synchronize()
    kg = keys.cpu().numpy().view(np.uint32)
    pg = perm.cpu().numpy()
    ko, po, nko = O.bin(x, y, z)
    assert nk == nko
    assert np.array_equal(kg, ko)
    assert np.array_equal(np.sort(pg), np.arange(len(x)))
    ks = kg[pg].astype(np.uint64)
    assert (np.diff(ks) >= 0).all()


def test_bin_boxes_uniform_particles(amrmg):
    boxes = hierarchies.nested_centred(32)
    G = amrmg.Hierarchy(32, 2, boxes=boxes)
    O = oracle.OracleHierarchy(32, 2, boxes=boxes)
    rng = np.random.default_rng(21)
    x, y, z = (rng.uniform(-0.05, 1.05, 200_000) for _ in range(3))  # some outside
    x[:3] = [np.nan, np.inf, 1e300]
    check(G, O, x, y, z)


@pytest.mark.parametrize("name", ["c1_small", "c2_fp64"])
def test_bin_workloads(amrmg, name):
    w = inputs.workload(name)
    parts = w.particles(scale=0.2 if name == "c2_fp64" else 1.0)
    dev = [torch.from_numpy(a).cuda() for a in parts]
    G = amrmg.Hierarchy(w.n0, w.lmax, particles=dev, tag_mode=w.tag_mode, tag_lambda=w.tag_lambda,
                        boxes=w.boxes or None)
    O = oracle.OracleHierarchy(w.n0, w.lmax, particles=parts, tag_mode=w.tag_mode, tag_lambda=w.tag_lambda,
                               boxes=w.boxes or None)
    assert G.nlevels == O.nlevels
    check(G, O, *parts[:3])


def test_bin_empty_and_errors(amrmg):
    G = amrmg.Hierarchy(16, 0)
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    keys, perm, nk = G.bin(e, e, e)
    assert nk == 8 and keys.numel() == 0
