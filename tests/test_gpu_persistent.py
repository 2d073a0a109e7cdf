"""Persistent program form and batched form (one cooperative kernel per
solve, rounds separated by a bounded grid barrier): the same operations in
the same order as the graph form, so results agree bit for bit; a batch of
uneven hierarchies gives each hierarchy the result it gets alone; the
barrier's bounded wait returns AMR_ETIMEOUT instead of hanging."""
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


CASES = {
    "single": (16, 0, None),
    "centred": (32, 1, hierarchies.centred(32)),
    "nested": (32, 2, hierarchies.nested_centred(32)),
    "notched": (24, 1, hierarchies.notched(24)),
    "channel1": (24, 1, hierarchies.channel(24, 1)),
}


def fill(H, seed):
    rng = np.random.default_rng(seed)
    for l in range(H.nlevels):
        H.set(l, "rho", rng.normal(size=H.shape(l)) * (H.mask(l) > 0))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_persistent_equals_graph(amrmg, name, precision):
    n0, lmax, boxes = CASES[name]
    A = amrmg.Hierarchy(n0, lmax, boxes=boxes, precision=precision)
    B = amrmg.Hierarchy(n0, lmax, boxes=boxes, precision=precision)
    fill(A, 51)
    fill(B, 51)
    sa = A.solve(eps=1e-11, persistent=True)
    sb = B.solve(eps=1e-11)
    assert sa["status"] == "AMR_OK"
    assert sa["iters"] == sb["iters"] and np.array_equal(sa["rel_res"], sb["rel_res"])
    for l in range(A.nlevels):
        for f in ("phi", "ex", "ey", "ez"):
            assert np.array_equal(A.get(l, f), B.get(l, f)), (l, f)
    # the recorded program is reused
    sa2 = A.solve(eps=1e-11, persistent=True)
    assert sa2["iters"] == sa["iters"]


def test_persistent_matches_oracle_config1(amrmg):
    w = inputs.workload("c1_small")
    parts = w.particles()
    dev = [torch.from_numpy(a).cuda() for a in parts]
    G = amrmg.Hierarchy(w.n0, w.lmax, boxes=w.boxes, particles=dev)
    st = G.solve(eps=1e-12, persistent=True)
    assert st["status"] == "AMR_OK"
    O = oracle.OracleHierarchy(w.n0, w.lmax, boxes=w.boxes, particles=parts)
    O.solve(eps=1e-13, bottom_rtol=1e-15)
    for l in range(O.nlevels):
        a, b = G.get(l, "phi"), O.get(l, "phi")
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("mode", ["graphs", "clusters", "rounds"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_alone(amrmg, precision, mode):
    """Uneven hierarchies (depth 0-2, bases 16-40, one with different
    tolerance behaviour) in one batch, in each of the batch forms (graph
    branches, persistent cluster program, lock-step rounds): each result
    equals its solo solve, bit for bit."""
    specs = [CASES["single"], CASES["centred"], CASES["nested"], CASES["notched"], CASES["channel1"],
             (40, 0, None), (24, 0, None)]
    batch, solo = [], []
    for i, (n0, lmax, boxes) in enumerate(specs):
        for lst in (batch, solo):
            H = amrmg.Hierarchy(n0, lmax, boxes=boxes, precision=precision)
            fill(H, 60 + i)
            lst.append(H)
    B = amrmg.Batch(batch, mode=mode, eps=1e-11)
    stats = B.solve()
    for i, (Hb, Hs) in enumerate(zip(batch, solo)):
        ss = Hs.solve(eps=1e-11, persistent=True)
        assert stats[i]["status"] == "AMR_OK"
        assert stats[i]["iters"] == ss["iters"], i
        for l in range(Hb.nlevels):
            for f in ("phi", "ex"):
                assert np.array_equal(Hb.get(l, f), Hs.get(l, f)), (i, l, f)
    # a second batched solve (same program) gives the same answer
    stats2 = B.solve()
    assert [s["iters"] for s in stats2] == [s["iters"] for s in stats]
    B.close()


def test_barrier_timeout_is_bounded(amrmg):
    n0, lmax, boxes = CASES["centred"]
    H = amrmg.Hierarchy(n0, lmax, boxes=boxes)
    fill(H, 70)
    rc = H.selftest_barrier_timeout(50)
    assert rc == amrmg.AMR_ETIMEOUT
    # the context and the hierarchy stay usable
    st = H.solve(eps=1e-11, persistent=True)
    assert st["status"] == "AMR_OK"


@pytest.mark.parametrize("mode", ["graphs", "clusters"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_matches_oracle(amrmg, precision, mode):
    """The same uneven batch against the oracle, hierarchy by hierarchy
    (phi 1e-10 and E 1e-9 relative L2 per level): the right-hand sides come
    from the host generator, the oracle gets them directly."""
    specs = [CASES["single"], CASES["centred"], CASES["nested"], CASES["notched"], CASES["channel1"],
             (40, 0, None), (24, 0, None)]
    hs, rhos = [], []
    for i, (n0, lmax, boxes) in enumerate(specs):
        H = amrmg.Hierarchy(n0, lmax, boxes=boxes, precision=precision)
        rng = np.random.default_rng(80 + i)
        r = [rng.normal(size=H.shape(l)) * (H.mask(l) > 0) for l in range(H.nlevels)]
        for l in range(H.nlevels):
            H.set(l, "rho", r[l])
        hs.append(H)
        rhos.append(r)
    B = amrmg.Batch(hs, mode=mode, eps=1e-12)
    stats = B.solve()
    for i, ((n0, lmax, boxes), H, r) in enumerate(zip(specs, hs, rhos)):
        assert stats[i]["status"] == "AMR_OK", (i, stats[i])
        O = oracle.OracleHierarchy(n0, lmax, boxes=boxes)
        for l in range(O.nlevels):
            assert np.array_equal(O.mask(l), H.mask(l)), (i, l)
            O.set(l, "rho", r[l])
        O.solve(eps=1e-13, bottom_rtol=1e-15)
        for l in range(O.nlevels):
            a, b = H.get(l, "phi"), O.get(l, "phi")
            assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b), (i, l)
            for f in ("ex", "ey", "ez"):
                a, b = H.get(l, f), O.get(l, f)
                assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b), (i, l, f)
    B.close()
