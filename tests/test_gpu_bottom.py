"""The level-0 multigrid below 32^3 cells as one thread-block-cluster launch
against the same operations launched one by one: identical operations in
identical order, so whole solves agree bit for bit (both precisions,
captured graph and host-driven loop, power-of-two and odd coarsest grids),
and the cluster path still matches the oracle."""
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
    "n64_single": (64, 0, None),      # multigrid 64 -> 32 -> 16 -> 8 (dense)
    "n40_single": (40, 0, None),      # 40 -> 20 -> 10 -> 5 (dense)
    "n32_nested": (32, 2, hierarchies.nested_centred(32)),
    "n48_centred": (48, 1, hierarchies.centred(48)),
}


def run(amrmg, monkeypatch, bottom, name, precision, **kw):
    monkeypatch.setenv("AMR_MG_BOTTOM", bottom)
    n0, lmax, boxes = CASES[name]
    H = amrmg.Hierarchy(n0, lmax, boxes=boxes, precision=precision)
    rng = np.random.default_rng(5)
    for l in range(H.nlevels):
        H.set(l, "rho", rng.normal(size=H.shape(l)) * (H.mask(l) > 0))
    st = H.solve(**kw)
    out = [H.get(l, "phi") for l in range(H.nlevels)]
    H.close()
    return st, out


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_cluster_bottom_equals_launches(amrmg, monkeypatch, name, precision, graph):
    kw = dict(eps=1e-30, max_iter=3, use_graph=graph)
    st0, ref = run(amrmg, monkeypatch, "0", name, precision, **kw)
    st1, got = run(amrmg, monkeypatch, "1", name, precision, **kw)
    assert st0["iters"] == st1["iters"]
    for l in range(len(ref)):
        assert np.array_equal(got[l], ref[l]), l


@pytest.mark.parametrize("nu", [(0, 2), (1, 0), (3, 1)])
def test_cluster_bottom_sweep_counts(amrmg, monkeypatch, nu):
    kw = dict(eps=1e-30, max_iter=2, nu_pre=nu[0], nu_post=nu[1], use_graph=False)
    _, ref = run(amrmg, monkeypatch, "0", "n64_single", "fp64", **kw)
    _, got = run(amrmg, monkeypatch, "1", "n64_single", "fp64", **kw)
    for l in range(len(ref)):
        assert np.array_equal(got[l], ref[l]), l


def test_cluster_bottom_matches_oracle(amrmg, monkeypatch):
    monkeypatch.setenv("AMR_MG_BOTTOM", "1")
    w = inputs.workload("c1_small")
    parts = w.particles()
    dev = [torch.from_numpy(a).cuda() for a in parts]
    G = amrmg.Hierarchy(w.n0, w.lmax, boxes=w.boxes, particles=dev)
    st = G.solve(eps=1e-12)
    assert st["status"] == "AMR_OK"
    O = oracle.OracleHierarchy(w.n0, w.lmax, boxes=w.boxes, particles=parts)
    O.solve(eps=1e-13, bottom_rtol=1e-15)
    for l in range(O.nlevels):
        a, b = G.get(l, "phi"), O.get(l, "phi")
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("faces", ["dirichlet", "robin", "periodic"])
def test_large_odd_coarsest_grid_solved_separably(amrmg, faces):
    """n0 = 104 = 8 x 13 coarsens 104 -> 52 -> 26 -> 13: the coarsest grid
    (13^3 = 2197 cells) is beyond the dense inverse's 11^3 and is solved
    separably (eigenvectors of the 1-D operator along x, y, z).  The solve
    reaches the oracle's potential at 1e-10 for every kind of face."""
    import oracle
    n0 = 104
    kw = {"dirichlet": {}, "robin": {"robin_d": 0.5}, "periodic": {"periodic": True}}[faces]
    G = amrmg.Hierarchy(n0, 0, **kw)
    O = oracle.OracleHierarchy(n0, 0, **{k: (v if k != "periodic" else True) for k, v in kw.items()})
    rng = np.random.default_rng(13)
    rho = rng.normal(size=G.shape(0))
    G.set(0, "rho", rho)
    O.set(0, "rho", rho)
    st = G.solve(eps=1e-12, max_iter=60)
    assert st["status"] == "AMR_OK", st
    O.solve(eps=1e-12, bottom_rtol=1e-14)
    a, b = G.get(0, "phi"), O.get(0, "phi")
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)
