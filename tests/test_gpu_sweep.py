"""Fused red-black sweeps (one out-of-place launch per sweep, shared-memory
plane ring with recomputed halo reds) against per-colour passes.

Every cell update uses the same expression and summation tree in both
kernels, so whole solves must agree bit for bit for every tile shape and
plane-chunk length, in both precisions, with coarse-fine faces (nested,
notched, one-cell channel hierarchies), tiles that overhang the box, and odd
sweep counts (which fall back to per-colour passes for the sweep that has
no out-of-place partner).  The forced fused path is also checked against
the oracle."""
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
    "single": (24, 0, None),
    "nested": (32, 2, hierarchies.nested_centred(32)),
    "notched": (24, 1, hierarchies.notched(24)),
    "channel1": (24, 1, hierarchies.channel(24, 1)),
}


def run(amrmg, monkeypatch, sweep, name, precision, **solve_kw):
    monkeypatch.setenv("AMR_SWEEP", sweep)
    n0, lmax, boxes = CASES[name]
    H = amrmg.Hierarchy(n0, lmax, boxes=boxes, precision=precision)
    rng = np.random.default_rng(77)
    for l in range(H.nlevels):
        H.set(l, "rho", rng.normal(size=H.shape(l)) * (H.mask(l) > 0))
    st = H.solve(**solve_kw)
    out = [H.get(l, "phi") for l in range(H.nlevels)]
    H.close()
    return st, out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_fused_equals_per_colour(amrmg, monkeypatch, name, precision):
    kw = dict(eps=1e-30, max_iter=3, use_graph=False)
    st0, ref = run(amrmg, monkeypatch, "colour", name, precision, **kw)
    for shape in range(5):
        for zc in (1, 3, 64):
            st, got = run(amrmg, monkeypatch, f"fused:{shape}:{zc}", name, precision, **kw)
            assert st["iters"] == st0["iters"]
            for l in range(len(ref)):
                assert np.array_equal(got[l], ref[l]), (shape, zc, l)


@pytest.mark.parametrize("nu", [(1, 1), (1, 3), (3, 2), (0, 2)])
def test_fused_odd_sweep_counts(amrmg, monkeypatch, nu):
    kw = dict(eps=1e-30, max_iter=2, nu_pre=nu[0], nu_post=nu[1], use_graph=False)
    _, ref = run(amrmg, monkeypatch, "colour", "nested", "fp64", **kw)
    _, got = run(amrmg, monkeypatch, "fused:1:4", "nested", "fp64", **kw)
    for l in range(len(ref)):
        assert np.array_equal(got[l], ref[l]), l


def test_autotuned_and_graph_equal_per_colour(amrmg, monkeypatch):
    kw = dict(eps=1e-30, max_iter=3)
    _, ref = run(amrmg, monkeypatch, "colour", "nested", "fp64", use_graph=False, **kw)
    _, auto = run(amrmg, monkeypatch, "auto", "nested", "fp64", **kw)
    for l in range(len(ref)):
        assert np.array_equal(auto[l], ref[l]), l


def test_fused_matches_oracle_config1(amrmg, monkeypatch):
    monkeypatch.setenv("AMR_SWEEP", "fused:2:8")
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


# Cell lists (the refined levels' colour passes, residual and prolongation
# over their valid cells, the restriction over the covered cells) change
# which threads do the work, not the expression per cell: the same bits as
# the passes over the whole box.
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["nested", "notched", "channel1"])
def test_cell_lists_equal_box_passes(amrmg, monkeypatch, name, precision):
    kw = dict(eps=1e-30, max_iter=3)
    monkeypatch.setenv("AMR_CELL_LISTS", "0")
    st0, ref = run(amrmg, monkeypatch, "colour", name, precision, **kw)
    monkeypatch.delenv("AMR_CELL_LISTS")
    st, got = run(amrmg, monkeypatch, "colour", name, precision, **kw)
    assert st["iters"] == st0["iters"]
    for l in range(len(ref)):
        assert np.array_equal(got[l], ref[l]), l
