"""Exact level-0 bottom solve (sine transforms along x and y, tridiagonal
solves along z) against the geometric-multigrid bottom and the oracle.

With a single level, one V-cycle is the bottom solve itself, so an exact
bottom leaves a residual at rounding level after ONE iteration; with
refinement levels both bottoms must converge to the same composite
solution."""
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


def filled(amrmg, n0, lmax, boxes, precision="fp64", seed=3):
    H = amrmg.Hierarchy(n0, lmax, boxes=boxes, precision=precision)
    rng = np.random.default_rng(seed)
    for l in range(H.nlevels):
        H.set(l, "rho", rng.normal(size=H.shape(l)) * (H.mask(l) > 0))
    return H


@pytest.mark.parametrize("n0", [8, 24, 32, 64])
def test_single_level_one_cycle_is_exact(amrmg, monkeypatch, n0):
    monkeypatch.setenv("AMR_BOTTOM", "dst")
    H = filled(amrmg, n0, 0, None)
    st = H.solve(eps=1e-30, max_iter=1)
    assert st["iters"] == 1
    assert st["rel_res"][0] <= 1e-12, st["rel_res"]


def test_single_level_matches_oracle(amrmg, monkeypatch):
    monkeypatch.setenv("AMR_BOTTOM", "dst")
    H = filled(amrmg, 32, 0, None, seed=8)
    H.solve(eps=1e-30, max_iter=1)
    O = oracle.OracleHierarchy(32, 0)
    O.set(0, "rho", H.get(0, "rho"))
    O.solve(eps=1e-13, bottom_rtol=1e-15)
    a, b = H.get(0, "phi"), O.get(0, "phi")
    assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["nested", "notched", "channel1"])
def test_dst_and_multigrid_bottoms_agree(amrmg, monkeypatch, case, precision):
    n0, lmax, boxes = {"nested": (32, 2, hierarchies.nested_centred(32)),
                       "notched": (24, 1, hierarchies.notched(24)),
                       "channel1": (24, 1, hierarchies.channel(24, 1))}[case]
    out = {}
    for bottom in ("dst", "mg"):
        monkeypatch.setenv("AMR_BOTTOM", bottom)
        H = filled(amrmg, n0, lmax, boxes, precision, seed=11)
        st = H.solve(eps=1e-12)
        assert st["status"] == "AMR_OK", (bottom, st)
        out[bottom] = [H.get(l, "phi") for l in range(H.nlevels)]
        H.close()
    for a, b in zip(out["dst"], out["mg"]):
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


def test_dst_bottom_config1_matches_oracle(amrmg, monkeypatch):
    monkeypatch.setenv("AMR_BOTTOM", "dst")
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


# The fast transforms (B. G. Lee's split of the cosine transform: the
# default for n0 = 128, AMR_BOTTOM=fast for every power of two from 32 to
# 128) against the folded matrix transforms and the oracle.

@pytest.mark.parametrize("n0", [32, 64, 128])
def test_fast_single_level_one_cycle_is_exact(amrmg, monkeypatch, n0):
    monkeypatch.setenv("AMR_BOTTOM", "fast")
    H = filled(amrmg, n0, 0, None, seed=5)
    assert H.bottom_solver() == "exact"
    st = H.solve(eps=1e-30, max_iter=1)
    assert st["iters"] == 1
    assert st["rel_res"][0] <= 1e-12, st["rel_res"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n0", [64, 128])
def test_fast_and_matrix_transforms_agree(amrmg, monkeypatch, n0, precision):
    out = {}
    for bottom in ("fast", "matrix"):
        monkeypatch.setenv("AMR_BOTTOM", bottom)
        H = filled(amrmg, n0, 0, None, precision, seed=21)
        H.solve(eps=1e-30, max_iter=1)
        out[bottom] = H.get(0, "phi")
        H.close()
    a, b = out["fast"], out["matrix"]
    # mixed: both bottoms are FP64 but write an FP32 correction, whose
    # rounding may differ by one FP32 unit where the FP64 values differ
    tol = 1e-12 if precision == "fp64" else 2.0 ** -22
    assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), np.linalg.norm(a - b) / np.linalg.norm(b)
    assert np.abs(a - b).max() <= tol * np.abs(b).max()


def test_fast_single_level_matches_oracle(amrmg, monkeypatch):
    monkeypatch.setenv("AMR_BOTTOM", "fast")
    H = filled(amrmg, 32, 0, None, seed=9)
    H.solve(eps=1e-30, max_iter=1)
    O = oracle.OracleHierarchy(32, 0)
    O.set(0, "rho", H.get(0, "rho"))
    O.solve(eps=1e-13, bottom_rtol=1e-15)
    a, b = H.get(0, "phi"), O.get(0, "phi")
    assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fast_and_multigrid_bottoms_agree_refined(amrmg, monkeypatch, precision):
    n0, lmax, boxes = 32, 2, hierarchies.nested_centred(32)
    out = {}
    for bottom in ("fast", "mg"):
        monkeypatch.setenv("AMR_BOTTOM", bottom)
        H = filled(amrmg, n0, lmax, boxes, precision, seed=13)
        st = H.solve(eps=1e-12)
        assert st["status"] == "AMR_OK", (bottom, st)
        out[bottom] = [H.get(l, "phi") for l in range(H.nlevels)]
        H.close()
    for a, b in zip(out["fast"], out["mg"]):
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)
