"""Regrid on the GPU (Sec. 4.2 AMR policies, amr_regrid_boxes) against the
oracle's regrid on identical fields: the new hierarchies' masks agree
exactly (integer work decided by the same FP64 comparisons on identical
values), and a solve warm-started through amr_transfer_phi reaches the
oracle's solution of the regridded hierarchy in fewer V-cycles than a cold
solve."""
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


def cuda(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def solved(amrmg):
    """c1-sized step tagged by density: 32^3, up to two levels, 1e4
    Gaussian particles; the oracle's converged phi copied to the GPU side so
    both regrid from identical fields."""
    w = inputs.workload("c1_small")
    parts = w.particles()
    dev = cuda(*parts)
    G = amrmg.Hierarchy(32, 2, particles=dev, tag_mode="rel", tag_lambda=0.1)
    O = oracle.OracleHierarchy(32, 2, particles=parts, tag_mode="rel", tag_lambda=0.1)
    assert G.nlevels == O.nlevels == 3
    O.solve(eps=1e-13, bottom_rtol=1e-15)
    O.average_down()
    O.efield()
    for l in range(O.nlevels):
        G.set(l, "phi", O.get(l, "phi"))
    G.field_from_phi()
    for l in range(O.nlevels):
        for f in ("ex", "ey", "ez"):
            a, b = G.get(l, f), O.get(l, f)
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    return G, O, parts, dev


@pytest.mark.parametrize("policy,lam", [("rel", 0.1), ("rel", 0.02), ("abs", 50.0), ("abs", 20.0), ("phi", 0.5),
                                        ("phi", 0.8), ("efield", 0.3), ("efield", 0.6)])
def test_regrid_masks_match_oracle(amrmg, solved, policy, lam):
    G, O, parts, dev = solved
    boxes = G.regrid_boxes(policy, lam, 2)
    R = O.regrid(policy, lam, 2, particles=parts)
    assert len({b[0] for b in boxes}) == R.nlevels - 1
    if R.nlevels == 1:
        return
    N = amrmg.Hierarchy(32, 2, boxes=boxes, particles=dev)
    assert N.nlevels == R.nlevels
    for l in range(R.nlevels):
        assert np.array_equal(N.mask(l), R.mask(l)), (policy, lam, l)


def test_warm_start_after_regrid(amrmg, solved):
    G, O, parts, dev = solved
    G.solve(eps=1e-12)
    boxes = G.regrid_boxes("phi", 0.5, 2)
    R = O.regrid("phi", 0.5, 2, particles=parts)
    R.solve(eps=1e-13, bottom_rtol=1e-15)
    cold = amrmg.Hierarchy(32, 2, boxes=boxes, particles=dev)
    st_cold = cold.solve(eps=1e-12)
    warm = amrmg.Hierarchy(32, 2, boxes=boxes, particles=dev)
    warm.transfer_phi_from(G)
    st_warm = warm.solve(eps=1e-12, warm_start=True)
    assert st_cold["status"] == st_warm["status"] == "AMR_OK"
    assert st_warm["iters"] < st_cold["iters"], (st_warm["iters"], st_cold["iters"])
    for l in range(R.nlevels):
        assert relerr(warm.get(l, "phi"), R.get(l, "phi")) <= 1e-10, l
        assert relerr(cold.get(l, "phi"), R.get(l, "phi")) <= 1e-10, l


def test_regrid_errors(amrmg, solved):
    G = solved[0]
    for kw in (dict(policy="boxes", tag_lambda=0.1, max_level=2), dict(policy="phi", tag_lambda=float("nan"),
                                                                         max_level=2),
               dict(policy="phi", tag_lambda=0.5, max_level=9)):
        with pytest.raises(amrmg.AmrError) as ei:
            G.regrid_boxes(**kw)
        assert ei.value.code == amrmg.AMR_EINVAL
    # a zero potential tags nothing: no refined level
    Z = amrmg.Hierarchy(16, 0)
    assert Z.regrid_boxes("phi", 0.5, 1) == []
