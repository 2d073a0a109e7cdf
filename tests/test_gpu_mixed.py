"""Mixed-precision form: FP32 smoothing and transfers inside an FP64
iterative-refinement loop (FP64 composite residual, interface corrections
and coarsest solve) must reach the FP64 oracle's answer at the same
tolerances as the plain FP64 solve."""
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


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = {
    "nested": (32, 2, hierarchies.nested_centred(32)),
    "notched": (24, 1, hierarchies.notched(24)),
    "channel1": (24, 1, hierarchies.channel(24, 1)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_matches_oracle(amrmg, name):
    n0, lmax, boxes = CASES[name]
    M = amrmg.Hierarchy(n0, lmax, boxes=boxes, precision="mixed")
    D = amrmg.Hierarchy(n0, lmax, boxes=boxes)
    O = oracle.OracleHierarchy(n0, lmax, boxes=boxes)
    rng = np.random.default_rng(41)
    for l in range(O.nlevels):
        rho = rng.normal(size=O.shape(l)) * (O.mask(l) > 0)
        for H in (M, D, O):
            H.set(l, "rho", rho)
    sm = M.solve(eps=1e-12)
    sd = D.solve(eps=1e-12)
    assert sm["status"] == "AMR_OK" and sm["rel_res"].max() <= 1e-12
    # FP32 inner cycles contract about as well as FP64 ones
    assert sm["iters"] <= sd["iters"] + 2
    O.solve(eps=1e-13, bottom_rtol=1e-15)
    for l in range(O.nlevels):
        assert relerr(M.get(l, "phi"), O.get(l, "phi")) <= 1e-10, l
        for f in ("ex", "ey", "ez"):
            assert relerr(M.get(l, f), O.get(l, f)) <= 1e-9, (l, f)


def test_mixed_config1_step(amrmg):
    w = inputs.workload("c1_small")
    parts = w.particles()
    dev = [torch.from_numpy(a).cuda() for a in parts]
    M = amrmg.Hierarchy(w.n0, w.lmax, boxes=w.boxes, particles=dev, precision="mixed")
    st = M.solve(eps=1e-10)
    assert st["status"] == "AMR_OK"
    O = oracle.OracleHierarchy(w.n0, w.lmax, boxes=w.boxes, particles=parts)
    O.solve(eps=1e-13, bottom_rtol=1e-15)
    # the stopping test bounds the residual, not the error: at 1e-10 the
    # potential error stays within 1e-8 (the field tolerances need a tighter
    # solve, checked above)
    for l in range(O.nlevels):
        assert relerr(M.get(l, "phi"), O.get(l, "phi")) <= 1e-8
    ex, ey, ez = M.gather(*dev[:3])
    oe = O.gather(*parts[:3])
    g = np.stack([t.cpu().numpy() for t in (ex, ey, ez)])
    assert relerr(g, np.stack(oe)) <= 1e-7


def test_mixed_graph_and_host_driven_agree(amrmg):
    n0, lmax, boxes = CASES["nested"]
    A = amrmg.Hierarchy(n0, lmax, boxes=boxes, precision="mixed")
    B = amrmg.Hierarchy(n0, lmax, boxes=boxes, precision="mixed")
    rng = np.random.default_rng(42)
    for l in range(A.nlevels):
        rho = rng.normal(size=A.shape(l)) * (A.mask(l) > 0)
        A.set(l, "rho", rho)
        B.set(l, "rho", rho)
    sa = A.solve(eps=1e-11)
    sb = B.solve(eps=1e-11, use_graph=False)
    assert sa["iters"] == sb["iters"]
    for l in range(A.nlevels):
        assert np.array_equal(A.get(l, "phi"), B.get(l, "phi"))
