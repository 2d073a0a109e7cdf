"""Per-launch kernel timers: the host-driven mode times every operation
alone; the graph mode runs the solve as a profiled copy of its captured
graph (same kernels and grouped launches, unrolled to the last solve's
V-cycle count, event-record nodes around each kernel node).  Both must
leave the answer unchanged, and the graph mode's per-kind times must fit
inside the solve's own device time."""
import numpy as np
import pytest

import hierarchies

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


def filled(amrmg, precision, seed=5):
    H = amrmg.Hierarchy(32, 2, boxes=hierarchies.nested_centred(32), precision=precision)
    rng = np.random.default_rng(seed)
    for l in range(H.nlevels):
        H.set(l, "rho", rng.normal(size=H.shape(l)) * (H.mask(l) > 0))
    return H


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_profile_matches_graph_solve(amrmg, precision):
    A, B = filled(amrmg, precision), filled(amrmg, precision)
    sa = A.solve(eps=1e-11)
    B.solve(eps=1e-11)  # the V-cycle count the profiled graph unrolls to
    B.profile(True, mode="graph")
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record()
    sb = B.solve(eps=1e-11)
    s1.record()
    torch.cuda.synchronize()
    prof = B.profile_read()
    B.profile(False)
    assert sb["iters"] == sa["iters"]
    # the same kernels in the same order: the same bits
    assert np.array_equal(sb["rel_res"], sa["rel_res"])
    for l in range(A.nlevels):
        assert np.array_equal(A.get(l, "phi"), B.get(l, "phi")), l
    total = sum(v[0] for v in prof.values())
    assert total > 0.0
    assert total <= s0.elapsed_time(s1), (total, s0.elapsed_time(s1))
    assert prof["rbgs"][1] > 0 and prof["residual"][1] > 0
    # the unprofiled graph solve still works afterwards
    sc = B.solve(eps=1e-11)
    assert sc["iters"] == sa["iters"]


def test_eager_profile_matches_graph_solve(amrmg):
    A, B = filled(amrmg, "fp64", 7), filled(amrmg, "fp64", 7)
    sa = A.solve(eps=1e-11)
    B.profile(True)
    sb = B.solve(eps=1e-11)
    prof = B.profile_read()
    B.profile(False)
    assert sb["iters"] == sa["iters"]
    for l in range(A.nlevels):
        a, b = A.get(l, "phi"), B.get(l, "phi")
        assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(a), l
    assert sum(v[1] for v in prof.values()) > 0
