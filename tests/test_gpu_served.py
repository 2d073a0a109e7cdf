"""Served form: the continuous-batching request loop.  Requests admitted
while others run overlap on the device; every result must be the same
alone and in the mix (within the solve tolerance: the deposit's FP64
atomics are not bitwise reproducible), admission respects the HBM budget,
and a request larger than the budget is refused."""
import numpy as np
import pytest

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


def stream(amrmg, n=12):
    g = np.random.default_rng(77)
    reqs = []
    t = 0.0
    for i in range(n):
        t += g.exponential(0.002)
        reqs.append(amrmg.make_request(int(g.integers(4, 9)) * 8, int(g.integers(0, 3)),
                                       int(np.exp(g.uniform(np.log(1e4), np.log(1e5)))), float(g.uniform(0.04, 0.1)),
                                       seed=1000 + i, arrival_s=t,
                                       precision="mixed" if i % 3 == 2 else "fp64"))
    return reqs


def test_same_alone_and_in_the_mix(amrmg):
    reqs = stream(amrmg)
    mix = amrmg.serve(reqs, budget_bytes=64 << 30, max_slots=6, realtime=True, eps=1e-11)
    for i, r in enumerate(reqs):
        assert mix[i]["status"] == 0, (i, mix[i])
        assert mix[i]["rel_res_max"] <= 1e-11
        assert mix[i]["admit_s"] >= mix[i]["arrival_s"] - 1e-9
        assert mix[i]["done_s"] >= mix[i]["admit_s"]
        alone = amrmg.serve([r], budget_bytes=64 << 30, max_slots=1, realtime=False, eps=1e-11)[0]
        assert alone["status"] == 0
        assert alone["iters"] == mix[i]["iters"], i
        a, b = np.array(alone["checksum"]), np.array(mix[i]["checksum"])
        assert np.abs(a - b).max() <= 1e-9 * np.abs(a).max(), (i, a, b)
    # requests really overlapped: some request was admitted before an
    # earlier one completed
    overlap = any(mix[j]["admit_s"] < mix[i]["done_s"] for i in range(len(reqs)) for j in range(i + 1, len(reqs)))
    assert overlap


def test_budget_admission(amrmg):
    reqs = stream(amrmg, 8)
    est = [amrmg.request_bytes(r) for r in reqs]
    budget = int(1.5 * max(est))
    res = amrmg.serve(reqs, budget_bytes=budget, max_slots=8, realtime=False, eps=1e-10)
    assert all(r["status"] == 0 for r in res)
    # at any instant the admitted requests' reservations fit in the budget
    events = sorted({r["admit_s"] for r in res})
    for t in events:
        live = sum(e for e, r in zip(est, res) if r["admit_s"] <= t < r["done_s"])
        assert live <= budget
    big = amrmg.make_request(64, 1, 10000, 0.05, seed=5)
    out = amrmg.serve([big], budget_bytes=1 << 20, max_slots=2, realtime=False)
    assert out[0]["status"] == amrmg.AMR_ENOMEM


def test_generated_bunch_statistics(amrmg):
    """The on-device generator draws the requested Gaussian: a single-level
    deposit of its particles has the right centre and spread."""
    r = amrmg.make_request(32, 0, 200000, 0.07, seed=9)
    res = amrmg.serve([r], budget_bytes=8 << 30, max_slots=1, realtime=False)[0]
    assert res["status"] == 0
    # sum E over a centred symmetric bunch is ~0 relative to sum |E|
    ex, ey, ez, mag = res["checksum"]
    assert max(abs(ex), abs(ey), abs(ez)) < 0.02 * mag
