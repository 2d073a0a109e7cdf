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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def with_fields(amrmg, reqs):
    """Each request with its own device buffer for Ex, Ey, Ez, phi."""
    bufs = [torch.zeros(4 * r.n_particles, dtype=torch.float64, device="cuda") for r in reqs]
    for r, b in zip(reqs, bufs):
        r.field_out = b.data_ptr()
    return bufs


def test_same_alone_and_in_the_mix(amrmg):
    # every request's gathered E and phi, element by element, alone and in
    # the mix (spec tolerances: phi 1e-10, E 1e-9, relative L2 and
    # largest difference relative to the largest value); the two runs differ
    # only in the order of the deposit's FP64 atomic additions
    reqs = stream(amrmg)
    mix_f = with_fields(amrmg, reqs)
    mix = amrmg.serve(reqs, budget_bytes=64 << 30, max_slots=6, realtime=True, eps=1e-11)
    torch.cuda.synchronize()
    for i, r in enumerate(reqs):
        assert mix[i]["status"] == 0, (i, mix[i])
        assert mix[i]["rel_res_max"] <= 1e-11
        assert mix[i]["admit_s"] >= mix[i]["arrival_s"] - 1e-9
        assert mix[i]["done_s"] >= mix[i]["admit_s"]
        one = [r]
        alone_f = with_fields(amrmg, one)
        alone = amrmg.serve(one, budget_bytes=64 << 30, max_slots=1, realtime=False, eps=1e-11)[0]
        torch.cuda.synchronize()
        assert alone["status"] == 0
        assert alone["iters"] == mix[i]["iters"], i
        n = r.n_particles
        a = alone_f[0].cpu().numpy().reshape(4, n)
        b = mix_f[i].cpu().numpy().reshape(4, n)
        assert np.isfinite(a).all() and np.abs(a[:3]).max() > 0
        assert rel_l2(b[:3], a[:3]) <= 1e-9, (i, rel_l2(b[:3], a[:3]))
        assert np.abs(b[:3] - a[:3]).max() <= 1e-9 * np.abs(a[:3]).max(), i
        assert rel_l2(b[3], a[3]) <= 1e-10, (i, rel_l2(b[3], a[3]))
        assert np.abs(b[3] - a[3]).max() <= 1e-10 * np.abs(a[3]).max(), i
        ca, cb = np.array(alone["checksum"]), np.array(mix[i]["checksum"])
        assert np.abs(ca - cb).max() <= 1e-9 * np.abs(ca).max(), (i, ca, cb)
    # requests really overlapped: some request was admitted before an
    # earlier one completed
    overlap = any(mix[j]["admit_s"] < mix[i]["done_s"] for i in range(len(reqs)) for j in range(i + 1, len(reqs)))
    assert overlap


def test_served_requests_match_oracle(amrmg):
    # host-generated bunches (the seeded input generator) through the same
    # request loop, several at once, against the oracle on the same
    # particles and the same density-tagged hierarchy
    import oracle
    from paper_1812_03689_gb300 import inputs
    specs = [(32, 1, 20000, 0.06, "fp64"), (40, 2, 30000, 0.08, "fp64"), (32, 2, 25000, 0.07, "mixed"),
             (48, 1, 15000, 0.1, "mixed")]
    host, dev, reqs = [], [], []
    for k, (n0, lmax, npart, sigma, prec) in enumerate(specs):
        parts = inputs.gaussian_bunches(inputs.rng(40, k), npart, [[0.5, 0.5, 0.5]], sigma, 1.0 / n0)
        host.append(parts)
        d = [torch.from_numpy(a).cuda() for a in parts]
        dev.append(d)
        reqs.append(amrmg.make_request(n0, lmax, npart, sigma, seed=k, precision=prec, particles=d))
    bufs = with_fields(amrmg, reqs)
    res = amrmg.serve(reqs, budget_bytes=32 << 30, max_slots=4, realtime=False, eps=1e-12)
    torch.cuda.synchronize()
    for k, ((n0, lmax, npart, sigma, prec), parts) in enumerate(zip(specs, host)):
        assert res[k]["status"] == 0, (k, res[k])
        O = oracle.OracleHierarchy(n0, lmax, particles=parts, tag_mode="rel", tag_lambda=0.1)
        assert O.nlevels == res[k]["n_levels"], k
        O.solve(eps=1e-13, bottom_rtol=1e-15)
        oex, oey, oez, ophi = O.gather(*parts[:3], with_phi=True)
        g = bufs[k].cpu().numpy().reshape(4, npart)
        E, oE = g[:3], np.stack([oex, oey, oez])
        assert rel_l2(E, oE) <= 1e-9, (k, rel_l2(E, oE))
        assert np.abs(E - oE).max() <= 1e-9 * np.abs(oE).max(), k
        assert rel_l2(g[3], ophi) <= 1e-10, (k, rel_l2(g[3], ophi))
        assert np.abs(g[3] - ophi).max() <= 1e-10 * np.abs(ophi).max(), k


def test_device_bytes_within_admission_estimate(amrmg):
    # what a request really holds on the device (its hierarchy plus the
    # slot's seven particle arrays) never exceeds the estimate admission
    # reserves for it
    specs = [(32, 0, 10000, 0.05), (32, 3, 50000, 0.03), (40, 2, 20000, 0.1), (64, 1, 100000, 0.1),
             (64, 3, 200000, 0.04), (96, 2, 100000, 0.06), (128, 2, 300000, 0.05), (56, 3, 30000, 0.1)]
    reqs = [amrmg.make_request(n0, lmax, npart, sigma, seed=300 + k, precision="mixed" if k % 2 else "fp64")
            for k, (n0, lmax, npart, sigma) in enumerate(specs)]
    res = amrmg.serve(reqs, budget_bytes=64 << 30, max_slots=4, realtime=False, eps=1e-10)
    for r, out in zip(reqs, res):
        assert out["status"] == 0, out
        held = out["device_bytes"] + 56 * r.n_particles
        est = amrmg.request_bytes(r)
        assert held <= est, (r.n0, r.max_level, out["n_levels"], held, est)


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


def test_hierarchy_byte_cap(amrmg):
    # amr_desc.max_device_bytes: creation fails with AMR_ENOMEM (nothing kept)
    # instead of holding more than the cap
    H = amrmg.Hierarchy(64, 0)
    need = H.device_bytes()
    H.close()
    with pytest.raises(amrmg.AmrError) as ei:
        amrmg.Hierarchy(64, 0, max_device_bytes=need // 2)
    assert ei.value.code == amrmg.AMR_ENOMEM and "max_device_bytes" in str(ei.value)
    G = amrmg.Hierarchy(64, 0, max_device_bytes=need + (1 << 20))
    assert G.device_bytes() <= need + (1 << 20)
    G.close()


@pytest.mark.timeout(300)
def test_budget_holds_when_a_request_outgrows_its_charge(amrmg):
    # A request is created under its charge as a hard cap.  Charged a fifth of
    # its estimate, a request's hierarchy outgrows the charge: the creation
    # fails, the charge goes back, and the request runs again alone with the
    # whole budget as the cap.  Every request completes with its solo result
    # and none ever holds more than the budget.
    big = amrmg.make_request(64, 3, 20000, 0.1, seed=701)
    small = [amrmg.make_request(32, 1, 20000, 0.06, seed=800 + k) for k in range(3)]
    reqs = [small[0], big, small[1], small[2]]
    solo = [amrmg.serve([r], budget_bytes=64 << 30, max_slots=1, realtime=False, eps=1e-10)[0] for r in reqs]
    assert all(s["status"] == 0 and not s["retried"] for s in solo), solo
    held = solo[1]["device_bytes"] + 56 * big.n_particles
    assert held > amrmg.request_bytes(big) // 5
    budget = held + (64 << 20)
    res = amrmg.serve(reqs, budget_bytes=budget, max_slots=4, realtime=False, admit_fraction=0.2, eps=1e-10)
    assert res[1]["retried"]
    for r, out, s in zip(reqs, res, solo):
        assert out["status"] == 0, out
        assert out["device_bytes"] + 56 * r.n_particles <= budget
        assert out["device_bytes"] == s["device_bytes"]
        assert np.abs(out["checksum"] - s["checksum"]).max() <= 1e-9 * np.abs(s["checksum"]).max()
