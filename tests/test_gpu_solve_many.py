"""amr_solve_many: independent hierarchies solved side by side (captured
graphs on several streams) give the same bits as each solved alone, for
uneven hierarchies of the batched workload plus one with Robin and one with
periodic faces (the latter solved after the others; each of its solves
neutralises rho again, a rounding-level change, so it is compared to 1e-12)."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_same_bits_as_alone(amrmg, precision):
    hs = []
    for r in inputs.batched_requests(10):
        parts = [torch.from_numpy(a).cuda() for a in r.particles(3)]
        hs.append(amrmg.Hierarchy(r.n0, r.lmax, particles=parts, precision=precision))
    r = inputs.batched_requests(12)[11]
    parts = [torch.from_numpy(a).cuda() for a in r.particles(3)]
    hs.append(amrmg.Hierarchy(r.n0, r.lmax, particles=parts, precision=precision, robin_d=0.5))
    hs.append(amrmg.Hierarchy(r.n0, r.lmax, particles=parts, precision=precision, periodic=True))
    alone = []
    for h in hs:
        st = h.solve(eps=1e-10)
        assert st["status"] == "AMR_OK"
        alone.append([h.get(l, "phi") for l in range(h.nlevels)])
    for n_streams in (1, 4, 16):
        stats = amrmg.solve_many(hs, n_streams=n_streams, eps=1e-10)
        assert all(s["status"] == "AMR_OK" and s["rel_res"].max() <= 1e-10 for s in stats)
        for i, (h, a) in enumerate(zip(hs, alone)):
            for l in range(h.nlevels):
                got = h.get(l, "phi")
                if i == len(hs) - 1:
                    # periodic: every solve subtracts the mean of rho again
                    # (a rounding-level change), so equal to 1e-12, not bitwise
                    assert np.abs(got - a[l]).max() <= 1e-12 * np.abs(a[l]).max(), (n_streams, i, l)
                else:
                    assert np.array_equal(got, a[l]), (n_streams, i, l)
    with pytest.raises(amrmg.AmrError):
        amrmg.solve_many([hs[0], hs[0]])
