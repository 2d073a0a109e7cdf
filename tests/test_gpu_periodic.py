"""Periodic faces on the GPU (Sec. 5.2) against the FFT closed form and the
FP64 oracle on identical inputs.  The operator is singular (constants):
both sides solve with the neutralised density and return the mean-free
potential, so potentials compare directly.  Tolerances as for the other
faces: operator applications 1e-12, converged potential 1e-10 and field
1e-9 (relative L2); iterates 1e-10 (the singular bottom problem is solved
by different methods on the two sides, equal up to a constant that the
final mean removal takes out)."""
import numpy as np
import pytest

import hierarchies
import oracle
from test_oracle_periodic import fft_solve

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
    "centred": (32, 1, hierarchies.centred(32)),
    "nested": (32, 2, hierarchies.nested_centred(32)),
    "notched": (24, 1, hierarchies.notched(24)),
}


def pair(amrmg, name, precision="fp64"):
    n0, lmax, boxes = CASES[name]
    G = amrmg.Hierarchy(n0, lmax, boxes=boxes, periodic=True, precision=precision)
    O = oracle.OracleHierarchy(n0, lmax, boxes=boxes, periodic=True)
    return G, O


def set_random(G, O, seed, fields=("rho",)):
    rng = np.random.default_rng(seed)
    for l in range(O.nlevels):
        m = O.mask(l) > 0
        for f in fields:
            v = rng.normal(size=O.shape(l)) * m
            G.set(l, f, v)
            O.set(l, f, v)


@pytest.mark.parametrize("n0", [16, 24, 40])
def test_single_level_matches_fft(amrmg, n0):
    G = amrmg.Hierarchy(n0, 0, periodic=True)
    rho = np.random.default_rng(n0).normal(size=(n0, n0, n0))
    G.set(0, "rho", rho)
    st = G.solve(eps=1e-12, max_iter=100)
    assert st["status"] == "AMR_OK", st
    assert relerr(G.get(0, "phi"), fft_solve(rho, 1.0 / n0)) <= 1e-11


@pytest.mark.parametrize("name", list(CASES))
def test_residual_and_field_parity(amrmg, name):
    G, O = pair(amrmg, name)
    set_random(G, O, 51, ("rho", "phi"))
    assert np.allclose(G.residual(), O.residual(), rtol=1e-12, atol=0)
    for l in range(O.nlevels):
        a, b = G.get(l, "res"), O.get(l, "res")
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), (name, l)
    G.field_from_phi()
    O.average_down()
    O.efield()
    for l in range(O.nlevels):
        for f in ("phi", "ex", "ey", "ez"):
            a, b = G.get(l, f), O.get(l, f)
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), (name, l, f)


@pytest.mark.parametrize("name", list(CASES))
def test_iterates_match_oracle(amrmg, name):
    G, O = pair(amrmg, name)
    set_random(G, O, 53)
    for k in (1, 2, 3):
        G.solve(eps=0.0, max_iter=k, bottom_cycles=60)
        O.solve(eps=0.0, max_iter=k, bottom_rtol=1e-16)
        for l in range(O.nlevels):
            e = relerr(G.get(l, "phi"), O.get(l, "phi"))
            assert e <= 1e-10, (name, k, l, e)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_converged_solution_parity(amrmg, name, precision):
    G, O = pair(amrmg, name, precision)
    set_random(G, O, 54)
    st = G.solve(eps=1e-12, max_iter=200)
    assert st["status"] == "AMR_OK" and st["rel_res"].max() <= 1e-12, st
    O.solve(eps=1e-13, max_iter=200, bottom_rtol=1e-15)
    for l in range(O.nlevels):
        assert np.abs(G.get(l, "rho") - O.get(l, "rho")).max() <= 1e-13 * np.abs(O.get(l, "rho")).max()
        assert relerr(G.get(l, "phi"), O.get(l, "phi")) <= 1e-10, (name, l)
        for f in ("ex", "ey", "ez"):
            assert relerr(G.get(l, f), O.get(l, f)) <= 1e-9, (name, l, f)


def test_particles_and_batch_rejection(amrmg):
    """A Gaussian bunch (deposit -> solve -> gather) against the oracle, and
    periodic hierarchies refused by the batched form."""
    from paper_1812_03689_gb300 import inputs
    w = inputs.workload("c1_small")
    parts = w.particles()
    dev = [torch.from_numpy(a).cuda() for a in parts]
    G = amrmg.Hierarchy(w.n0, w.lmax, boxes=w.boxes, particles=dev, periodic=True)
    O = oracle.OracleHierarchy(w.n0, w.lmax, boxes=w.boxes, particles=parts, periodic=True)
    st = G.solve(eps=1e-12)
    assert st["status"] == "AMR_OK"
    O.solve(eps=1e-13, bottom_rtol=1e-15)
    ex, ey, ez = G.gather(*dev[:3])
    g = np.stack([t.cpu().numpy() for t in (ex, ey, ez)])
    assert relerr(g, np.stack(O.gather(*parts[:3]))) <= 1e-9
    with pytest.raises(amrmg.AmrError) as ei:
        amrmg.Batch([G])
    assert ei.value.code == amrmg.AMR_EINVAL
