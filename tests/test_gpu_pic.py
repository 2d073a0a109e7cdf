"""The particle side of the space-charge step on the GPU (domain transform,
grid rescale, kick-drift push, beam moments) against the numpy oracle, and
a multi-step run of five neighbouring bunches (the paper's multi-bunch
layout, Sec. 6.3) with a regrid every two steps, GPU against oracle step
for step.

Transform, rescale and push are rounded element-wise arithmetic on both
sides: bit-exact.  Moments are FP64 sums in different orders: 1e-12.  The
multi-step run compares positions at 1e-9 and the centre bunch's moments
at 1e-9 after the last step (the field parity of one solve is 1e-9)."""
import numpy as np
import pytest

import oracle
from oracle import pic

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


def host(ts):
    return [t.cpu().numpy() for t in ts]


def bunches(nb=5, n=2000, seed=11):
    g = np.random.default_rng(seed)
    xs, ys, zs = [], [], []
    for b in range(nb):
        xs.append(g.normal(1.0 * (b - nb // 2), 0.25, n))
        ys.append(g.normal(0.0, 0.25, n))
        zs.append(g.normal(0.0, 0.25, n))
    return [np.concatenate(a) for a in (xs, ys, zs)]


def test_transform_push_moments_bit_exact(amrmg):
    x, y, z = bunches()
    c = (0.1, -0.2, 0.05)
    u, v, w, S = amrmg.domain_transform(*cuda(x, y, z), centre=c, delta=0.2)
    ou, ov, ow, oS = pic.domain_transform(x, y, z, c, 0.2)
    assert S == oS
    for a, b in zip(host((u, v, w)), (ou, ov, ow)):
        assert np.array_equal(a, b)
    g = np.random.default_rng(3)
    mom = [g.normal(size=len(x)) for _ in range(3)]
    E = [g.normal(size=len(x)) for _ in range(3)]
    pos_d, mom_d, E_d = cuda(x, y, z), cuda(*mom), cuda(*E)
    amrmg.push(pos_d, mom_d, E_d, -1.5, 0.01)
    pos_o, mom_o = pic.push([x, y, z], mom, E, -1.5, 0.01)
    for a, b in zip(host(pos_d) + host(mom_d), pos_o + mom_o):
        assert np.array_equal(a, b)
    mg = amrmg.moments(*pos_d)
    mo = pic.moments(*pos_o)
    for k in ("centroid", "sigma", "xi"):
        assert np.allclose(mg[k], mo[k], rtol=1e-12, atol=1e-13), k


def test_empty_and_degenerate(amrmg):
    e = torch.zeros(0, dtype=torch.float64, device="cuda")
    with pytest.raises(amrmg.AmrError):
        amrmg.domain_transform(e, e, e)          # no extent
    amrmg.push([e, e, e], [e, e, e], [e, e, e], 1.0, 0.1)
    one = torch.ones(1, dtype=torch.float64, device="cuda")
    m = amrmg.moments(one, one, one)
    assert np.allclose(m["sigma"], 0.0) and np.allclose(m["xi"], 0.0)


def test_rescale_matches_oracle(amrmg):
    x, y, z = bunches(n=1000)
    q = np.full(len(x), 1.0 / len(x))
    u, v, w, S = pic.domain_transform(x, y, z, (0, 0, 0), 0.2)
    G = amrmg.Hierarchy(32, 1, particles=cuda(u, v, w, q), tag_mode="rel", tag_lambda=0.1)
    O = oracle.OracleHierarchy(32, 1, particles=(u, v, w, q), tag_mode="rel", tag_lambda=0.1)
    O.solve(eps=1e-13, bottom_rtol=1e-15)
    O.average_down()
    O.efield()
    for l in range(O.nlevels):
        G.set(l, "phi", O.get(l, "phi"))
    G.field_from_phi()
    G.rescale_fields(S)
    pic.rescale_fields(O, S)
    for l in range(O.nlevels):
        for f in ("phi", "ex", "ey", "ez"):
            a, b = G.get(l, f), O.get(l, f)
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), (l, f)


def test_five_bunch_run_with_regrid(amrmg):
    """Five neighbouring Gaussian bunches in particle space, total charge 1:
    each step maps them into the cube, deposits, solves (1e-12 on the GPU,
    1e-13 in the oracle), rescales, gathers and pushes; every second step
    the hierarchy is regridded by density from the current one (GPU:
    amr_regrid_boxes; oracle: its own regrid); solves start cold (phi was
    rescaled to particle space)."""
    x, y, z = bunches(n=2000)
    n = len(x)
    q = np.full(n, 1.0 / n)
    qm, dt, steps = 40.0, 0.05, 4
    mom = [np.zeros(n) for _ in range(3)]
    pos_o, mom_o = [x, y, z], mom
    pos_d, mom_d, q_d = cuda(x, y, z), cuda(*mom), cuda(q)[0]
    G = O = None
    for k in range(steps):
        # GPU
        u, v, w, S = amrmg.domain_transform(*pos_d, delta=0.2)
        if G is None:
            G = amrmg.Hierarchy(32, 2, particles=(u, v, w, q_d), tag_mode="rel", tag_lambda=0.1)
        elif k % 2 == 0:
            boxes = G.regrid_boxes("rel", 0.1, 2)
            N = amrmg.Hierarchy(32, 2, boxes=boxes)
            N.transfer_phi_from(G)
            G = N
        G.deposit(u, v, w, q_d)
        st = G.solve(eps=1e-12)
        assert st["status"] == "AMR_OK"
        G.rescale_fields(S)
        E_d = G.gather(u, v, w)
        amrmg.push(pos_d, mom_d, E_d, qm, dt)
        # oracle
        ou, ov, ow, oS = pic.domain_transform(*pos_o, (0, 0, 0), 0.2)
        if O is None:
            O = oracle.OracleHierarchy(32, 2, particles=(ou, ov, ow, q), tag_mode="rel", tag_lambda=0.1)
        elif k % 2 == 0:
            O = O.regrid("rel", 0.1, 2, particles=(ou, ov, ow, q))
        else:
            O.deposit(ou, ov, ow, q)
        O.solve(eps=1e-13, bottom_rtol=1e-15)
        O.average_down()
        O.efield()
        pic.rescale_fields(O, oS)
        E_o = O.gather(ou, ov, ow)
        pos_o, mom_o = pic.push(pos_o, mom_o, E_o, qm, dt)
        assert abs(S - oS) <= 1e-12 * oS
        assert G.nlevels == O.nlevels
        for l in range(O.nlevels):
            assert np.array_equal(G.mask(l), O.mask(l)), (k, l)
    got = np.stack(host(pos_d))
    want = np.stack(pos_o)
    moved = np.linalg.norm(want - np.stack([x, y, z]))
    assert moved > 1e-3 * np.linalg.norm(want)          # the bunches did expand
    assert np.linalg.norm(got - want) <= 1e-9 * moved
    centre = slice(2 * 2000, 3 * 2000)
    mg = amrmg.moments(*[t[centre].contiguous() for t in pos_d])
    mo = pic.moments(*[a[centre] for a in pos_o])
    for key in ("sigma", "xi"):
        assert np.allclose(mg[key], mo[key], rtol=1e-9), key
