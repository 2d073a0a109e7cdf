"""The allocation-free norm entry point (amr_masked_norms_noalloc) against
the library's own norms (amr_residual's stopping test).

Callers that cannot allocate device memory (a thread in the middle of a
CUDA graph capture, callers that own the memory pool, real-time loops) use
the allocation-free entry point; it must give the same norms as the
regular path, call after call (its scratch array keeps the previous call's
contents).  This file is collected last on purpose.
"""
import ctypes

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


def noalloc_norms(amrmg, v, mask, covered_too):
    dv = torch.from_numpy(np.ascontiguousarray(v.ravel())).cuda()
    dm = torch.from_numpy(np.ascontiguousarray(mask.ravel().astype(np.uint8))).cuda()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    rc = amrmg._lib.amr_masked_norms_noalloc(ctypes.c_void_p(dv.data_ptr()), ctypes.c_void_p(dm.data_ptr()),
                                              dv.numel(), int(covered_too), ctypes.c_void_p(out.data_ptr()),
                                              ctypes.c_void_p(s.cuda_stream))
    assert rc == 0, amrmg.last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_norms_match_the_library_norms(amrmg):
    H = amrmg.Hierarchy(32, 2, boxes=hierarchies.nested_centred(32))
    rng = np.random.default_rng(90)
    for call in range(2):  # two calls in a row: the shared scratch is reused
        for l in range(H.nlevels):
            m = H.mask(l) > 0
            H.set(l, "rho", rng.normal(size=H.shape(l)) * m)
            H.set(l, "phi", rng.normal(size=H.shape(l)) * m)
        for p, k in ((2, 0), (1, 1), ("inf", 2)):
            rel = H.residual(norm=p)
            rn = []
            for l in range(H.nlevels):
                mask = H.mask(l)
                r = noalloc_norms(amrmg, H.get(l, "res"), mask, 0)
                b = noalloc_norms(amrmg, H.get(l, "rho"), mask, 1)
                val = (np.sqrt(r[0]), np.sqrt(b[0])) if p == 2 else (r[k], b[k])
                rn.append(val)
            bmax = max(b for _, b in rn)
            for l, (r, b) in enumerate(rn):
                want = rel[l]
                got = r / (b if b > 0 else bmax)
                assert abs(got - want) <= 1e-12 * abs(want), (call, p, l, got, want)


def test_noalloc_rejects_oversize_and_handles_empty(amrmg):
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    rc = amrmg._lib.amr_masked_norms_noalloc(ctypes.c_void_p(v.data_ptr()), None, (1 << 26) + 1, 0,
                                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    assert rc == amrmg.AMR_EINVAL and "maximum" in amrmg.last_error()
    out.fill_(7.0)
    rc = amrmg._lib.amr_masked_norms_noalloc(ctypes.c_void_p(v.data_ptr()), None, 0, 0,
                                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert out.cpu().numpy().tolist() == [0.0, 0.0, 0.0]


def test_noalloc_norms_propagate_nan(amrmg):
    # a diverged field: one NaN among finite values makes all three norms NaN,
    # like the library's own norms (the max is taken on the bits of |v|)
    v = np.linspace(-3.0, 2.0, 5000)
    v[1234] = np.nan
    mask = np.ones(v.size, dtype=np.uint8)
    for call in range(2):
        out = noalloc_norms(amrmg, v, mask, 0)
        assert np.isnan(out).all(), (call, out)
    # masked out, the NaN does not count: max |v| is 3 exactly
    mask[1234] = 0
    out = noalloc_norms(amrmg, v, mask, 0)
    assert out[2] == 3.0 and np.isfinite(out).all()
    # an infinite element gives an infinite max (inf sorts below NaN, above the rest)
    v[1234] = -np.inf
    mask[1234] = 2
    out = noalloc_norms(amrmg, v, mask, 1)
    assert out[2] == np.inf
