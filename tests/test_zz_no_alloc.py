"""The allocation-free apply (gmrf_apply_posterior_noalloc) against the
allocating gmrf_apply_posterior.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  The entry point serves
callers that cannot allocate device memory at the moment they need the
product (allocator callbacks, latency-critical loops, fully pooled memory);
its scratch is a fixed array inside the library, shared by all calls, so the
test checks two calls in a row (stale scratch from the first must not leak
into the second).
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12     # same tolerance as the FP64 apply parity test


def _entry():
    from paper_2503_08343_gb300 import build, gmrf
    build.build()
    lib = gmrf.load()
    f = lib.gmrf_apply_posterior_noalloc
    f.restype = C.c_int32
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]
    return gmrf, lib, f


def test_noalloc_apply_matches_the_allocating_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    gmrf, lib, f = _entry()
    from paper_2503_08343_gb300 import workloads as W
    pr, ob = W.c2_matern(n=96, m=400, seed=12)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    rng = np.random.default_rng(5)
    for call in range(2):
        x = rng.normal(size=post.N) * (1.0 + call)
        want = post.apply(x)[0]
        xd = torch.tensor(x, device="cuda")
        yd = torch.full_like(xd, float("nan"))
        q = C.c_double()
        st = f(post.h, C.c_void_p(xd.data_ptr()), C.c_void_p(yd.data_ptr()), C.byref(q))
        assert st == 0, lib.gmrf_last_error().decode()
        y = yd.cpu().numpy()
        assert np.max(np.abs(y - want)) <= TOL * np.max(np.abs(want))
        assert q.value == pytest.approx(float(x @ want), rel=TOL)


def test_noalloc_apply_rejects_systems_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    gmrf, lib, f = _entry()
    from paper_2503_08343_gb300 import workloads as W
    pr, ob = W.c2_matern(n=520, m=50, seed=3)          # 270 400 unknowns > 262 144
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    xd = torch.zeros(post.N, dtype=torch.float64, device="cuda")
    yd = torch.zeros_like(xd)
    st = f(post.h, C.c_void_p(xd.data_ptr()), C.c_void_p(yd.data_ptr()), None)
    assert st == 1
    assert "262144" in lib.gmrf_last_error().decode()
