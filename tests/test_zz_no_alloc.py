"""The allocation-free apply (gmrf_apply_posterior_noalloc) against the
allocating gmrf_apply_posterior.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  The entry point serves
callers that cannot allocate device memory at the moment they need the
product (allocator callbacks, latency-critical loops, fully pooled memory);
its scratch is a fixed array inside the library, shared by all calls, so the
test makes calls in a row on posteriors of every stencil geometry, the
largest first (stale scratch from an earlier, bigger call must not leak into
a later, smaller one).
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


def _check_calls(gmrf, lib, f, post, rng, calls):
    torch = pytest.importorskip("torch")
    for call in range(calls):
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


def test_noalloc_apply_matches_the_allocating_entry_point_on_two_calls():
    pytest.importorskip("torch")
    gmrf, lib, f = _entry()
    from paper_2503_08343_gb300 import workloads as W
    pr, ob = W.c2_matern(n=96, m=400, seed=12)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    _check_calls(gmrf, lib, f, post, np.random.default_rng(5), 2)


def test_noalloc_apply_every_geometry_largest_first():
    # 2D space-time (marching kernel), 1D space-time with linear collocation
    # rows, then a small 2D spatial posterior: each call uses less scratch
    # than the one before it
    pytest.importorskip("torch")
    gmrf, lib, f = _entry()
    from paper_2503_08343_gb300 import workloads as W
    st2, ob2 = W.c5_st2d(n=40, nt=40, m=800, seed=9)              # 64 000 unknowns
    st1, ob1 = W.c1_st1d(nx=70, nt=60, m=40, seed=4)              # 4 200 unknowns
    ob1 = dict(ob1, colloc_sigma=0.05, colloc_c=0.5, burgers_nu=0.01)
    sp2, obs2 = W.c2_matern(n=33, m=60, seed=8, kappa=6.0)        # 1 089 unknowns
    rng = np.random.default_rng(11)
    for pr, ob in ((st2, ob2), (st1, ob1), (sp2, obs2)):
        post = gmrf.Posterior(gmrf.Prior(pr), ob)
        _check_calls(gmrf, lib, f, post, rng, 2)


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
