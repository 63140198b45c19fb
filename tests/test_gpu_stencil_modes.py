"""Every mode of the fused stencil kernels, FP32 and FP64, element by element
against the oracle's assembled operator (gmrf_stencil_step through the C ABI).

In the FP32-inner / FP64-refinement solver the FP32 stencil modes only
precondition: a wrong FP32 apply or Chebyshev step would still give correct
means, just after more iterations.  So each mode is checked here directly:

  apply             out = Q x
  residual          out = b - Q x
  Chebyshev         out2 = c1 d + c2 D^-1 (b - Q x),  out = x + out2
  Chebyshev-from-0  x1 = c0 D^-1 b, then the Chebyshev step with x = d = x1
  PCG               p' = d + beta x, out = Q p', iterate b + alpha x (the
                    conjugate-gradient iteration's vector work around the apply)

with Q the level's posterior precision (Sec. 3.1: Q + A^T Q_eps A, collocation
rows included) and D its diagonal.  The reference is computed in FP64 from the
inputs as the kernel sees them (rounded to FP32 for the FP32 kernels).  The
tolerance is the forward-error bound of the arithmetic, element by element:
|out - ref| <= gamma * m, where m is the same expression evaluated on
absolute values (|B|^T |B| |x| + |A|^T Q_eps |A| |x| for Q x, since the kernel
forms B^T (B x) and the observation term) and gamma = 64 u in FP32 (u = 2^-24:
a few dozen roundings on each path) and 1e-12 in FP64 (see GAMMA).  The per-RHS
dot products the kernel also returns (x^T Q x, |r|^2, b^T x_new) get twice
gamma on the sum of absolute terms (each thread adds a few dozen FP32 terms
before the FP64 reduction).

Geometries: the tiled 2D and 1D space-time kernel, the marching 2D space-time
kernel, ragged tiles, periodic tori (seam tiles), dense observations, linear and linearised Burgers
collocation rows and their FEM Crank-Nicolson form, Matern transition noise, the full-size 2D Matern workload (512^2, 10 000
observations, 65 right-hand sides) and the first coarse multigrid level
(rediscretised prior with the point data interpolated on the coarse mesh).
"""
import zlib

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import infer, observe
from paper_2503_08343_gb300 import gmrf
from paper_2503_08343_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

U = {0: 2.0 ** -24, 1: 2.0 ** -53}
# bound factor per unit roundoff: FP32 64 u; FP64 1e-12 / u (~4500), since the
# library and the oracle compute the observation weights from the coordinates
# by different formulas: they agree to a few ulps of x / h (~1e-14 here), and
# an observation placed on a node can get a rounding-level weight on a
# neighbour in one of them and exactly zero in the other, which the |A| in the
# bound cannot see (measured up to 1.9e-13 of the bound; without observations
# the FP64 kernel stays within 4e-15)
GAMMA = {0: 64 * 2.0 ** -24, 1: 1e-12}
C0, C1, C2 = 0.37, 0.61, 0.83


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2503_08343_gb300 import build
    build.build()
    return gmrf.load()


def _linear_colloc(form="collocation"):
    pr, ob = W.c1_st1d(nx=37, nt=21, m=30, seed=5)
    f = np.random.default_rng(3).normal(size=(37 - 2) * (21 - 1))
    return pr, dict(ob, colloc_sigma=0.05, colloc_c=0.5, burgers_nu=0.01, colloc_f=f, colloc_form=form)


CASES = {
    "matern45_ragged": (lambda: W.c2_matern(n=45, m=150, seed=7, kappa=8.0), 5),
    "steady_advdiff40": (lambda: (W.prior_steady_advdiff2d(40, 10.0, nu=0.05, c=1.0),
                                  W.node_obs(W.prior_steady_advdiff2d(40, 10.0, nu=0.05, c=1.0), 0.03, 0.05,
                                             W.fourier_modes(np.random.default_rng(1), 8, 2, 4), seed=3)), 4),
    "st1d_37x21_ragged": (lambda: W.c1_st1d(nx=37, nt=21, m=30, seed=5), 6),
    "st1d_linear_collocation": (_linear_colloc, 3),
    "st1d_linear_fem_cn": (lambda: _linear_colloc("fem_cn"), 3),
    "st1d_linear_colloc_strided": (lambda: (_linear_colloc()[0], dict(_linear_colloc()[1], colloc_stride=(3, 2))), 3),
    "st1d_noise_ragged": (lambda: (dict(W.c1_st1d(nx=37, nt=21, m=30, seed=5)[0], noise_kappa=8.0, decay=0.15),
                                   W.c1_st1d(nx=37, nt=21, m=30, seed=5)[1]), 5),
    "st2d_20x20x12_march": (lambda: W.c5_st2d(n=20, nt=12, m=300, seed=5), 3),
    "st2d_24x24x10_dense_obs": (lambda: W.c5_st2d(n=24, nt=10, m=5000, seed=3), 2),
    # periodic boundary: tiles at the seam take their halo from the other side
    "matern_torus40_ragged": (lambda: W.c2_matern_periodic(n=41, m=300, seed=9, kappa=8.0), 5),
    "advdiff_torus32": (lambda: (W.periodic(W.prior_steady_advdiff2d(33, 6.0, nu=0.2, c=1.1)),
                                 W.point_obs(W.periodic(W.prior_steady_advdiff2d(33, 6.0, nu=0.2, c=1.1)), 2000, 0.05,
                                             W.periodic_fourier(np.random.default_rng(2), 6, 3), seed=4)), 3),
}


def _bound_matrix(post, jabs=None):
    """|B|^T |B| + |A|^T Q_eps |A|: the absolute-value form of how the
    kernel evaluates Q (the stacked root twice, then the observation rows).
    jabs replaces |A| on the collocation rows (the last rows of A)."""
    aB = abs(post.B)
    aA = abs(post.A)
    if jabs is not None:
        aA = sp.vstack([aA[:aA.shape[0] - jabs.shape[0]], jabs]).tocsr()
    return (aB.T @ aB + aA.T @ sp.diags(post.rinv) @ aA).tocsr()


def _colloc_abs(pr, ob, u):
    """|J| as the kernel forms the linearised Burgers rows: each coefficient
    is a fixed part (time and diffusion terms) plus terms linear in the
    linearisation point, and it rounds on the size of those terms, not of
    their sum (an advection tap can cancel the diffusion tap).  The convective
    part J(v) - J(0) is linear in v and each of its coefficients reads u at
    one or two nodes of a level, at x distance 0, 1 or 2; the absolute-value
    form of such a coefficient is the largest |J(v) - J(0)| over v = s |u|
    with the sign patterns s = 1, (-1)^x and (+1 for x mod 4 in {0, 1}, -1
    otherwise), which give every such pair of nodes both equal and opposite
    signs."""
    nx = pr["n"][0]
    nu = ob["burgers_nu"]
    J0 = observe.pde_rows(pr, ob, np.zeros_like(u), nu)[0].tocsr()
    x = np.arange(u.size) % nx
    conv = None
    for sgn in (np.ones(u.size), (-1.0) ** x, np.where(x % 4 < 2, 1.0, -1.0)):
        c = abs(observe.pde_rows(pr, ob, sgn * np.abs(u), nu)[0].tocsr() - J0)
        conv = c if conv is None else conv.maximum(c)
    return (abs(J0) + conv).tocsr()


def _check_modes(post_gpu, post_o, k, level, prec, seed, modes=(0, 1, 2, 3, 4), jabs=None):
    rng = np.random.default_rng(seed)
    N = post_o.Q.shape[0]
    rnd = lambda: rng.normal(size=(k, N))
    x, b, d = rnd(), rnd(), rnd()
    if prec == 0:
        f32 = lambda v: v.astype(np.float32).astype(np.float64)
        x, b, d = f32(x), f32(b), f32(d)
        c0, c1, c2 = (float(np.float32(c)) for c in (C0, C1, C2))
    else:
        c0, c1, c2 = C0, C1, C2
    Q = post_o.Qpost
    M = _bound_matrix(post_o, jabs)
    dinv = 1.0 / Q.diagonal()
    g, gd = GAMMA[prec], 2 * GAMMA[prec]
    Qx = (Q @ x.T).T
    Mx = (M @ np.abs(x).T).T

    def close(got, want, bound, what):
        err = np.abs(got - want)
        bad = err > g * bound + 1e-300
        assert not bad.any(), (what, float((err / np.maximum(bound, 1e-300)).max()), int(bad.sum()))

    if 0 in modes:
        out, _, dots = post_gpu.stencil_step(0, x=x, level=level, precision=prec)
        close(out, Qx, Mx, "apply")
        assert np.all(np.abs(dots - np.sum(x * Qx, axis=1)) <= gd * np.sum(np.abs(x) * Mx, axis=1))
    if 1 in modes:
        out, _, dots = post_gpu.stencil_step(1, x=x, b=b, level=level, precision=prec)
        r = b - Qx
        br = np.abs(b) + Mx
        close(out, r, br, "residual")
        assert np.all(np.abs(dots - np.sum(r * r, axis=1)) <= gd * np.sum(2 * (np.abs(r) + g * br) * br, axis=1))
    if 2 in modes:
        out, out2, dots = post_gpu.stencil_step(2, x=x, b=b, d=d, level=level, precision=prec, c1=c1, c2=c2)
        dn = c1 * d + c2 * dinv * (b - Qx)
        bdn = abs(c1) * np.abs(d) + abs(c2) * dinv * (np.abs(b) + Mx)
        close(out2, dn, bdn, "chebyshev d")
        close(out, x + dn, np.abs(x) + 2 * bdn, "chebyshev x")
        assert np.all(np.abs(dots - np.sum(b * (x + dn), axis=1))
                      <= gd * np.sum(np.abs(b) * (np.abs(x) + 2 * bdn), axis=1))
    if 4 in modes and post_o.prior["kind"] != "advdiff_st2d":     # the marching kernel has no PCG mode
        # p' = d + beta x, q = Q p', iterate b + alpha x (x the previous
        # direction, d the preconditioned residual)
        al, be = (c1, c2) if prec == 1 else (float(np.float32(0.31)), float(np.float32(0.57)))
        q, pn, dots, xn = post_gpu.stencil_step(4, x=x, b=b, d=d, level=level, precision=prec, c1=al, c2=be)
        pref = d + be * x
        apn = np.abs(d) + abs(be) * np.abs(x)
        close(pn, pref, apn, "pcg direction")
        Qp = (Q @ pref.T).T
        Mp = (M @ apn.T).T
        close(q, Qp, 2 * Mp, "pcg apply")
        close(xn, b + al * x, np.abs(b) + abs(al) * np.abs(x), "pcg iterate")
        assert np.all(np.abs(dots - np.sum(pref * Qp, axis=1)) <= gd * np.sum(2 * apn * Mp, axis=1))
    if 3 in modes:
        out, out2, dots = post_gpu.stencil_step(3, b=b, level=level, precision=prec, c0=c0, c1=c1, c2=c2)
        x1 = c0 * dinv * b
        ax1 = np.abs(x1)
        Qx1 = (Q @ x1.T).T
        dn = c1 * x1 + c2 * dinv * (b - Qx1)
        bdn = abs(c1) * ax1 + abs(c2) * dinv * (np.abs(b) + (M @ ax1.T).T)
        close(out2, dn, bdn + ax1, "chebyshev-from-zero d")
        close(out, x1 + dn, 2 * (ax1 + bdn), "chebyshev-from-zero x")
        assert np.all(np.abs(dots - np.sum(b * (x1 + dn), axis=1))
                      <= gd * np.sum(np.abs(b) * 2 * (ax1 + bdn), axis=1))


def _coarse_prior(pr, dims):
    pc = dict(pr)
    pc["n"] = tuple(int(v) for v in dims)
    if pr.get("bc") == "periodic":      # level dims count torus nodes; the prior counts both ends
        pc["n"] = (pc["n"][0] + 1, pc["n"][1] + 1, 1)
    return pc


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "fp64"])
@pytest.mark.parametrize("name", list(CASES))
def test_stencil_modes_match_the_oracle_operator(name, prec):
    mk, k = CASES[name]
    pr, ob = mk()
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    _check_modes(post, infer.condition(pr, ob), k, 0, prec, seed=zlib.crc32(name.encode()) % 1000)


@pytest.mark.parametrize("name", ["matern45_ragged", "steady_advdiff40", "st1d_37x21_ragged", "st1d_noise_ragged",
                                  "st2d_20x20x12_march", "st2d_24x24x10_dense_obs", "matern_torus40_ragged"])
def test_stencil_modes_on_the_first_coarse_level(name):
    # the coarse operator is the rediscretised prior with the same point data
    # interpolated on the coarse mesh
    mk, k = CASES[name]
    pr, ob = mk()
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    dims = post.level_info()[1][:3]
    orc = infer.condition(_coarse_prior(pr, dims), ob)
    assert orc.Q.shape[0] == int(np.prod(dims))
    _check_modes(post, orc, k, 1, 0, seed=11)


@pytest.mark.parametrize("form", ["collocation", "fem_cn", "noise", "strided", "fem_cn_strided"])
def test_stencil_modes_burgers_linearised(form):
    # collocation (or FEM Crank-Nicolson) rows of the Burgers residual
    # linearised at the Gauss-Newton iterate the library holds after one step
    # (Sec. 3.3); "strided": collocation points on every fourth node in x and
    # t (sigma 1e-3, as in the Gauss-Newton test)
    pr, ob = W.c3_burgers(nx=65, nt=33, m=40)
    if form == "noise":         # Matern transition noise in the prior, collocation rows
        pr = dict(pr, noise_kappa=12.0)
    else:
        ob = dict(ob, colloc_form=form.replace("_strided", "").replace("strided", "collocation"))
    if form.endswith("strided"):
        ob = dict(ob, colloc_stride=(4, 4), colloc_sigma=1e-3)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    u, _ = post.solve_mean()
    d = np.zeros_like(u)
    try:
        post.gauss_newton_step(u, d, opts=gmrf.default_opts(max_refine=3))
    except gmrf.GmrfError:
        pass            # a step stopped at its caps still leaves the rows linearised at the returned u
    orc = infer.condition(pr, ob, linearise_at=u)
    jabs = _colloc_abs(pr, ob, u)
    for prec in (0, 1):
        _check_modes(post, orc, 5, 0, prec, seed=21 + prec, modes=(0, 1, 4), jabs=jabs)


def test_stencil_modes_full_size_matern_65_rhs():
    # the bench workload: 512^2, 10 000 observations, 65 right-hand sides (FP32)
    pr, ob = W.c2_matern()
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    _check_modes(post, infer.condition(pr, ob), 65, 0, 0, seed=5)
