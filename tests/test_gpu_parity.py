"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances:
* FP64 operator apply: relative 1e-12 (same arithmetic, different summation order);
* posterior means and same-draw samples: relative 1e-6 (max-norm);
* same-draw Rao-Blackwellised variances: relative 1e-3 (sample count stated per test);
* normal draws: absolute 1e-12 (same Philox words; libm rounding may differ).
"""
import math

import numpy as np
import pytest

from oracle import fem, infer, linalg, rng
from paper_2503_08343_gb300 import gmrf
from paper_2503_08343_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

MEAN_TOL = 1e-6
VAR_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2503_08343_gb300 import build
    build.build()
    return gmrf.load()


def _steady_case():
    pr = W.prior_steady_advdiff2d(40, 10.0, nu=0.05, c=1.0)
    ob = W.node_obs(pr, 0.03, 0.05, W.fourier_modes(np.random.default_rng(1), 8, 2, 4), seed=3)
    return pr, ob


def _noise_case():
    pr, ob = W.c1_st1d(nx=37, nt=21, m=40, seed=9)
    return dict(pr, noise_kappa=10.0, decay=0.1), ob


def _torus_advdiff_case():
    pr = W.periodic(W.prior_steady_advdiff2d(41, 8.0, nu=0.1, c=1.5))
    ob = W.point_obs(pr, 250, 0.05, W.periodic_fourier(np.random.default_rng(8), 10, 4), seed=8)
    return pr, ob


CASES = {
    "matern64": lambda: W.c2_matern(n=64, m=400, seed=2),
    "matern45_ragged": lambda: W.c2_matern(n=45, m=150, seed=7, kappa=8.0),
    "st1d_c1_full": lambda: W.c1_st1d(),
    "st1d_37x21_ragged": lambda: W.c1_st1d(nx=37, nt=21, m=30, seed=5),
    "st2d_20x20x12": lambda: W.c5_st2d(n=20, nt=12, m=300, seed=5),
    "steady_advdiff40": _steady_case,
    # periodic boundary (App. B, N_k = 1): 64^2 torus with two coarse levels,
    # and a 40^2 torus with partial tiles at the seam
    "matern_torus64": lambda: W.c2_matern_periodic(n=65, m=400, seed=3, kappa=10.0),
    "advdiff_torus40": lambda: _torus_advdiff_case(),
    # Matern transition noise and AR(1) decay in the 1D space-time prior (App. A)
    "st1d_noise_37x21": lambda: _noise_case(),
}


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _elementwise(got, want, Qpost, tol):
    """Element by element: |got - want| <= tol (|want| + s) with s the
    conditional standard deviation 1/sqrt(Q_ii) of the node, a per-node scale
    that follows the solution across orders of magnitude (Dirichlet rows:
    eps = 1e-4) and does not vanish where the mean crosses zero."""
    s = 1.0 / np.sqrt(Qpost.diagonal())
    err = np.abs(got - want)
    lim = tol * (np.abs(want) + s)
    return float(np.max(err / lim))


@pytest.fixture(scope="module")
def built():
    out = {}
    for name, mk in CASES.items():
        pr, ob = mk()
        gp = gmrf.Prior(pr)
        post = gmrf.Posterior(gp, ob)
        orc = infer.condition(pr, ob)
        out[name] = (pr, ob, gp, post, orc, linalg.cholesky(orc.Qpost))
    return out


def test_normal_draws_match_the_oracle_generator():
    for (seed, stream, s0) in [(1002, 0, 0), (7, 1, 5), (2 ** 40 + 3, 0, 63)]:
        g = gmrf.normals(seed, stream, s0, 3, 1001)
        for s in range(3):
            o = rng.normals(seed, stream, s0 + s, 1001)
            assert np.max(np.abs(g[s] - o)) < 1e-12


def test_normal_draws_match_the_oracle_generator_in_volume():
    # 2^20 draws per (stream, sample): the table-driven logarithm's branch
    # next to u = 1 (about 1 uniform in 128) and every table entry are hit
    for (seed, stream, s0) in [(31, 0, 2), (2 ** 33 + 5, 1, 17)]:
        g = gmrf.normals(seed, stream, s0, 2, 1 << 20)
        for s in range(2):
            o = rng.normals(seed, stream, s0 + s, 1 << 20)
            assert np.max(np.abs(g[s] - o)) < 1e-12
            assert np.min(np.abs(o)) < 1e-4 and np.max(np.abs(o)) > 4.5


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_apply_matches_assembled_posterior_precision(built, name):
    pr, ob, gp, post, orc, _ = built[name]
    x = np.random.default_rng(0).normal(size=(5, orc.Q.shape[0]))
    y = post.apply(x)
    want = (orc.Qpost @ x.T).T
    assert _rel(y, want) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_posterior_mean(built, name):
    pr, ob, gp, post, orc, L = built[name]
    mu, info = post.solve_mean()
    want = infer.posterior_mean(orc, L)
    assert info["converged"] == 1
    assert _rel(mu, want) < MEAN_TOL, info
    assert _elementwise(mu, want, orc.Qpost, MEAN_TOL) <= 1.0


@pytest.mark.parametrize("name", list(CASES))
def test_samples_with_identical_draws(built, name):
    pr, ob, gp, post, orc, L = built[name]
    seed, ns = 1001, 6
    mu, xs, info = post.sample(ns, seed)
    want = infer.perturbation_samples(orc, seed, range(ns), L)
    assert _rel(xs, want) < MEAN_TOL
    assert _rel(mu, infer.posterior_mean(orc, L)) < MEAN_TOL
    assert _elementwise(xs, want, orc.Qpost, MEAN_TOL) <= 1.0


@pytest.mark.parametrize("name", list(CASES))
def test_rbmc_variance_with_identical_draws(built, name):
    pr, ob, gp, post, orc, L = built[name]
    seed, ns = 77, 16
    mu, var, se, info = post.marginal_var(ns, seed)
    xs = infer.perturbation_samples(orc, seed, range(ns), L)
    want = infer.rbmc_variance(orc.Qpost, xs)
    assert _rel(var, want) < VAR_TOL
    # element by element, Dirichlet rows (variance eps2 = 1e-8) included
    assert np.all(np.abs(var - want) <= VAR_TOL * want)
    assert np.all(se >= 0)


def test_c1_variances_against_takahashi_statistically(built):
    # 256 samples (the C1 configuration); |v - v_exact| <= 4 stderr on >= 99 % of nodes
    pr, ob, gp, post, orc, L = built["st1d_c1_full"]
    mu, var, se, info = post.marginal_var(256, 1001)
    exact = linalg.takahashi_diag(L)
    ok = np.abs(var - exact) <= 4 * se + 1e-12 * exact
    assert ok.mean() >= 0.99
    assert _rel(mu, infer.posterior_mean(orc, L)) < MEAN_TOL


def test_prior_only_posterior_has_zero_mean():
    pr = W.prior_matern2d(33, 5.0)
    ob = dict(coords=np.zeros((0, 2)), y=np.zeros(0), sigma=np.zeros(0))
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    mu, info = post.solve_mean()
    assert np.all(mu == 0.0)
    _, xs, _ = post.sample(2, 5, mean=False)
    orc = infer.condition(pr, ob)
    assert _rel(xs, infer.perturbation_samples(orc, 5, range(2))) < MEAN_TOL


def test_observations_on_edges_corners_and_duplicates():
    pr = W.prior_matern2d(17, 4.0)
    c = np.array([[0.0, 0.0], [1.0, 1.0], [1.0, 0.3], [0.5, 0.5], [0.5, 0.5], [0.25, 0.125], [1 / 16, 5 / 16]])
    ob = dict(coords=c, y=np.arange(len(c), dtype=float), sigma=np.full(len(c), 0.1))
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    mu, _ = post.solve_mean()
    orc = infer.condition(pr, ob)
    assert _rel(mu, infer.posterior_mean(orc)) < MEAN_TOL


def test_device_tensors_in_and_out_and_update_data():
    torch = pytest.importorskip("torch")
    pr, ob = W.c2_matern(n=48, m=120, seed=9)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    y2 = np.asarray(ob["y"]) * -0.5 + 0.1
    post.update_data(torch.tensor(y2, device="cuda"))
    out = torch.empty(post.N, dtype=torch.float64, device="cuda")
    post.solve_mean(out=out)
    ob2 = dict(ob, y=y2)
    assert _rel(out.cpu().numpy(), infer.posterior_mean(infer.condition(pr, ob2))) < MEAN_TOL


def test_plain_fp64_single_rhs_path_agrees():
    pr, ob = W.c2_matern(n=40, m=100, seed=4)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    opts = gmrf.default_opts(precision=1, batched=0, max_inner=400)
    mu, xs, info = post.sample(3, 11, opts=opts)
    orc = infer.condition(pr, ob)
    assert _rel(xs, infer.perturbation_samples(orc, 11, range(3))) < MEAN_TOL
    assert _rel(mu, infer.posterior_mean(orc)) < MEAN_TOL


def test_plain_fp64_path_on_densely_observed_coarse_levels():
    # 32^3 space-time grid with 5000 observations: on the 16^3 coarse level
    # every node of a tile carries an observation entry, and the FP64 tables
    # (256 x 27 coefficients per tile) no longer fit in shared memory beside
    # the staged inputs, so the kernel reads them from global memory
    pr, ob = W.c5_st2d(n=32, nt=32, m=5000, seed=8)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    assert [lv[:3] for lv in post.level_info()][:2] == [(32, 32, 32), (16, 16, 16)]
    mu32, info32 = post.solve_mean()
    mu64, info64 = post.solve_mean(opts=gmrf.default_opts(precision=1, batched=0, max_inner=2000))
    assert info32["converged"] == 1 and info64["converged"] == 1
    assert _rel(mu64, mu32) < 1e-8


def test_invalid_arguments_are_rejected():
    bad = W.prior_matern2d(2, 4.0)
    with pytest.raises(gmrf.GmrfError) as e:
        gmrf.Prior(bad)
    assert e.value.status == 1
    pr = W.prior_matern2d(9, 4.0)
    gp = gmrf.Prior(pr)
    with pytest.raises(gmrf.GmrfError) as e:
        gmrf.Posterior(gp, dict(coords=np.array([[0.5, 0.5]]), y=np.array([1.0]), sigma=np.array([0.0])))
    assert e.value.status == 1


def test_iteration_caps_report_no_convergence():
    pr, ob = W.c2_matern(n=64, m=200, seed=2)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    opts = gmrf.default_opts(max_refine=1, max_inner=2, rtol=1e-14)
    with pytest.raises(gmrf.GmrfError) as e:
        post.solve_mean(opts=opts)
    assert e.value.status == 3


def test_wall_clock_limit_reports_timeout():
    pr, ob = W.c2_matern(n=64, m=200, seed=2)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    opts = gmrf.default_opts(timeout_s=1e-9)
    with pytest.raises(gmrf.GmrfError) as e:
        post.solve_mean(opts=opts)
    assert e.value.status == 6
    mu, info = post.solve_mean()        # the handle stays usable
    assert info["converged"] == 1


@pytest.mark.slow
def test_full_size_matern_512_in_the_bench_configuration():
    # The bench workload (512 x 512, 10 000 observations, mean + 64 samples,
    # default options): mean against banded Cholesky, variances against the
    # oracle's estimator on the same 64 draws.
    pr, ob = W.c2_matern()
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    seed = W.DRAW_SEED["c2"]
    mu, var, se, info = post.marginal_var(64, seed)
    orc = infer.condition(pr, ob)
    L = linalg.cholesky(orc.Qpost)
    assert _rel(mu, infer.posterior_mean(orc, L)) < MEAN_TOL
    xs = infer.perturbation_samples(orc, seed, range(64), L)
    want = infer.rbmc_variance(orc.Qpost, xs)
    assert _rel(var, want) < VAR_TOL
    assert np.all(np.abs(var - want) <= VAR_TOL * want)


def test_bounded_tile_wait_failure_is_reported_and_the_handle_recovers():
    # The staged-tile waits of the stencil kernels give up without polling
    # (gmrf_test_set_wait_cap(-1)): the copies are still landing, so the CTAs
    # record the device flag, drain their in-flight copies with the normal cap
    # and return.  The solve and the FP64 apply must report GMRF_E_CUDA; with
    # the default cap restored the same handle solves correctly again.
    lib = gmrf.load()
    pr, ob = W.c2_matern(n=96, m=300, seed=6)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    x = np.random.default_rng(2).normal(size=post.N)
    try:
        lib.gmrf_test_set_wait_cap(-1)
        with pytest.raises(gmrf.GmrfError) as e:
            post.solve_mean()
        assert e.value.status == 4
        with pytest.raises(gmrf.GmrfError) as e:
            post.apply(x)
        assert e.value.status == 4
    finally:
        lib.gmrf_test_set_wait_cap(0)
    mu, info = post.solve_mean()
    assert info["converged"] == 1
    orc = infer.condition(pr, ob)
    assert _rel(mu, infer.posterior_mean(orc)) < MEAN_TOL
    assert _rel(post.apply(x)[0], orc.Qpost @ x) < 1e-12


def test_reserved_batch_allocates_nothing_later():
    # after gmrf_reserve(17), mean + 16 samples + variances and the mean alone
    # (a batch of 1 needs its own reservation) leave the free device memory
    # unchanged
    torch = pytest.importorskip("torch")
    pr, ob = W.c2_matern(n=130, m=500, seed=11)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    post.reserve(17)
    post.reserve(1)
    var = torch.empty(post.N, dtype=torch.float64, device="cuda")
    mu = torch.empty_like(var)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for seed in (3, 4):
        post.marginal_var(16, seed, out=var)
        post.solve_mean(out=mu)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    orc = infer.condition(pr, ob)
    assert _rel(mu.cpu().numpy(), infer.posterior_mean(orc)) < MEAN_TOL
