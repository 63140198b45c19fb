"""Log marginal likelihood and its gradient on the GPU against the oracle.

The library takes the prior terms exactly (log det Q and 1/2 tr(Q^-1 dQ) from
the diagonal blocks of the root), the posterior trace by Hutchinson probes from
one batched posterior solve [mean + probes], and log det Q_u|y by stochastic
Lanczos quadrature on the same probes.

* Same probes: the gradient equals the oracle's estimator with the prior trace
  exact and the posterior trace on the same Rademacher probes with exact
  solves (oracle.infer.hutchinson_grad(..., prior_trace="exact")) to relative
  1e-6.
* The gradient agrees with the exact dense gradient (itself pinned by central
  finite differences, h = 1e-4) within 4 standard errors.
* The value agrees with the oracle's exact log marginal likelihood within 4
  standard errors (16^3 and 8^3 replicas of the 2D space-time workload and
  the other prior kinds); its exact part log det Q to 1e-10.
"""
import numpy as np
import pytest

from oracle import fem, infer, linalg
from paper_2503_08343_gb300 import gmrf
from paper_2503_08343_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

NAMES = ["log_kappa", "log_tau", "log_sigma", "c", "nu"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2503_08343_gb300 import build
    build.build()
    return gmrf.load()


CASES = {
    "st2d_16cubed": lambda: W.c5_st2d(n=16, nt=16, m=300, seed=5),
    "st2d_8cubed": lambda: W.c5_st2d(n=8, nt=8, m=60, seed=6),
    "st1d_24x20": lambda: W.c1_st1d(nx=24, nt=20, m=40, seed=7),
    "steady_advdiff_24": lambda: (W.prior_steady_advdiff2d(24, 8.0, nu=0.05, c=1.2),
                                  W.point_obs(W.prior_steady_advdiff2d(24, 8.0, nu=0.05, c=1.2), 80, 0.1,
                                              lambda z: np.sin(4 * z[:, 0]) * z[:, 1], seed=9)),
    "matern_24": lambda: W.c2_matern(n=24, m=60, seed=4, kappa=6.0),
    "advdiff_torus_24": lambda: (W.periodic(W.prior_steady_advdiff2d(25, 7.0, nu=0.1, c=0.9)),
                                 W.point_obs(W.periodic(W.prior_steady_advdiff2d(25, 7.0, nu=0.1, c=0.9)), 90, 0.1,
                                             W.periodic_fourier(np.random.default_rng(3), 6, 3), seed=10)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_gradient_matches_oracle_estimator_and_exact_gradient(name):
    pr, ob = CASES[name]()
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    seed, S = 77, 32
    ll, g, se, info = post.loglik_grad(S, seed)
    assert info["converged"] == 1
    est, est_se = infer.hutchinson_grad(pr, ob, seed, S, prior_trace="exact")
    exact = infer.log_marginal_likelihood_grad(pr, ob)
    names = NAMES if pr["kind"] != "matern2d" else ["log_kappa", "log_tau", "log_sigma"]
    for i, nm in enumerate(NAMES):
        if nm not in names:
            assert g[i] == 0.0            # the Matern kind has no advection or diffusion parameter
            continue
        assert abs(g[i] - est[nm]) <= 1e-6 * max(1.0, abs(est[nm])), (nm, g[i], est[nm])
        assert se[i] == pytest.approx(est_se[nm], rel=1e-4, abs=1e-9)
        assert abs(g[i] - exact[nm]) <= 4.0 * se[i] + 1e-8 * max(1.0, abs(exact[nm])), (nm, g[i], exact[nm], se[i])


@pytest.mark.parametrize("name", list(CASES))
def test_log_marginal_likelihood_value(name):
    pr, ob = CASES[name]()
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    ll, g, se, info = post.loglik_grad(32, 91)
    li = info["loglik"]
    assert li["lanczos_converged"] == 1, li
    want = infer.log_marginal_likelihood(pr, ob)
    assert abs(ll - want) <= 4.0 * li["loglik_stderr"], (ll, want, li)
    assert li["logdet_prior"] == pytest.approx(linalg.logdet(linalg.cholesky(fem.prior_precision(pr))), rel=1e-10)
    # the estimate of log det Q_u|y is unbiased: its error is the Monte Carlo error
    post_o = infer.condition(pr, ob)
    ld_post = linalg.logdet(linalg.cholesky(post_o.Qpost))
    assert abs(li["logdet_post"] - ld_post) <= 8.0 * li["loglik_stderr"]


def test_value_is_not_computed_for_gradient_only_calls():
    pr, ob = CASES["st2d_8cubed"]()
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    ll, g, se, info = post.loglik_grad(16, 3, value=False)
    assert ll is None and "loglik" not in info
    _, g2, _, _ = post.loglik_grad(16, 3)
    assert np.array_equal(g, g2)


def test_autograd_function_value_and_gradient():
    import torch
    pr, ob = CASES["st1d_24x20"]()
    theta0 = gmrf.hyper_of(pr, ob)
    pr2, ob2 = gmrf.with_hyper(pr, ob, theta0)
    assert pr2["kappa0"] == pytest.approx(pr["kappa0"]) and pr2["tau"] == pytest.approx(pr["tau"])
    theta = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    ll = gmrf.log_marginal_likelihood(theta, pr, ob, nprobes=16, seed=5)
    (3.0 * ll).backward()
    want_ll, want_g, want_se, want_info = gmrf.Posterior(gmrf.Prior(pr2), ob2).loglik_grad(16, 5)
    assert ll.item() == pytest.approx(want_ll, rel=1e-12)
    assert np.allclose(theta.grad.numpy(), 3.0 * want_g, rtol=1e-12, atol=0)
    # the value is the log marginal likelihood (within its standard error)
    exact0 = infer.log_marginal_likelihood(pr2, ob2)
    assert abs(ll.item() - exact0) <= 4.0 * want_info["loglik"]["loglik_stderr"]
    # central differences of the returned value (same probes) against the
    # returned gradient: two unbiased estimates of the same derivative from
    # the same probes, so they agree within a few gradient standard errors
    h = 1e-3
    for i in range(5):
        tp, tm = theta0.copy(), theta0.copy()
        tp[i] += h
        tm[i] -= h
        fp = gmrf.log_marginal_likelihood(torch.tensor(tp), pr, ob, nprobes=16, seed=5).item()
        fm = gmrf.log_marginal_likelihood(torch.tensor(tm), pr, ob, nprobes=16, seed=5).item()
        fd = (fp - fm) / (2 * h)
        assert abs(fd - want_g[i]) <= 6.0 * want_se[i] + 1e-4 * max(1.0, abs(want_g[i])), (i, fd, want_g[i], want_se[i])
    # one gradient-ascent step on the hyper-parameters moves the exact objective up
    step = 1e-3 * theta.grad.numpy() / np.linalg.norm(theta.grad.numpy())
    pr3, ob3 = gmrf.with_hyper(pr, ob, theta0 + step)
    assert infer.log_marginal_likelihood(pr3, ob3) > exact0
