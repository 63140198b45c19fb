"""FEM (Galerkin-tested) Crank-Nicolson PDE observations on the implicit-Euler
space-time prior (Sec. 3.1 FEM observations; Sec. 5, Crank-Nicolson FEM
observations of Burgers' equation) on the GPU against the oracle.

* Linear advection-diffusion rows (colloc 3): the posterior mean and
  same-draw samples, in the energy norm of Q_u|y at 1e-6 and in the max-norm
  at 1e-6 plus four times the oracle's own FP64 uncertainty (one refinement
  step of its Cholesky solution), as for the collocation rows.
* Burgers rows (colloc 4): Gauss-Newton iterates, step lengths and the first
  Newton decrement against the oracle's exact-solve Gauss-Newton, and
  Laplace samples at the returned point.
Every stencil mode with these rows is in test_gpu_stencil_modes.py.
"""
import math

import numpy as np
import pytest

from oracle import infer, linalg, observe
from paper_2503_08343_gb300 import gmrf
from paper_2503_08343_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2503_08343_gb300 import build
    build.build()
    return gmrf.load()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _burgers_fem(n, nt, nu, sigma):
    pr, ob = W.c3_burgers(nx=n, nt=nt, m=60, seed=3, nu=nu)
    return pr, dict(ob, colloc_form="fem_cn", colloc_sigma=sigma)


def _linear_fem(n, sigma):
    # rows int phi_i f of the manufactured solution u* = exp(-t) sin(pi x) of
    # u_t + c u_x - nu u_xx = f (f sampled at the row's node and the level
    # midpoint, times h: any right-hand side serves the parity test)
    c, nu = 0.5, 0.05
    pr = W.prior_st1d(n, n, c, nu, tau=1.0, kappa0=5.0)
    i, k = observe.colloc_rows(pr)
    h = 1.0 / (n - 1)
    x = np.linspace(0, 1, n)[i]
    t = (np.linspace(0, 1, n)[k] + np.linspace(0, 1, n)[k - 1]) / 2
    f = h * ((-1 + nu * math.pi ** 2) * np.exp(-t) * np.sin(math.pi * x) + c * math.pi * np.exp(-t) * np.cos(math.pi * x))
    xs = np.linspace(0, 1, n)
    ob = dict(coords=np.array([[0.3, 0.4], [0.7, 0.9]]), y=np.array([0.5, 0.2]), sigma=np.array([0.1, 0.1]),
              ic_sigma=1e-6, ic_values=np.sin(math.pi * xs), colloc_sigma=sigma, colloc_c=c, colloc_f=f, burgers_nu=nu,
              colloc_form="fem_cn")
    return pr, ob


@pytest.mark.parametrize("n,sigma", [(33, 1e-4), (49, 1e-6)])
def test_linear_fem_cn_posterior_mean_and_samples(n, sigma):
    pr, ob = _linear_fem(n, sigma)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    mu, xs, info = post.sample(3, 77)
    assert info["converged"] == 1
    orc = infer.condition(pr, ob)
    L = linalg.cholesky(orc.Qpost)
    H = orc.Qpost
    hn = lambda v: float(np.sqrt(v @ (H @ v)))
    mu_o = infer.posterior_mean(orc, L)
    corr = np.max(np.abs(linalg.solve(L, orc.b - H @ mu_o)))
    assert hn(mu - mu_o) <= 1e-6 * hn(mu_o)
    assert np.max(np.abs(mu - mu_o)) <= 1e-6 * np.max(np.abs(mu_o)) + 4.0 * corr
    xs_o = infer.perturbation_samples(orc, 77, range(3), L)
    for s in range(3):
        assert hn(xs[s] - xs_o[s]) <= 1e-6 * hn(xs_o[s]), s


@pytest.mark.parametrize("n,nt,nu,sigma", [(65, 33, 0.05, 1e-4), (65, 33, 0.02, 1e-6)])
def test_burgers_fem_cn_gauss_newton_iterates(n, nt, nu, sigma):
    pr, ob = _burgers_fem(n, nt, nu, sigma)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    u_gpu, info = post.solve_mean()
    u_or = infer.posterior_mean(infer.condition(pr, ob))
    assert _rel(u_gpu, u_or) < 1e-6
    u_gpu = u_or.copy()
    d_gpu = np.zeros_like(u_gpu)
    for step in range(3):
        u_next, d_or, alpha_or, dec_or = infer.gauss_newton_step(pr, ob, u_or)
        dec, alpha, info = post.gauss_newton_step(u_gpu, d_gpu)
        assert info["converged"] == 1
        assert alpha == alpha_or, step
        H = infer.condition(pr, ob, linearise_at=u_or).Qpost
        hn = lambda v: float(np.sqrt(v @ (H @ v)))
        assert hn(d_gpu - d_or) <= 1e-6 * hn(d_or), step
        if step == 0:
            assert dec == pytest.approx(dec_or, rel=1e-6)
        assert _rel(u_gpu, u_next) < 1e-6, step
        u_or = u_next


def test_burgers_fem_cn_laplace_samples():
    pr, ob = _burgers_fem(65, 33, 0.05, 1e-4)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    u = infer.posterior_mean(infer.condition(pr, ob))
    d = np.zeros_like(u)
    for _ in range(4):
        post.gauss_newton_step(u, d)
    mu, xs, info = post.sample(4, 321)
    assert info["converged"] == 1
    lap = infer.condition(pr, ob, linearise_at=u)
    L = linalg.cholesky(lap.Qpost)
    assert _rel(xs, infer.perturbation_samples(lap, 321, range(4), L)) < 1e-6
    assert _rel(mu, linalg.solve(L, lap.b)) < 1e-6
