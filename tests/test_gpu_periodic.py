"""Periodic boundary (App. B, N_k = 1) on the GPU at full size, against the
DFT solution (tests/torus_symbol.py; no Cholesky).

With every node of the 512^2 torus observed once with equal noise sigma,
Q_u|y = Q + sigma^-2 I is circulant: the posterior mean is one DFT solve and
the posterior variance is the same at every node,
(1/N) sum_w 1/(|b(w)|^2 + sigma^-2).  The library solves it with its
multigrid-preconditioned mixed-precision PCG on the torus (seam tiles take
their halo from the other side, transfers wrap), so the mean must agree to
relative 1e-6 and the Rao-Blackwellised variance, averaged over the
262 144 nodes, to 1 % (64 samples).  The medium-size parity cases (oracle
Cholesky) are in test_gpu_parity.py and test_gpu_stencil_modes.py.
"""
import numpy as np
import pytest

from paper_2503_08343_gb300 import gmrf
from paper_2503_08343_gb300 import workloads as W

import torus_symbol as TS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2503_08343_gb300 import build
    build.build()
    return gmrf.load()


@pytest.mark.parametrize("sigma", [0.1, 0.02])
def test_full_size_torus_all_nodes_observed_matches_the_dft_solve(sigma):
    pr, ob = W.c2_matern_periodic(n=513, all_nodes=True, sigma=sigma, seed=11)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    assert post.N == 512 * 512
    mu, info = post.solve_mean()
    assert info["converged"] == 1
    want = TS.all_nodes_mean(pr, ob["y"], sigma)
    err = np.max(np.abs(mu - want)) / np.max(np.abs(want))
    assert err <= 1e-6, (err, info)


def test_full_size_torus_variance_closed_form():
    sigma = 0.1
    pr, ob = W.c2_matern_periodic(n=513, all_nodes=True, sigma=sigma, seed=12)
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    mean, var, se, info = post.marginal_var(64, 5)
    assert info["converged"] == 1
    b, m = TS.symbol(pr)
    want = float(np.mean(1.0 / (np.abs(b) ** 2 + 1.0 / sigma ** 2)))
    assert abs(float(np.mean(var)) - want) <= 1e-2 * want
    # translation invariance: no seam or tile pattern in the estimate
    v = var.reshape(m, m)
    assert abs(float(np.mean(v[:, 0])) - want) <= 5e-2 * want and abs(float(np.mean(v[0, :])) - want) <= 5e-2 * want


def test_torus_prior_logdet_is_the_symbol_sum():
    pr = W.periodic(W.prior_steady_advdiff2d(65, 6.0, nu=0.2, c=1.3))
    ld, _ = gmrf.prior_logdet(pr)
    b, m = TS.symbol(pr)
    assert ld == pytest.approx(float(np.sum(np.log(np.abs(b) ** 2))), rel=1e-11)
