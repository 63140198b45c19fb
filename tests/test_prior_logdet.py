"""The library's exact prior log-determinant and prior trace terms
(gmrf_prior_logdet, host code: no GPU) against the oracle.

log det Q by the oracle's banded Cholesky, 1/2 tr(Q^-1 dQ/dtheta) by its dense
inverse and exact dQ/dtheta.  The library takes both from the diagonal blocks
of the block lower-bidiagonal root (closed form for symmetric blocks, banded LU
and the band of the inverse otherwise), so agreement at 1e-10 checks that
reduction as well as the arithmetic.  Periodic priors (a single circulant
block on the torus) take the sums over the 2D DFT symbol.
"""
import numpy as np
import pytest

from oracle import fem, infer, linalg
from paper_2503_08343_gb300 import gmrf
from paper_2503_08343_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")

NAMES = ("log_kappa", "log_tau", "c", "nu")


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2503_08343_gb300 import build
    build.build()
    return gmrf.load()


PRIORS = [
    W.prior_st2d(8, 8, 0.5, 0.0, 0.01, 10.0),               # advection: banded LU path
    W.prior_st2d(9, 6, 0.5, 0.2, 0.03, 7.0),                # both velocity components
    W.prior_st2d(8, 5, 0.0, 0.0, 0.03, 7.0),                # no advection: closed form
    W.prior_st1d(12, 7, 0.5, 0.05),
    W.prior_matern2d(11, 5.0),
    W.prior_steady_advdiff2d(10, 5.0, 0.05, 1.2),
    dict(W.prior_st2d(7, 4, 0.3, 0.0, 0.02, 6.0), hi=(1.0, 2.0, 0.5)),   # hx != hy
    dict(W.prior_st1d(14, 6, 0.5, 0.05), noise_kappa=9.0, decay=0.2),   # Matern transition noise, AR decay
    dict(W.prior_st1d(11, 5, 0.0, 0.05), noise_kappa=5.0),
    dict(W.prior_st2d(8, 5, 0.3, 0.0, 0.02, 6.0), decay=0.4),
    W.periodic(W.prior_matern2d(13, 5.0)),                  # torus: DFT symbol
    W.periodic(W.prior_steady_advdiff2d(11, 5.0, 0.05, 1.2)),
    dict(W.periodic(W.prior_steady_advdiff2d(9, 4.0, 0.1, 0.7)), hi=(1.0, 1.5, 0.0)),
]


@pytest.mark.parametrize("prior", PRIORS, ids=lambda p: f"{p['kind']}_{p['n']}_{p['cx']}_{p.get('bc', 'dir')}_{p.get('noise_kappa', 0)}_{p.get('decay', 0)}")
def test_prior_logdet_and_traces_match_the_oracle(prior):
    ld, tr = gmrf.prior_logdet(prior)
    want = linalg.logdet(linalg.cholesky(fem.prior_precision(prior)))
    assert ld == pytest.approx(want, rel=1e-10)
    exact = infer.prior_trace_terms(prior)
    for i, name in enumerate(NAMES):
        assert tr[i] == pytest.approx(exact[name], rel=1e-10, abs=1e-10 * max(1.0, abs(exact[name]))), name


def test_prior_logdet_larger_grid():
    # 26 x 26 x 9 space-time grid (6 084 unknowns, banded Cholesky in the oracle)
    prior = W.prior_st2d(26, 9, 0.5, 0.0, 0.01, 10.0)
    ld, tr = gmrf.prior_logdet(prior)
    assert ld == pytest.approx(linalg.logdet(linalg.cholesky(fem.prior_precision(prior))), rel=1e-10)
    # log tau: Q ~ tau^-2 on every non-boundary row, so the trace is minus their count
    assert tr[1] == pytest.approx(-float((~fem.boundary_mask(prior)).sum()), rel=1e-12)
