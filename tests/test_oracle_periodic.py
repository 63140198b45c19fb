"""Pins of the oracle's periodic boundary (App. B, N_k = 1) against closed
forms that do not go through its element loops.

On the torus every operator of the structured P1 mesh is circulant, so it is
diagonalised by the 2D DFT; tests/torus_symbol.py derives the symbols of the
root B and of Q = B^T B by hand from the element integrals.  Pins:

* B v and Q v equal their DFT forms (a row or column left out of the mirror
  condensation, a wrong mass or a wrong sign of the advection fails);
* the prior variance at every node equals (1/N) sum_w 1/|b(w)|^2 (Takahashi
  on the oracle's Cholesky factor, 1e-10) and log det Q = sum_w log |b(w)|^2;
* point rows: a point on x = hi or y = hi is its mirror on x = lo or y = lo,
  and a point in the last cell shares its weight with column 0;
* all torus nodes observed with equal noise: Q_u|y is circulant and the
  posterior mean is a DFT solve (1e-10);
* the exact derivative of B against central differences of prior_root.
"""
import math

import numpy as np
import pytest

from oracle import fem, infer, linalg, observe
from paper_2503_08343_gb300 import workloads as W

import torus_symbol as TS


_symbol = TS.symbol
_apply_symbol = TS.apply_symbol


PRIORS = {
    "matern_24": lambda: W.periodic(W.prior_matern2d(25, 6.0)),
    "matern_16_k20": lambda: W.periodic(W.prior_matern2d(17, 20.0)),
    "advdiff_20": lambda: W.periodic(W.prior_steady_advdiff2d(21, 5.0, nu=0.3, c=1.7)),
}


@pytest.mark.parametrize("name", list(PRIORS))
def test_root_and_precision_are_the_circulants_of_the_closed_form_symbol(name):
    pr = PRIORS[name]()
    b, m = _symbol(pr)
    B = fem.prior_root(pr)
    Q = fem.prior_precision(pr)
    assert B.shape == (m * m, m * m)
    v = np.random.default_rng(3).normal(size=m * m)
    # (B v)_n = sum_d B[n, n + d] v_(n+d): the symbol uses exp(+i w.d), i.e. b
    # as written (the advection stencil's offsets are those of the columns)
    Bv = _apply_symbol(b, v, m)
    assert np.max(np.abs(B @ v - Bv)) <= 1e-12 * np.max(np.abs(Bv))
    Qv = _apply_symbol(np.abs(b) ** 2, v, m)
    assert np.max(np.abs(Q @ v - Qv)) <= 1e-12 * np.max(np.abs(Qv))


@pytest.mark.parametrize("name", list(PRIORS))
def test_prior_variance_and_log_det_closed_form(name):
    pr = PRIORS[name]()
    b, m = _symbol(pr)
    lam = np.abs(b) ** 2
    L = linalg.cholesky(fem.prior_precision(pr))
    var = linalg.takahashi_diag(L)
    want = np.mean(1.0 / lam)
    assert np.max(np.abs(var - want)) <= 1e-10 * want
    assert linalg.logdet(L) == pytest.approx(float(np.sum(np.log(lam))), rel=1e-12, abs=1e-9)


def test_point_rows_wrap_to_the_mirror_nodes():
    pr = PRIORS["matern_24"]()
    m = pr["n"][0] - 1
    h = 1.0 / m
    pts = np.array([[1.0, 0.3], [0.0, 0.3], [0.37, 1.0], [0.37, 0.0], [1.0, 1.0], [0.0, 0.0],
                    [1.0 - 0.25 * h, 0.5 + 0.1 * h]])
    A = observe.point_matrix(pr, pts).toarray()
    assert A.shape == (len(pts), m * m)
    assert np.allclose(A.sum(axis=1), 1.0, atol=1e-14)
    for a, b in ((0, 1), (2, 3), (4, 5)):
        assert np.max(np.abs(A[a] - A[b])) <= 1e-14, (a, b)
    assert abs(A[5, 0] - 1.0) <= 1e-14
    # near the seam: weight on the last column and on column 0 (the mirror of x = hi)
    j = int(0.5 * m)
    assert A[6, j * m + m - 1] > 0.2 and A[6, j * m + 0] > 0.5


def test_all_nodes_observed_posterior_mean_is_a_dft_solve():
    pr, ob = W.c2_matern_periodic(n=25, kappa=6.0, all_nodes=True, sigma=0.2, seed=4)
    post = infer.condition(pr, ob)
    mu = infer.posterior_mean(post)
    want = TS.all_nodes_mean(pr, ob["y"], 0.2)
    assert np.max(np.abs(mu - want)) <= 1e-10 * np.max(np.abs(want))


@pytest.mark.parametrize("name", ["matern_24", "advdiff_20"])
def test_root_derivative_against_central_differences(name):
    pr = PRIORS[name]()
    theta = {"log_kappa": math.log(pr["kappa"]), "log_tau": math.log(pr["tau"]), "c": pr["cx"], "nu": pr["nu"]}
    names = ["log_kappa", "log_tau"] + (["c", "nu"] if pr["kind"] != "matern2d" else [])
    for nm in names:
        hstep = 1e-6

        def root(v):
            q = dict(pr)
            if nm == "log_kappa":
                q["kappa"] = math.exp(v)
            elif nm == "log_tau":
                q["tau"] = math.exp(v)
            elif nm == "c":
                q["cx"] = v
            else:
                q["nu"] = v
            return fem.prior_root(q).toarray()

        fd = (root(theta[nm] + hstep) - root(theta[nm] - hstep)) / (2 * hstep)
        dB = fem.prior_root_derivative(pr, nm).toarray()
        assert np.max(np.abs(dB - fd)) <= 1e-6 * max(1.0, np.max(np.abs(dB))), nm
