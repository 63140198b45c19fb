"""Pins of the oracle's Matern transition noise and AR(1) decay in the
space-time prior (App. A: the spatial noise W_s of the transition is a
Matern field; the decay scales the previous level).

With no dynamics (c = nu = 0, so G = Ml) each transition reads
u^k = rho u^(k-1) + Ml^-1 w, w ~ N(0, tau^2 dt Ml Sigma_s Ml), so from Q alone:

* the conditional covariance of the last level given the others (its
  diagonal block inverted) is tau^2 dt Sigma_s on the interior, where the
  unit-variance Matern covariance Sigma_s = (tau_s^2 K Ml^-1 K)^-1 is computed
  here independently by the discrete sine transform of the tridiagonal
  Toeplitz K = kappa_s^2 h + [-1 2 -1]/h (1D, Dirichlet, lumped mass h);
* its conditional mean is rho times the previous level;
* far from the boundary Sigma_s has variance one within the discretisation
  error (the unit-variance normalisation of tau_s);
* the exact root derivative matches central differences of the root.
"""
import math

import numpy as np
import pytest

from oracle import fem, infer
from paper_2503_08343_gb300 import workloads as W


def _sigma_s_dst(m, h, kappa):
    j = np.arange(1, m + 1)
    lam = kappa ** 2 * h + (2.0 - 2.0 * np.cos(j * np.pi / (m + 1))) / h
    V = np.sqrt(2.0 / (m + 1)) * np.sin(np.outer(j, j) * np.pi / (m + 1))
    tau_s = 1.0 / math.sqrt(4.0 * kappa ** 3)
    return (h / tau_s ** 2) * (V * (1.0 / lam ** 2)) @ V.T


def _prior(nx=41, nt=4, ks=12.0, decay=0.0, c=0.0, nu=0.0):
    return dict(W.prior_st1d(nx, nt, c, nu, tau=0.7, kappa0=6.0), noise_kappa=ks, decay=decay)


@pytest.mark.parametrize("decay", [0.0, 0.3])
def test_last_level_conditional_covariance_and_mean(decay):
    pr = _prior(decay=decay)
    nx, _, nt = pr["n"]
    h, _, dt = fem.grid_spacing(pr)
    Q = fem.prior_precision(pr).toarray()
    last = slice((nt - 1) * nx, nt * nx)
    prev = slice((nt - 2) * nx, (nt - 1) * nx)
    I = np.arange(1, nx - 1)
    Qkk = Q[last, last]
    cov = np.linalg.inv(Qkk)[np.ix_(I, I)]
    want = pr["tau"] ** 2 * dt * _sigma_s_dst(nx - 2, h, pr["noise_kappa"])
    assert np.max(np.abs(cov - want)) <= 1e-10 * np.max(np.abs(want))
    # conditional mean of the last level: -Q_kk^-1 Q_k,k-1 u^(k-1) = rho u^(k-1) on the interior
    A = -np.linalg.solve(Qkk, Q[last, prev])[np.ix_(I, I)]
    assert np.max(np.abs(A - (1.0 - decay) * np.eye(nx - 2))) <= 1e-10


def test_matern_noise_has_unit_variance_away_from_the_boundary():
    # kappa_s h = 0.04, centre six ranges from the boundary
    nx, ks = 401, 10.0
    sig = _sigma_s_dst(nx - 2, 1.0 / (nx - 1), ks)
    v = sig[(nx - 2) // 2, (nx - 2) // 2]
    assert abs(v - 1.0) < 0.01, v


def test_white_noise_limit_is_unchanged():
    base = W.prior_st1d(15, 5, 0.4, 0.03)
    B0 = fem.prior_root(base).toarray()
    B1 = fem.prior_root(dict(base, noise_kappa=0.0, decay=0.0)).toarray()
    assert np.array_equal(B0, B1)


@pytest.mark.parametrize("name", ["log_kappa", "log_tau", "c", "nu"])
def test_root_derivative_with_matern_noise(name):
    pr = _prior(nx=13, nt=4, ks=9.0, decay=0.2, c=0.6, nu=0.04)
    th = {"log_kappa": math.log(pr["kappa0"]), "log_tau": math.log(pr["tau"]), "c": pr["cx"], "nu": pr["nu"]}
    eps = 1e-6

    def root(v):
        q = dict(pr)
        if name == "log_kappa":
            q["kappa0"] = math.exp(v)
            q["kappa"] = q["kappa0"]
        elif name == "log_tau":
            q["tau"] = math.exp(v)
        elif name == "c":
            q["cx"] = v
        else:
            q["nu"] = v
        return fem.prior_root(q).toarray()

    fd = (root(th[name] + eps) - root(th[name] - eps)) / (2 * eps)
    dB = fem.prior_root_derivative(pr, name).toarray()
    assert np.max(np.abs(dB - fd)) <= 1e-6 * max(1.0, np.max(np.abs(dB)))
