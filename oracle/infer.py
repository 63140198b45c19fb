"""Conditioning, sampling, variances, Gauss-Newton and the log marginal
likelihood, by the plain definitions (float64, banded Cholesky solves).

Test infrastructure (see the package docstring).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import fem, linalg, observe, rng


@dataclass
class Posterior:
    prior: dict
    B: sp.csr_matrix          # prior root, Q = B^T B
    Q: sp.csr_matrix          # prior precision
    A: sp.csr_matrix          # all observation rows (point data, IC, collocation)
    rinv: np.ndarray          # Q_eps diagonal, 1 / sigma^2 per row
    y: np.ndarray             # observed values per row (offset already removed)
    Qpost: sp.csr_matrix      # Q + A^T Q_eps A
    b: np.ndarray             # A^T Q_eps y


def _point_rows(prior, obs):
    A = observe.point_matrix(prior, np.asarray(obs["coords"], dtype=np.float64))
    y = np.asarray(obs["y"], dtype=np.float64) - np.asarray(obs.get("offset", 0.0))
    rinv = 1.0 / np.asarray(obs["sigma"], dtype=np.float64) ** 2
    return A, rinv, y


def condition(prior: dict, obs: dict, linearise_at: np.ndarray | None = None) -> Posterior:
    """Affine conditioning, Sec. 3.1: Q_u|y = Q + A^T Q_eps A and the
    right-hand side A^T Q_eps (y - A mu - b) with prior mean mu = 0.

    Observation rows, in order: point data; initial-condition rows when
    obs["ic_sigma"] is set (values obs["ic_values"], default the Burgers
    initial condition -sin(pi x)); collocation rows when obs["colloc_sigma"]
    is set, in the form obs["colloc_form"]: "collocation" (default) or
    "fem_cn" (Galerkin-tested Crank-Nicolson rows, observe.fem_cn_residual).
    obs["colloc_stride"] = (sx, st) keeps the rows with i % sx == 0 and
    k % st == 0 (observe.colloc_active; the others get zero weight).
    Linear collocation (obs["colloc_c"] given) uses the constant
    advection speed and right-hand side obs["colloc_f"]; Burgers collocation
    is linearised at `linearise_at` (Sec. 3.3: f(u) ~ f(u_k) + J (u - u_k),
    i.e. rows J with data J u_k - f(u_k)); without it the collocation rows
    are left out (the data-only posterior of Fig. 1).
    """
    B = fem.prior_root(prior)
    Q = (B.T @ B).tocsr()
    A, rinv, y = _point_rows(prior, obs)
    rows, rinvs, ys = [A], [rinv], [y]
    nx, ny, nt = prior["n"]
    if obs.get("ic_sigma") is not None:
        Aic = observe.ic_matrix(prior)
        xs = fem.axis_nodes(prior["lo"][0], prior["hi"][0], nx)
        yic = obs.get("ic_values")
        if yic is None:
            yic = -np.sin(np.pi * xs)
        rows.append(Aic)
        rinvs.append(np.full(Aic.shape[0], 1.0 / obs["ic_sigma"] ** 2))
        ys.append(np.asarray(yic, dtype=np.float64))
    if obs.get("colloc_sigma") is not None:
        nu = obs.get("burgers_nu", prior["nu"])
        if obs.get("colloc_c") is not None:
            J, _ = observe.pde_rows(prior, obs, np.zeros(Q.shape[0]), nu, advect=obs["colloc_c"])
            f = obs.get("colloc_f")
            yc = np.zeros(J.shape[0]) if f is None else np.asarray(f, dtype=np.float64)
        elif linearise_at is not None:
            J, F = observe.pde_rows(prior, obs, linearise_at, nu)
            yc = J @ linearise_at - F
        else:
            J = None
        if J is not None:
            rows.append(J)
            rinvs.append(observe.colloc_active(prior, obs) / obs["colloc_sigma"] ** 2)
            ys.append(yc)
    Aall = sp.vstack(rows).tocsr()
    rinv_all = np.concatenate(rinvs)
    y_all = np.concatenate(ys)
    Qpost = (Q + Aall.T @ sp.diags(rinv_all) @ Aall).tocsr()
    b = Aall.T @ (rinv_all * y_all)
    return Posterior(prior, B, Q, Aall, rinv_all, y_all, Qpost, b)


def posterior_mean(post: Posterior, L=None) -> np.ndarray:
    """mu_u|y = Q_u|y^-1 A^T Q_eps y (Sec. 3.1 eq. posterior-mean), by one
    forward and one backward banded solve (Sec. 3.2)."""
    if L is None:
        L = linalg.cholesky(post.Qpost)
    return linalg.solve(L, post.b)


def marginal_variance(post: Posterior, L=None) -> np.ndarray:
    """Exact diag(Q_u|y^-1) by the Takahashi recursion (Sec. 3.2)."""
    if L is None:
        L = linalg.cholesky(post.Qpost)
    return linalg.takahashi_diag(L)


def sample_rhs(post: Posterior, seed: int, samples) -> np.ndarray:
    """Right-hand sides L z for perturbation samples (Sec. 3.2): with the
    left root L = [B^T, A^T Q_eps^1/2] of Q_u|y = B^T B + A^T Q_eps A (the
    root of a sum) and z = (z1, z2) ~ N(0, I), Q_u|y^-1 L z ~ N(0, Q_u|y^-1).
    z1 (one per row of B) and z2 (one per observation row) are the Philox
    streams 0 and 1 of each sample index.  Returns [len(samples), N]."""
    N = post.Q.shape[0]
    M = post.A.shape[0]
    out = np.empty((len(samples), N))
    sq = np.sqrt(post.rinv)
    for r, s in enumerate(samples):
        z1 = rng.normals(seed, rng.STREAM_PRIOR, int(s), N)
        z2 = rng.normals(seed, rng.STREAM_OBS, int(s), M)
        out[r] = post.B.T @ z1 + post.A.T @ (sq * z2)
    return out


def perturbation_samples(post: Posterior, seed: int, samples, L=None) -> np.ndarray:
    """Zero-mean samples x_s = Q_u|y^-1 L z_s (Sec. 3.2); add the mean for
    posterior samples."""
    if L is None:
        L = linalg.cholesky(post.Qpost)
    R = sample_rhs(post, seed, samples)
    return linalg.solve(L, R.T).T


def rbmc_variance(Qpost: sp.csr_matrix, xs: np.ndarray) -> np.ndarray:
    """Simple Rao-Blackwellised Monte Carlo variance (Siden et al. 2018;
    Sec. 3.2): Var(x_i) = E[Var(x_i | x_-i)] + Var(E[x_i | x_-i]), where for
    a GMRF Var(x_i | x_-i) = 1 / Q_ii and E[x_i | x_-i] = -sum_{j != i}
    Q_ij x_j / Q_ii.  With zero-mean samples x_s:
    v_i = 1/Q_ii + (1/ns) sum_s (sum_{j != i} Q_ij x_{s,j} / Q_ii)^2."""
    d = Qpost.diagonal()
    off = (Qpost - sp.diags(d)).tocsr()
    acc = np.zeros(Qpost.shape[0])
    for x in xs:
        e = (off @ x) / d
        acc += e * e
    return 1.0 / d + acc / len(xs)


# ---------------------------------------------------------------------------
# Gauss-Newton for Burgers collocation (Sec. 3.3)


def neg_log_post(post_lin: Posterior, prior_Q: sp.csr_matrix, obs: dict, prior: dict,
                 u: np.ndarray) -> float:
    """-log pi(u) of eq. nonlinear-post-density up to a constant, prior mean 0:
    1/2 u^T Q u + 1/2 sum_rows Q_eps (y - f(u))^2 over point data, IC rows and
    the (nonlinear) Burgers collocation rows."""
    nx, _, nt = prior["n"]
    val = 0.5 * float(u @ (prior_Q @ u))
    A, rinv, y = _point_rows(prior, obs)
    r = y - A @ u
    val += 0.5 * float(np.sum(rinv * r * r))
    if obs.get("ic_sigma") is not None:
        xs = fem.axis_nodes(prior["lo"][0], prior["hi"][0], nx)
        yic = obs.get("ic_values")
        yic = -np.sin(np.pi * xs) if yic is None else yic
        r = yic - u[:nx]
        val += 0.5 * float(np.sum(r * r)) / obs["ic_sigma"] ** 2
    if obs.get("colloc_sigma") is not None:
        _, f = observe.pde_rows(prior, obs, u, obs.get("burgers_nu", prior["nu"]))
        val += 0.5 * float(np.sum(observe.colloc_active(prior, obs) * f * f)) / obs["colloc_sigma"] ** 2
    return val


def gauss_newton_step(prior: dict, obs: dict, u: np.ndarray, c1: float = 1e-4,
                      max_halvings: int = 20):
    """One Gauss-Newton step on -log pi (Sec. 3.3, eq. nonlinear-mode):
    H = Q + J^T Q_eps J at u, gradient g = Q u - sum_rows J^T Q_eps (y - f(u)),
    direction d = -H^-1 g, then Armijo backtracking from alpha = 1, halving,
    sufficient decrease c1.  Returns (u_next, d, alpha, decrement d^T H d)."""
    post = condition(prior, obs, linearise_at=u)
    H = post.Qpost
    # gradient: H u - b where b = A^T Q_eps (J u - f(u) for collocation, y otherwise)
    g = H @ u - post.b
    L = linalg.cholesky(H)
    d = -linalg.solve(L, g)
    f0 = neg_log_post(post, post.Q, obs, prior, u)
    slope = float(g @ d)
    alpha = 1.0
    for _ in range(max_halvings + 1):
        f1 = neg_log_post(post, post.Q, obs, prior, u + alpha * d)
        if f1 <= f0 + c1 * alpha * slope:
            break
        alpha *= 0.5
    dec = float(d @ (H @ d))
    return u + alpha * d, d, alpha, dec


# ---------------------------------------------------------------------------
# log marginal likelihood of point data (hyper-parameter learning)


def log_marginal_likelihood(prior: dict, obs: dict) -> float:
    """l = log N(y; 0, A Q^-1 A^T + R), evaluated through the GMRF identity
    l = 1/2 logdet Q - 1/2 logdet Q_u|y - 1/2 logdet R - 1/2 y^T R^-1 y
        + 1/2 b^T mu - (M/2) log 2 pi,  b = A^T R^-1 y, mu = Q_u|y^-1 b.
    Not in the paper (which fixes its hyper-parameters); standard Gaussian
    algebra (Rue & Held 2005)."""
    post = condition(prior, obs)
    Lq = linalg.cholesky(post.Q)
    Lp = linalg.cholesky(post.Qpost)
    mu = linalg.solve(Lp, post.b)
    M = post.A.shape[0]
    return (0.5 * linalg.logdet(Lq) - 0.5 * linalg.logdet(Lp)
            + 0.5 * float(np.sum(np.log(post.rinv)))
            - 0.5 * float(np.sum(post.rinv * post.y * post.y))
            + 0.5 * float(post.b @ mu) - 0.5 * M * math.log(2.0 * math.pi))


HYPER = ("log_kappa", "log_tau", "log_sigma", "c", "nu")


def with_hyper(prior: dict, obs: dict, theta: dict):
    """Copies of (prior, obs) with hyper-parameters replaced; theta keys from
    HYPER; kappa acts on kappa0 (the initial block) for space-time priors and
    c on the x velocity."""
    pr = dict(prior)
    ob = dict(obs)
    if "log_kappa" in theta:
        pr["kappa"] = math.exp(theta["log_kappa"])
        if pr["kind"].startswith("advdiff_st"):
            pr["kappa0"] = pr["kappa"]
    if "log_tau" in theta:
        pr["tau"] = math.exp(theta["log_tau"])
    if "log_sigma" in theta:
        ob["sigma"] = np.full(len(obs["y"]), math.exp(theta["log_sigma"]))
    if "c" in theta:
        pr["cx"] = theta["c"]
    if "nu" in theta:
        pr["nu"] = theta["nu"]
    return pr, ob


def hyper_of(prior: dict, obs: dict) -> dict:
    return {"log_kappa": math.log(prior["kappa0"] if prior["kind"].startswith("advdiff_st") else prior["kappa"]),
            "log_tau": math.log(prior["tau"]),
            "log_sigma": math.log(float(np.asarray(obs["sigma"])[0])),
            "c": prior["cx"], "nu": prior["nu"]}


def dQ_dtheta(prior: dict, name: str) -> sp.csr_matrix:
    """Derivative of the prior precision Q = B^T B with respect to one
    hyper-parameter: dQ = dB^T B + B^T dB with the exact root derivative
    fem.prior_root_derivative."""
    B = fem.prior_root(prior)
    dB = fem.prior_root_derivative(prior, name)
    return (dB.T @ B + B.T @ dB).tocsr()


def log_marginal_likelihood_grad(prior: dict, obs: dict) -> dict:
    """Exact gradient of l with respect to (log kappa, log tau, log sigma, c,
    nu) by dense traces (tiny grids only):
    dl = 1/2 tr(Q^-1 dQ) - 1/2 tr(Q_u|y^-1 dQ_u|y) - 1/2 mu^T dQ_u|y mu
         + mu^T db - 1/2 y^T dR^-1 y + 1/2 tr(R dR^-1),
    with dQ_u|y = dQ + A^T dR^-1 A and db = A^T dR^-1 y.  Only point data are
    used (no collocation rows)."""
    post = condition(prior, obs)
    Qd = post.Q.toarray()
    Pd = post.Qpost.toarray()
    Qi = np.linalg.inv(Qd)
    Pi = np.linalg.inv(Pd)
    mu = Pi @ post.b
    A = post.A.toarray()
    y = post.y
    grad = {}
    for name in HYPER:
        if name == "log_sigma":
            # R^-1 = exp(-2 s) I  ->  dR^-1 = -2 R^-1
            drinv = -2.0 * post.rinv
            dP = A.T @ (drinv[:, None] * A)
            db = A.T @ (drinv * y)
            grad[name] = (-0.5 * np.sum(Pi * dP) - 0.5 * mu @ dP @ mu + mu @ db
                          - 0.5 * np.sum(drinv * y * y) + 0.5 * np.sum(drinv / post.rinv))
            continue
        dQ = dQ_dtheta(prior, name).toarray()
        grad[name] = 0.5 * np.sum(Qi * dQ) - 0.5 * np.sum(Pi * dQ) - 0.5 * mu @ dQ @ mu
    return grad


def hutchinson_grad(prior: dict, obs: dict, seed: int, nprobe: int, prior_trace: str = "hutchinson") -> dict:
    """The same gradient with the trace terms replaced by Hutchinson
    estimates on Rademacher probes v_s (Philox stream 2, sample s):
    tr(X^-1 dX) ~ (1/S) sum_s (X^-1 v_s)^T dX v_s, exact solves.  With
    prior_trace="exact" only the posterior trace is estimated and the prior
    one, 1/2 tr(Q^-1 dQ), is taken exactly (dense, tiny grids).  Pinned
    through hutchinson_grad_probes: over all 2^N sign vectors of a tiny
    problem the estimate is the exact gradient."""
    N = condition(prior, obs).Q.shape[0]
    V = np.stack([rng.rademacher(seed, s, N) for s in range(nprobe)])
    return hutchinson_grad_probes(prior, obs, V, prior_trace)


def prior_trace_terms(prior: dict) -> dict:
    """1/2 tr(Q^-1 dQ/dtheta) for theta in (log_kappa, log_tau, c, nu), by a
    dense inverse (tiny grids only)."""
    Qi = np.linalg.inv(fem.prior_precision(prior).toarray())
    return {name: 0.5 * float(np.sum(Qi * dQ_dtheta(prior, name).toarray()))
            for name in ("log_kappa", "log_tau", "c", "nu")}


def hutchinson_grad_probes(prior: dict, obs: dict, V: np.ndarray, prior_trace: str = "hutchinson") -> dict:
    """The Hutchinson gradient on given probe vectors V [S][N]: the mean over
    the probes of the gradient terms with tr(X^-1 dX) replaced by
    v^T X^-1 dX v, and its standard error.  prior_trace="exact" keeps the
    prior trace exact (see hutchinson_grad)."""
    post = condition(prior, obs)
    Lq = linalg.cholesky(post.Q)
    Lp = linalg.cholesky(post.Qpost)
    mu = linalg.solve(Lp, post.b)
    nprobe = V.shape[0]
    Wq = linalg.solve(Lq, V.T).T
    Wp = linalg.solve(Lp, V.T).T
    A = post.A
    y = post.y
    exact_prior = prior_trace_terms(prior) if prior_trace == "exact" else None
    grad, stderr = {}, {}
    for name in HYPER:
        if name == "log_sigma":
            drinv = -2.0 * post.rinv
            dP = (A.T @ sp.diags(drinv) @ A).tocsr()
            db = A.T @ (drinv * y)
            tp = np.array([Wp[s] @ (dP @ V[s]) for s in range(nprobe)])
            val = (-0.5 * tp - 0.5 * mu @ (dP @ mu) + mu @ db
                   - 0.5 * np.sum(drinv * y * y) + 0.5 * np.sum(drinv / post.rinv))
        else:
            dQ = dQ_dtheta(prior, name)
            tp = np.array([Wp[s] @ (dQ @ V[s]) for s in range(nprobe)])
            if exact_prior is None:
                tq = 0.5 * np.array([Wq[s] @ (dQ @ V[s]) for s in range(nprobe)])
            else:
                tq = np.full(nprobe, exact_prior[name])
            val = tq - 0.5 * tp - 0.5 * mu @ (dQ @ mu)
        grad[name] = float(np.mean(val))
        stderr[name] = float(np.std(val, ddof=1) / math.sqrt(nprobe)) if nprobe > 1 else float("inf")
    return grad, stderr
