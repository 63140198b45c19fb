"""Pins for the oracle's inference (no GPU): dense GP conditioning (Woodbury
route, eq. gp-posterior-cov), Kalman / RTS smoothing of the state-space model
(Sec. 2.4), manufactured-solution convergence of collocation, exactness of
the Rao-Blackwellised estimator in expectation, Philox statistics, the
Gaussian marginal likelihood with finite-difference gradients, and the
Burgers Jacobian by finite differences."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.stats as st

from oracle import fem, infer, linalg, observe, rng
from paper_2503_08343_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def test_point_weights_interpolate_linear_functions_exactly():
    for prior in (W.prior_matern2d(9, 3.0), W.prior_st1d(9, 7, 0.3, 0.01), W.prior_st2d(6, 5, 0.2, 0.1, 0.01, 3.0)):
        ob = W.point_obs(prior, 40, 0.1, lambda z: np.zeros(len(z)), seed=5)
        A = observe.point_matrix(prior, ob["coords"])
        nx, ny, nt = prior["n"]
        lo, hi = prior["lo"], prior["hi"]
        X = np.tile(np.linspace(lo[0], hi[0], nx), ny * nt)
        Y = np.tile(np.repeat(np.linspace(lo[1], hi[1], ny), nx), nt) if ny > 1 else 0 * X
        T = np.repeat(np.linspace(lo[2], hi[2], nt), nx * ny) if nt > 1 else 0 * X
        c = ob["coords"]
        assert np.allclose(A.sum(axis=1), 1.0)
        assert (A.data >= -1e-14).all()
        assert np.allclose(A @ X, c[:, 0])
        if prior["kind"] == "advdiff_st1d":
            assert np.allclose(A @ T, c[:, 1])
        elif ny > 1:
            assert np.allclose(A @ Y, c[:, 1])
            if nt > 1:
                assert np.allclose(A @ T, c[:, 2])


@pytest.mark.parametrize("prior", [W.prior_matern2d(12, 4.0), W.prior_st1d(10, 9, 0.5, 0.02),
                                   W.prior_st2d(6, 5, 0.4, 0.0, 0.02, 4.0)], ids=lambda p: p["kind"])
def test_conditioning_matches_dense_gp(prior):
    ob = W.point_obs(prior, 30, 0.05, lambda z: np.sin(3 * z[:, 0]) + z[:, -1], seed=11)
    post = infer.condition(prior, ob)
    C = np.linalg.inv(post.Q.toarray())
    A = post.A.toarray()
    S = A @ C @ A.T + np.diag(1.0 / post.rinv)
    mean_gp = C @ A.T @ np.linalg.solve(S, post.y)
    cov_gp = C - C @ A.T @ np.linalg.solve(S, A @ C)
    L = linalg.cholesky(post.Qpost)
    mu = infer.posterior_mean(post, L)
    var = infer.marginal_variance(post, L)
    assert np.allclose(mu, mean_gp, rtol=1e-9, atol=1e-10 * np.abs(mean_gp).max())
    assert np.allclose(var, np.diag(cov_gp), rtol=1e-9)
    assert (var <= np.diag(C) * (1 + 1e-12)).all()       # posterior var <= prior var


def _kalman_rts(prior, times_idx, obs_rows, yv, rinv):
    """Textbook Kalman filter + RTS smoother on u^(k) = A u^(k-1) + e, e ~ N(0, F),
    u^(0) ~ N(0, Q1^-1), observations at grid time levels only."""
    S, ml, Badv, dim = fem.spatial_mesh(prior)
    sb = fem.spatial_boundary(prior)
    nt = prior["n"][2]
    dt = (prior["hi"][2] - prior["lo"][2]) / (nt - 1)
    tau, eps2 = prior["tau"], prior["eps2"]
    K0 = fem.constrain(prior["kappa0"] ** 2 * sp.diags(ml) + S, sb).toarray()
    G = fem.constrain(sp.diags(ml) + dt * (prior["nu"] * S + Badv), sb).toarray()
    Mc = np.diag(np.where(sb, 0.0, ml))
    tau0 = fem.matern_tau_unit(prior["kappa0"], dim)
    Q1 = K0.T @ np.diag(np.where(sb, 1.0 / eps2, (tau0 / tau) ** 2 / ml)) @ K0
    Gi = np.linalg.inv(G)
    Atr = Gi @ Mc
    F = Gi @ np.diag(np.where(sb, eps2, tau * tau * dt * ml)) @ Gi.T
    Ns = len(ml)
    mp, Pp, mf, Pf = [], [], [], []
    m, P = np.zeros(Ns), np.linalg.inv(Q1)
    for k in range(nt):
        if k > 0:
            m, P = Atr @ m, Atr @ P @ Atr.T + F
        mp.append(m)
        Pp.append(P)
        sel = [r for r in range(len(times_idx)) if times_idx[r] == k]
        if sel:
            H = obs_rows[sel]
            Sk = H @ P @ H.T + np.diag(1.0 / rinv[sel])
            Kg = P @ H.T @ np.linalg.inv(Sk)
            m = m + Kg @ (yv[sel] - H @ m)
            P = P - Kg @ H @ P
        mf.append(m)
        Pf.append(P)
    ms, Ps = [None] * nt, [None] * nt
    ms[-1], Ps[-1] = mf[-1], Pf[-1]
    for k in range(nt - 2, -1, -1):
        Ck = Pf[k] @ Atr.T @ np.linalg.inv(Pp[k + 1])
        ms[k] = mf[k] + Ck @ (ms[k + 1] - mp[k + 1])
        Ps[k] = Pf[k] + Ck @ (Ps[k + 1] - Pp[k + 1]) @ Ck.T
    return np.concatenate(ms), np.concatenate([np.diag(P) for P in Ps])


@pytest.mark.parametrize("prior", [W.prior_st1d(9, 8, 0.7, 0.02), W.prior_st2d(5, 6, 0.3, 0.1, 0.02, 4.0)],
                         ids=lambda p: p["kind"])
def test_space_time_posterior_matches_kalman_smoother(prior):
    nx, ny, nt = prior["n"]
    r = np.random.default_rng(3)
    m = 12
    k_idx = r.integers(0, nt, size=m)
    tk = prior["lo"][2] + (prior["hi"][2] - prior["lo"][2]) * k_idx / (nt - 1)
    if ny == 1:
        coords = np.stack([r.uniform(0, 1, m), tk], axis=1)
    else:
        coords = np.stack([r.uniform(0, 1, m), r.uniform(0, 1, m), tk], axis=1)
    ob = dict(coords=coords, y=r.normal(size=m), sigma=np.full(m, 0.1))
    post = infer.condition(prior, ob)
    L = linalg.cholesky(post.Qpost)
    mu = infer.posterior_mean(post, L)
    var = infer.marginal_variance(post, L)
    Ns = nx * ny
    A = post.A.toarray()
    Hs = np.stack([A[r_, k_idx[r_] * Ns:(k_idx[r_] + 1) * Ns] for r_ in range(m)])
    ms, vs = _kalman_rts(prior, k_idx, Hs, post.y, post.rinv)
    assert np.allclose(mu, ms, rtol=1e-7, atol=1e-9)
    assert np.allclose(var, vs, rtol=1e-7, atol=1e-14)


def test_collocation_mean_converges_to_manufactured_solution():
    # u* = exp(-t) sin(pi x) solves u_t + c u_x - nu u_xx = f with
    # f = (-1 + nu pi^2) e^-t sin(pi x) + c pi e^-t cos(pi x); condition on
    # the collocated PDE and the initial condition (sigma 1e-6): the
    # posterior mean approaches u* at O(h^2 + dt).
    c, nu = 0.5, 0.05
    errs = []
    for n in (9, 17, 33):
        prior = W.prior_st1d(n, n, c, nu, tau=1.0, kappa0=5.0)
        i, k = observe.colloc_rows(prior)
        x = np.linspace(0, 1, n)[i]
        t = np.linspace(0, 1, n)[k]
        f = (-1 + nu * math.pi ** 2) * np.exp(-t) * np.sin(math.pi * x) + c * math.pi * np.exp(-t) * np.cos(math.pi * x)
        xs = np.linspace(0, 1, n)
        ob = dict(coords=np.zeros((0, 2)), y=np.zeros(0), sigma=np.zeros(0),
                  ic_sigma=1e-6, ic_values=np.sin(math.pi * xs),
                  colloc_sigma=1e-6, colloc_c=c, colloc_f=f, burgers_nu=nu)
        post = infer.condition(prior, ob)
        mu = infer.posterior_mean(post)
        X = np.tile(xs, n)
        T = np.repeat(np.linspace(0, 1, n), n)
        errs.append(np.abs(mu - np.exp(-T) * np.sin(math.pi * X)).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[1] > 1.6 and errs[1] / errs[2] > 1.6


def test_rbmc_estimator_is_exact_in_expectation():
    # E[(sum_{j!=i} Q_ij x_j)^2] = (O S O^T)_ii with O = Q - D, S = Q^-1;
    # then 1/Q_ii + (O S O^T)_ii / Q_ii^2 = S_ii exactly.
    prior = W.prior_matern2d(8, 3.0)
    ob = W.point_obs(prior, 10, 0.1, lambda z: z[:, 0], seed=1)
    post = infer.condition(prior, ob)
    Qd = post.Qpost.toarray()
    d = np.diag(Qd)
    O = Qd - np.diag(d)
    S = np.linalg.inv(Qd)
    expect = 1.0 / d + np.diag(O @ S @ O.T) / d ** 2
    assert np.allclose(expect, np.diag(S), rtol=1e-9)


def test_rbmc_on_perturbation_samples_within_stderr():
    prior = W.prior_st1d(12, 10, 0.5, 0.02)
    ob = W.point_obs(prior, 15, 0.05, lambda z: z[:, 0], seed=4)
    post = infer.condition(prior, ob)
    L = linalg.cholesky(post.Qpost)
    exact = infer.marginal_variance(post, L)
    ns = 400
    xs = infer.perturbation_samples(post, 77, range(ns), L)
    # sample covariance of the perturbations matches Q^-1 (the left root works)
    assert np.allclose(np.mean(xs * xs, axis=0), exact, rtol=0.25)
    d = post.Qpost.diagonal()
    off = (post.Qpost - sp.diags(d)).tocsr()
    terms = np.stack([((off @ x) / d) ** 2 for x in xs])
    est = infer.rbmc_variance(post.Qpost, xs)
    assert np.allclose(est, 1.0 / d + terms.mean(axis=0))
    se = terms.std(axis=0, ddof=1) / math.sqrt(ns)
    ok = np.abs(est - exact) <= 4.0 * se + 1e-15
    assert ok.mean() >= 0.99


def test_philox_streams_statistics():
    z = rng.normals(1234, 0, 3, 200001)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert abs(st.kurtosis(z)) < 0.05
    assert st.kstest(z, "norm").pvalue > 1e-3
    z2 = rng.normals(1234, 1, 3, 1000)
    z3 = rng.normals(1234, 0, 4, 1000)
    z4 = rng.normals(1235, 0, 3, 1000)
    for other in (z2, z3, z4):
        assert abs(np.corrcoef(z[:1000], other)[0, 1]) < 0.15
    # a prefix of a longer draw is the shorter draw (counter-based)
    assert np.array_equal(rng.normals(1234, 0, 3, 11), z[:11])
    v = rng.rademacher(9, 2, 100000)
    assert set(np.unique(v)) == {-1.0, 1.0} and abs(v.mean()) < 0.02


def test_philox_known_answer_vectors():
    # published known-answer vectors (tests/golden/philox4x32_10_kat.txt):
    # a wrong multiplier, round constant, word order or round count fails
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(w, 16) for w in r]
        out = rng.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_philox_is_a_bijection_on_counters():
    j = np.arange(1 << 16, dtype=np.uint64)
    w = rng.philox4x32_10(j, 5, 0, 0, 123, 456)
    packed = (w[0] << np.uint64(32)) | w[1]
    assert len(np.unique(packed)) == len(j)


def _dense_loglik(prior, ob):
    post = infer.condition(prior, ob)
    A = post.A.toarray()
    Cy = A @ np.linalg.inv(post.Q.toarray()) @ A.T + np.diag(1.0 / post.rinv)
    return st.multivariate_normal(mean=np.zeros(len(post.y)), cov=Cy).logpdf(post.y)


@pytest.mark.parametrize("prior", [W.prior_st2d(5, 5, 0.5, 0.0, 0.01, 10.0), W.prior_matern2d(9, 4.0)],
                         ids=lambda p: p["kind"])
def test_loglik_matches_dense_gaussian_and_fd_gradient(prior):
    ob = W.point_obs(prior, 25, 0.1, lambda z: np.cos(2 * z[:, 0]) + z[:, 1], seed=8)
    assert infer.log_marginal_likelihood(prior, ob) == pytest.approx(_dense_loglik(prior, ob), rel=1e-9)
    g = infer.log_marginal_likelihood_grad(prior, ob)
    th = infer.hyper_of(prior, ob)
    for name in infer.HYPER:
        if prior["kind"] == "matern2d" and name in ("c", "nu"):
            continue
        h = 1e-4
        tp, tm = dict(th), dict(th)
        tp[name] += h
        tm[name] -= h
        fp = infer.log_marginal_likelihood(*infer.with_hyper(prior, ob, tp))
        fm = infer.log_marginal_likelihood(*infer.with_hyper(prior, ob, tm))
        fd = (fp - fm) / (2 * h)
        assert g[name] == pytest.approx(fd, rel=1e-5, abs=1e-6 * max(1.0, abs(fd))), name


def test_logdet_prior_tau_derivative_closed_form():
    # the space-time prior scales as tau^-2 off the boundary, so
    # 1/2 tr(Q^-1 dQ/dlog tau) = -(number of non-boundary DOFs)
    prior = W.prior_st2d(5, 4, 0.5, 0.0, 0.01, 6.0)
    Q = fem.prior_precision(prior).toarray()
    dQ = infer.dQ_dtheta(prior, "log_tau").toarray()
    nint = int((~fem.boundary_mask(prior)).sum())
    assert 0.5 * np.trace(np.linalg.solve(Q, dQ)) == pytest.approx(-nint, rel=1e-8)


def test_hutchinson_gradient_unbiased_within_stderr():
    prior = W.prior_st2d(5, 5, 0.5, 0.0, 0.01, 10.0)
    ob = W.point_obs(prior, 25, 0.1, lambda z: np.cos(2 * z[:, 0]) + z[:, 1], seed=8)
    exact = infer.log_marginal_likelihood_grad(prior, ob)
    est, se = infer.hutchinson_grad(prior, ob, seed=99, nprobe=64)
    for name in infer.HYPER:
        assert abs(est[name] - exact[name]) <= 4.0 * se[name] + 1e-9, name


def test_hutchinson_estimator_over_all_sign_vectors_is_exact():
    # sum over all 2^N Rademacher vectors of v v^T is 2^N I exactly, so the
    # estimator averaged over the full enumeration equals the exact gradient:
    # a dropped term, a wrong sign or a transposed solve fails here
    prior = W.prior_st1d(4, 3, 0.5, 0.05)
    ob = W.point_obs(prior, 5, 0.2, lambda z: np.sin(3 * z[:, 0]) + z[:, 1], seed=4)
    N = W.n_nodes(prior)
    assert N == 12
    k = np.arange(2 ** N)[:, None]
    V = 1.0 - 2.0 * ((k >> np.arange(N)[None, :]) & 1)
    exact = infer.log_marginal_likelihood_grad(prior, ob)
    for mode in ("hutchinson", "exact"):      # both traces estimated / the prior one exact
        est, _ = infer.hutchinson_grad_probes(prior, ob, V, prior_trace=mode)
        for name in infer.HYPER:
            assert abs(est[name] - exact[name]) <= 1e-9 * max(1.0, abs(exact[name])), (mode, name, est[name], exact[name])


def test_burgers_jacobian_matches_finite_differences():
    prior = W.prior_st1d(9, 6, 1.0, 0.01, x0=-1.0, x1=1.0)
    u = np.random.default_rng(2).normal(size=9 * 6)
    J = observe.burgers_jacobian(prior, u, 0.05).toarray()
    h = 1e-6
    Jfd = np.empty_like(J)
    for j in range(len(u)):
        e = np.zeros_like(u)
        e[j] = h
        Jfd[:, j] = (observe.burgers_residual(prior, u + e, 0.05) - observe.burgers_residual(prior, u - e, 0.05)) / (2 * h)
    assert np.allclose(J, Jfd, rtol=1e-6, atol=1e-4)


def _objective_complex(prior, ob, Q, A, u):
    """-log pi(u) written with complex-safe arithmetic for complex-step
    directional derivatives (independent of the Jacobian)."""
    n = prior["n"][0]
    xs = np.linspace(prior["lo"][0], prior["hi"][0], n)
    v = 0.5 * (u @ (Q @ u))
    r = ob["y"] - A @ u
    v += 0.5 * np.sum(r * r / ob["sigma"] ** 2)
    r = -np.sin(np.pi * xs) - u[:n]
    v += 0.5 * np.sum(r * r) / ob["ic_sigma"] ** 2
    f = observe.burgers_residual(prior, u, ob["burgers_nu"])
    return v + 0.5 * np.sum(f * f) / ob["colloc_sigma"] ** 2


@pytest.mark.slow
def test_gauss_newton_reaches_a_stationary_point_near_the_cole_hopf_truth():
    n = 33
    prior, ob = W.c3_burgers(nx=n, nt=n, m=40, seed=3, nu=0.05)
    Q = fem.prior_precision(prior)
    A = observe.point_matrix(prior, ob["coords"])
    u0 = infer.posterior_mean(infer.condition(prior, ob))
    u = u0
    vals = [infer.neg_log_post(None, Q, ob, prior, u)]
    for _ in range(6):
        u, d, alpha, dec = infer.gauss_newton_step(prior, ob, u)
        vals.append(infer.neg_log_post(None, Q, ob, prior, u))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(vals, vals[1:]))
    assert vals[-1] < 1e-10 * vals[0]
    # stationarity of the true nonlinear objective: complex-step directional
    # derivatives along random directions drop by > 1e9 from the start
    r = np.random.default_rng(0)
    for _ in range(3):
        e = r.normal(size=u.size)
        e /= np.linalg.norm(e)
        s1 = np.imag(_objective_complex(prior, ob, Q, A, u + 1e-30j * e)) / 1e-30
        s0 = np.imag(_objective_complex(prior, ob, Q, A, u0 + 1e-30j * e)) / 1e-30
        assert abs(s1) < 1e-9 * abs(s0)
    xs = np.linspace(-1, 1, n)
    T = np.repeat(np.linspace(0, 1, n), n)
    X = np.tile(xs, n)
    truth = W.cole_hopf_burgers(X, T, 0.05)
    assert np.abs(u - truth).max() < 0.05


def test_collocation_stride_is_conditioning_on_the_active_rows_only():
    # zero-weight rows observe nothing: the posterior equals conditioning on
    # the active rows alone (rows x % sx == 0, k % st == 0)
    import scipy.sparse as sp
    pr, ob = W.c3_burgers(nx=17, nt=9, m=10)
    u = np.random.default_rng(4).normal(size=17 * 9) * 0.1
    obs = dict(ob, colloc_stride=(3, 2))
    post = infer.condition(pr, obs, linearise_at=u)
    act = observe.colloc_active(pr, obs)
    i, k = observe.colloc_rows(pr)
    assert np.array_equal(act, (i % 3 == 0) & (k % 2 == 0)) and act.sum() == 5 * 4
    J, F = observe.pde_rows(pr, obs, u, obs["burgers_nu"])
    Ja = J[np.flatnonzero(act)]
    full = infer.condition(pr, dict(ob, colloc_sigma=None))
    Qa = full.Qpost + (Ja.T @ Ja) / obs["colloc_sigma"] ** 2
    ba = full.b + Ja.T @ ((Ja @ u - F[act]) / obs["colloc_sigma"] ** 2)
    assert abs(post.Qpost - Qa).max() <= 1e-9 * abs(Qa).max()
    assert np.max(np.abs(post.b - ba)) <= 1e-9 * np.max(np.abs(ba))


def test_single_interior_node_reduces_to_scalar_conditioning():
    # 3 x 3 Matern grid (Sec. 2.2, App. B): the eight boundary nodes are
    # Dirichlet rows with precision 1/eps2 and no coupling, the centre row of
    # B is kappa^2 h^2 + 4 (lumped mass h^2, the 5-point stiffness diagonal 4),
    # so Q_cc = tau^2 (kappa^2 h^2 + 4)^2 / h^2.  One observation at the centre
    # (barycentric weight 1) makes the posterior a scalar Gaussian update.
    kappa, tau, eps2, y, sigma = 4.0, 0.3, 1e-8, 0.7, 0.1
    pr = dict(W.c2_matern(n=3, m=1, seed=1, kappa=kappa)[0], tau=tau, eps2=eps2)
    ob = {"coords": np.array([[0.5, 0.5]]), "y": np.array([y]), "sigma": np.array([sigma])}
    post = infer.condition(pr, ob)
    h = 0.5
    q_c = tau ** 2 * (kappa ** 2 * h ** 2 + 4.0) ** 2 / h ** 2
    Q = post.Q.toarray()
    want = np.diag(np.full(9, 1.0 / eps2))
    want[4, 4] = q_c
    assert np.allclose(Q, want, rtol=1e-13, atol=0.0)
    prec = q_c + 1.0 / sigma ** 2
    mu = infer.posterior_mean(post)
    var = infer.marginal_variance(post)
    assert mu[4] == pytest.approx((y / sigma ** 2) / prec, rel=1e-13)
    assert np.all(np.delete(mu, 4) == 0.0)
    assert var[4] == pytest.approx(1.0 / prec, rel=1e-12)
    assert np.allclose(np.delete(var, 4), eps2, rtol=1e-12)
