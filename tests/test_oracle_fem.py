"""Pins for the oracle's prior assembly (no GPU).

Each test ties oracle.fem to something other than itself: hand-derived P1
stencils, the block formula of App. A built through dense inverses of the
state-space model, symmetry / positive definiteness, and the sine-series
closed form of the Dirichlet Matern variance.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, linalg
from paper_2503_08343_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def _row(X, i):
    r = X.getrow(i).tocoo()
    return dict(zip(r.col.tolist(), r.data.tolist()))


def test_p1_1d_stencils():
    # hand derivation: S = (1/h)[-1 2 -1], lumped mass h, advection c[-1/2 0 1/2]
    n, c = 7, 0.8
    x = np.linspace(0.0, 1.5, n)
    h = x[1] - x[0]
    S, ml, Badv = fem.p1_1d(x, c)
    r = _row(S, 3)
    assert r[2] == pytest.approx(-1 / h) and r[3] == pytest.approx(2 / h) and r[4] == pytest.approx(-1 / h)
    assert ml[3] == pytest.approx(h) and ml[0] == pytest.approx(h / 2)
    ra = _row(Badv, 3)
    assert ra[2] == pytest.approx(-c / 2) and ra[4] == pytest.approx(c / 2) and abs(ra.get(3, 0.0)) < 1e-15


def test_p1_2d_stencils_on_5x5():
    # On the mesh split along (i,j)->(i+1,j+1) the P1 Laplacian is the
    # 5-point stencil (hypotenuse couplings cancel), lumped mass h^2, and the
    # x-advection row is (h/6)[+x: 2, -x: -2, (+1,+1): 1, (-1,-1): -1,
    # (0,+1): -1, (0,-1): 1] (derived by hand from the six triangles).
    n = 5
    xs = np.linspace(0, 1, n)
    h = xs[1] - xs[0]
    S, ml, Bx = fem.p1_2d(xs, xs, 1.0, 0.0)
    i0 = 2 * n + 2
    r = {k: v for k, v in _row(S, i0).items() if abs(v) > 1e-14}
    assert r == pytest.approx({i0: 4.0, i0 - 1: -1.0, i0 + 1: -1.0, i0 - n: -1.0, i0 + n: -1.0})
    assert ml[i0] == pytest.approx(h * h)
    assert ml.sum() == pytest.approx(1.0)
    rb = {k: v for k, v in _row(Bx, i0).items() if abs(v) > 1e-14}
    want = {i0 + 1: 2, i0 - 1: -2, i0 + n + 1: 1, i0 - n - 1: -1, i0 + n: -1, i0 - n: 1}
    assert rb == pytest.approx({k: v * h / 6 for k, v in want.items()})
    # y-advection is the mirror image
    _, _, By = fem.p1_2d(xs, xs, 0.0, 1.0)
    rby = {k: v for k, v in _row(By, i0).items() if abs(v) > 1e-14}
    wanty = {i0 + n: 2, i0 - n: -2, i0 + n + 1: 1, i0 - n - 1: -1, i0 + 1: -1, i0 - 1: 1}
    assert rby == pytest.approx({k: v * h / 6 for k, v in wanty.items()})


def test_p1_2d_reproduces_linear_functions():
    # int phi_i d/dx (x) = int phi_i = ml_i  and  S applied to a linear
    # function vanishes at interior nodes
    n = 6
    xs = np.linspace(0, 2, n)
    ys = np.linspace(-1, 1, n)
    S, ml, Bx = fem.p1_2d(xs, ys, 1.0, 0.0)
    X = np.tile(xs, n)
    Y = np.repeat(ys, n)
    assert np.allclose(Bx @ X, ml)
    interior = ~fem.spatial_boundary(dict(n=(n, n, 1)))
    assert np.allclose((S @ (3 * X - 2 * Y + 1))[interior], 0.0, atol=1e-12)


PRIORS = [
    W.prior_matern2d(6, 3.0),
    W.prior_steady_advdiff2d(6, 4.0, nu=0.05, c=1.5),
    W.prior_st1d(7, 5, c=0.5, nu=0.01),
    W.prior_st2d(5, 4, cx=0.5, cy=0.2, nu=0.02, kappa=5.0),
]


@pytest.mark.parametrize("prior", PRIORS, ids=lambda p: p["kind"])
def test_Q_symmetric_positive_definite(prior):
    Q = fem.prior_precision(prior)
    D = Q.toarray()
    assert np.max(np.abs(D - D.T)) <= 1e-13 * np.max(np.abs(D))
    assert np.linalg.eigvalsh(D).min() > 0.0
    linalg.cholesky(Q)    # succeeds


@pytest.mark.parametrize("prior", [PRIORS[2], PRIORS[3]], ids=lambda p: p["kind"])
def test_space_time_matches_appendix_A_blocks(prior):
    # App. A: u^1 ~ N(0, Q1^-1), u^(i+1) | u^i ~ N(A u^i, F) gives the block
    # tridiagonal Q_ST with diagonal Q1 + A^T F^-1 A, ..., F^-1 + A^T F^-1 A,
    # F^-1 and off-diagonals -A^T F^-1 (reading: Q1 is a precision).  Build
    # A = G^-1 Mlc and F = G^-1 Sw G^-T by dense inversion and compare.
    S, ml, Badv, dim = fem.spatial_mesh(prior)
    sb = fem.spatial_boundary(prior)
    nt = prior["n"][2]
    dt = (prior["hi"][2] - prior["lo"][2]) / (nt - 1)
    tau, eps2 = prior["tau"], prior["eps2"]
    K0 = fem.constrain(prior["kappa0"] ** 2 * sp.diags(ml) + S, sb).toarray()
    G = fem.constrain(sp.diags(ml) + dt * (prior["nu"] * S + Badv), sb).toarray()
    Mc = np.diag(np.where(sb, 0.0, ml))
    tau0 = fem.matern_tau_unit(prior["kappa0"], dim)
    Minv0 = np.diag(np.where(sb, 1.0 / eps2, (tau0 / tau) ** 2 / ml))
    Q1 = K0.T @ Minv0 @ K0
    # on the boundary K0 and G are the identity, so the variance is eps2
    Sw = np.diag(np.where(sb, eps2, tau * tau * dt * ml))
    Gi = np.linalg.inv(G)
    A = Gi @ Mc
    F = Gi @ Sw @ Gi.T
    Fi = np.linalg.inv(F)
    Ns = len(ml)
    Qst = np.zeros((Ns * nt, Ns * nt))
    blk = lambda k, l: (slice(k * Ns, (k + 1) * Ns), slice(l * Ns, (l + 1) * Ns))
    for k in range(nt):
        D = Q1.copy() if k == 0 else Fi.copy()
        if k < nt - 1:
            D += A.T @ Fi @ A
            Qst[blk(k, k + 1)] = -A.T @ Fi
            Qst[blk(k + 1, k)] = -Fi @ A
        Qst[blk(k, k)] = D
    Q = fem.prior_precision(prior).toarray()
    assert np.allclose(Q, Qst, rtol=1e-9, atol=1e-9 * np.abs(Q).max())


def _dirichlet_matern_var(n, kappa, tau, a, b):
    """Sine-series variance of the interior block Q_int = tau^2/h^2 K_int^2,
    K_int = kappa^2 h^2 I + L5 with the eigenpairs of the Dirichlet 5-point
    Laplacian: v_jk(a,b) = (2/(n-1)) sin(j pi a/(n-1)) sin(k pi b/(n-1)),
    lambda_jk = 4 sin^2(j pi / (2(n-1))) + 4 sin^2(k pi / (2(n-1)))."""
    h = 1.0 / (n - 1)
    j = np.arange(1, n - 1)
    sa = np.sin(j * np.pi * a / (n - 1))
    sb_ = np.sin(j * np.pi * b / (n - 1))
    lam1 = 4.0 * np.sin(j * np.pi / (2 * (n - 1))) ** 2
    lam = kappa * kappa * h * h + lam1[:, None] + lam1[None, :]
    v2 = (2.0 / (n - 1)) ** 2 * (sa[:, None] * sb_[None, :]) ** 2
    return (h * h / (tau * tau)) * np.sum(v2 / lam ** 2)


def test_takahashi_matches_dirichlet_sine_series():
    n, kappa = 14, 6.0
    prior = W.prior_matern2d(n, kappa)
    L = linalg.cholesky(fem.prior_precision(prior))
    var = linalg.takahashi_diag(L)
    for (a, b) in [(1, 1), (3, 7), (6, 6), (12, 5)]:
        want = _dirichlet_matern_var(n, kappa, prior["tau"], a, b)
        assert var[b * n + a] == pytest.approx(want, rel=1e-10)
    # boundary DOFs have variance eps2 (App. B)
    assert var[0] == pytest.approx(prior["eps2"], rel=1e-9)


def test_matern_variance_tends_to_one_in_the_interior():
    # Away from the boundary the lumped-P1 Matern approaches the continuum
    # unit variance 1/(4 pi kappa^2 tau^2) = 1.  Measured at n = 129, kappa =
    # 20 (kappa h ~ 0.16): within 3 %.
    n, kappa = 129, 20.0
    c = (n - 1) // 2
    v = _dirichlet_matern_var(n, kappa, 1.0 / math.sqrt(4 * math.pi * kappa ** 2), c, c)
    assert abs(v - 1.0) < 0.03


def _t0_block(prior):
    """The t = 0 block of the space-time root and its precision B0^T B0."""
    nx, ny, _ = prior["n"]
    Ns = nx * ny
    B0 = fem.prior_root(prior).tocsr()[:Ns, :Ns]
    return (B0.T @ B0).tocsr()


def test_initial_block_unit_variance_1d():
    # tau0 of the space-time initial block (App. A Q1; unit-variance Matern
    # alpha = 2 with kappa0, Lindgren et al. 2011: sigma^2 = 1/(4 kappa^3 tau^2)
    # in 1D).  Wide grid: kappa0 h = 0.05 on [0, 4], centre 2 = 5.8 ranges
    # (range sqrt(12)/kappa0) from the boundary.  The discrete variance there
    # is given independently by the sine series of the Dirichlet
    # tridiagonal Laplacian: Q1_int = (tau0^2/h) K^2, K = kappa0^2 h I + T/h,
    # T = tridiag(-1, 2, -1) with eigenvalues 4 sin^2(pi k / (2(n-1))) and
    # normalised eigenvectors sqrt(2/(n-1)) sin(pi k j / (n-1)).  Measured:
    # 1.00031 (discretisation error 3e-4); a kappa^3 <-> kappa^2 slip or a
    # wrong constant moves it by a factor of kappa0 or more.
    nx, k0 = 801, 10.0
    prior = W.prior_st1d(nx, 2, 0.5, 0.01, kappa0=k0, x0=0.0, x1=4.0)
    var = linalg.takahashi_diag(linalg.cholesky(_t0_block(prior)))
    c = (nx - 1) // 2
    h = 4.0 / (nx - 1)
    k = np.arange(1, nx - 1)
    mu = k0 * k0 * h + 4.0 * np.sin(np.pi * k / (2 * (nx - 1))) ** 2 / h
    series_tau1 = h * np.sum((2.0 / (nx - 1)) * np.sin(np.pi * k * c / (nx - 1)) ** 2 / mu ** 2)
    tau0 = fem.matern_tau_unit(k0, 1)
    assert var[c] == pytest.approx(series_tau1 / tau0 ** 2, rel=1e-9)
    assert abs(var[c] - 1.0) < 1e-3


def test_initial_block_unit_variance_2d():
    # as above in 2D (sigma^2 = 1/(4 pi kappa^2 tau^2)): kappa0 h = 0.05 on
    # [0, 1.7]^2, centre 3 ranges (sqrt(8)/kappa0) from the boundary; the
    # centre variance of the assembled t = 0 block by one sparse solve
    # e_c^T Q1^-1 e_c, against the Dirichlet 5-point sine series and against
    # the continuum value 1.  Measured: 1.0023.
    n, k0, side = 341, 10.0, 1.7
    prior = W.prior_st2d(n, 2, 0.5, 0.0, 0.01, k0)
    prior["hi"] = (side, side, 1.0)
    Q1 = _t0_block(prior).tocsc()
    c = (n - 1) // 2
    e = np.zeros(n * n)
    e[c * n + c] = 1.0
    import scipy.sparse.linalg as spl
    v = spl.spsolve(Q1, e)[c * n + c]
    h = side / (n - 1)
    j = np.arange(1, n - 1)
    lam1 = 4.0 * np.sin(j * np.pi / (2 * (n - 1))) ** 2
    lam = k0 * k0 * h * h + lam1[:, None] + lam1[None, :]
    sj = np.sin(j * np.pi * c / (n - 1))
    v2 = (2.0 / (n - 1)) ** 2 * (sj[:, None] * sj[None, :]) ** 2
    series_tau1 = h * h * np.sum(v2 / lam ** 2)
    tau0 = fem.matern_tau_unit(k0, 2)
    assert v == pytest.approx(series_tau1 / tau0 ** 2, rel=1e-8)
    assert abs(v - 1.0) < 5e-3


@pytest.mark.parametrize("prior", [W.prior_st2d(6, 5, 0.5, 0.2, 0.03, 7.0), W.prior_st1d(9, 6, 0.5, 0.05),
                                   W.prior_matern2d(8, 5.0), W.prior_steady_advdiff2d(8, 5.0, 0.05, 1.2)],
                         ids=lambda p: p["kind"])
def test_root_derivative_matches_central_differences(prior):
    # the exact dB/dtheta against central differences of the assembled root
    # (h = 1e-5: truncation O(h^2) and rounding ~1e-16/h, far below 1e-8)
    from oracle import infer
    th = infer.hyper_of(prior, {"sigma": [1.0]})
    for name in ("log_kappa", "log_tau", "c", "nu"):
        h = 1e-5
        tp, tm = dict(th), dict(th)
        tp[name] += h
        tm[name] -= h
        dummy = {"y": [0.0], "sigma": [1.0]}
        Bp = fem.prior_root(infer.with_hyper(prior, dummy, tp)[0])
        Bm = fem.prior_root(infer.with_hyper(prior, dummy, tm)[0])
        fd = ((Bp - Bm) / (2 * h)).toarray()
        ex = fem.prior_root_derivative(prior, name).toarray()
        if prior["kind"] == "matern2d" and name in ("c", "nu"):
            assert not ex.any() and not fd.any()
            continue
        assert np.abs(fd - ex).max() <= 1e-8 * np.abs(ex).max(), name


def test_takahashi_matches_dense_inverse_on_random_band():
    rng = np.random.default_rng(0)
    N, bw = 40, 5
    R = np.zeros((N, N))
    for d in range(bw + 1):
        v = rng.normal(size=N - d)
        R += np.diag(v, -d)
    Qd = R @ R.T + N * np.eye(N)
    L = linalg.cholesky(sp.csr_matrix(Qd))
    assert np.allclose(linalg.takahashi_diag(L), np.diag(np.linalg.inv(Qd)), rtol=1e-12)
    b = rng.normal(size=N)
    assert np.allclose(linalg.solve(L, b), np.linalg.solve(Qd, b), rtol=1e-12)
    assert linalg.logdet(L) == pytest.approx(np.linalg.slogdet(Qd)[1], rel=1e-12)
