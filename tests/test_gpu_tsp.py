"""The time-stepping preconditioner of the 1D space-time solves, applied on
its own (gmrf_stencil_step mode 5), against the dense matrix it stands for.

With collocation rows (Sec. 3.1, 3.3) or Matern transition noise (App. A)
the solver preconditions with z = M r = Jt^-1 W^-1 Jt^-T r, where Jt is
square, one row per node, block lower-bidiagonal in time:

* boundary nodes: the prior's Dirichlet rows (identity, weight 1 / eps^2);
* level 0: the initial-condition rows (identity, weight 1 / ic_sigma^2) when
  the initial condition is observed, else the prior's initial-level rows
  (weight 1);
* levels k >= 1: the PDE rows (collocation or FEM Crank-Nicolson, the
  oracle's Jacobian at the linearisation point; weight 1 / colloc_sigma^2)
  where the PDE is observed, the white-noise prior root's rows elsewhere
  (weight 1; with Matern transition noise the weight of a level's prior rows
  is T_P^2, T_P the level's T_K restricted to those rows).

Jt and W are assembled here from the oracle's prior root, noise transform
and PDE Jacobian, and M r is formed by dense solves in FP64.  The kernel's
partition solve reorders the eliminations, so the result agrees to 64 unit
roundoffs times the condition numbers of Jt and T_P (relative to the largest
entry).
Cases: every row kind, strided collocation points (mixed PDE and prior rows
on one level), no observed initial condition, noise with and without
(Burgers) collocation, and a level wider than the kernel's 128 lanes
(several rows per lane).
"""
import numpy as np
import pytest

from oracle import fem, infer, observe
from paper_2503_08343_gb300 import gmrf
from paper_2503_08343_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2503_08343_gb300 import build
    build.build()
    return gmrf.load()


def _linear(nx, nt, stride=None, form="collocation", ic=True, noise=0.0, colloc=True):
    pr, ob = W.c1_st1d(nx=nx, nt=nt, m=30, seed=5)
    if noise:
        pr = dict(pr, noise_kappa=noise, decay=0.1)
    if colloc:
        ob = dict(ob, colloc_sigma=1e-3, colloc_c=0.5, burgers_nu=0.01, colloc_form=form)
    if ic:
        ob = dict(ob, ic_sigma=1e-3, ic_values=np.zeros(nx))
    if stride:
        ob = dict(ob, colloc_stride=stride)
    return pr, ob


def _burgers(nx, nt, stride=None, noise=0.0, form="collocation"):
    pr, ob = W.c3_burgers(nx=nx, nt=nt, m=60, seed=3, nu=0.05)
    if noise:
        pr = dict(pr, noise_kappa=noise)
    if stride:
        ob = dict(ob, colloc_stride=stride)
    if form != "collocation":
        ob = dict(ob, colloc_form=form, colloc_sigma=1e-4)
    return pr, ob


CASES = {
    "linear_colloc_33x17": lambda: (_linear(33, 17), False),
    "linear_colloc_strided_33x17": lambda: (_linear(33, 17, stride=(3, 2)), False),
    "linear_colloc_no_ic_33x17": lambda: (_linear(33, 17, ic=False), False),
    "linear_fem_cn_33x17": lambda: (_linear(33, 17, form="fem_cn"), False),
    "linear_fem_cn_strided_33x17": lambda: (_linear(33, 17, form="fem_cn", stride=(2, 3)), False),
    "noise_data_only_33x17": lambda: (_linear(33, 17, noise=8.0, colloc=False), False),
    "noise_no_ic_33x17": lambda: (_linear(33, 17, noise=8.0, colloc=False, ic=False), False),
    "linear_colloc_wide_300x6": lambda: (_linear(300, 6, stride=(3, 2)), False),
    "noise_wide_300x6": lambda: (_linear(300, 6, noise=8.0, colloc=False), False),
    "burgers_65x33": lambda: (_burgers(65, 33), True),
    "burgers_strided_65x33": lambda: (_burgers(65, 33, stride=(4, 4)), True),
    "burgers_noise_strided_65x33": lambda: (_burgers(65, 33, stride=(8, 8), noise=15.0), True),
    "burgers_fem_cn_strided_65x33": lambda: (_burgers(65, 33, stride=(4, 2), form="fem_cn"), True),
}


def _dense_tsp(pr, ob, u):
    """(Jt, Wr, largest condition number of a T_P) of the preconditioner,
    W = Wr Wr, dense, from the oracle's pieces."""
    nx, _, nt = pr["n"]
    N = nx * nt
    Bw = fem.prior_root(dict(pr, noise_kappa=0.0)).toarray()
    TK = fem.noise_transform(pr).toarray()
    noise = pr.get("noise_kappa", 0.0) > 0.0
    bnd = np.zeros(N, bool)
    bnd[0::nx] = True
    bnd[nx - 1::nx] = True
    has_ic = ob.get("ic_sigma") is not None
    pde = {}
    qeps = 0.0
    if ob.get("colloc_sigma") is not None:
        J, _ = observe.pde_rows(pr, ob, u, ob.get("burgers_nu", pr["nu"]), advect=ob.get("colloc_c"))
        J = J.toarray()
        ci, ck = observe.colloc_rows(pr)
        act = observe.colloc_active(pr, ob)
        pde = {ck[j] * nx + ci[j]: J[j] for j in range(len(ci)) if act[j]}
        qeps = 1.0 / ob["colloc_sigma"] ** 2
    Jt = np.zeros((N, N))
    Wm = np.zeros((N, N))
    prior_rows = [[] for _ in range(nt)]
    for r in range(N):
        k, x = divmod(r, nx)
        if bnd[r]:
            Jt[r, r] = 1.0
            Wm[r, r] = 1.0 / pr["eps2"]
        elif k == 0 and has_ic:
            Jt[r, r] = 1.0
            Wm[r, r] = 1.0 / ob["ic_sigma"] ** 2
        elif r in pde:
            Jt[r] = pde[r]
            Wm[r, r] = qeps
        else:
            row = Bw[r].copy()
            row[bnd] = 0.0
            Jt[r] = row
            Wm[r, r] = 1.0
            if k >= 1:
                prior_rows[k].append(x)
    # W = Wr Wr with Wr block diagonal (T_P on a level's prior rows under
    # Matern transition noise), so that W^-1 is two solves with Wr and the
    # reference does not square the conditioning of T_P
    Wr = np.diag(np.sqrt(np.diag(Wm)))
    cond_t = 1.0
    if noise:
        for k in range(1, nt):
            P = np.array(prior_rows[k], dtype=int)
            if len(P) == 0:
                continue
            idx = k * nx + P
            Wr[np.ix_(idx, idx)] = TK[np.ix_(P, P)]
            cond_t = max(cond_t, np.linalg.cond(TK[np.ix_(P, P)]))
    return Jt, Wr, cond_t


def _linearisation_point(post, pr, ob):
    """Linearises the GPU posterior's Burgers rows (a Gauss-Newton step leaves
    them linearised at the point it returns) and returns that point."""
    u = infer.posterior_mean(infer.condition(pr, ob))
    d = np.zeros_like(u)
    try:
        post.gauss_newton_step(u, d, opts=gmrf.default_opts(max_refine=2, max_inner=20))
    except gmrf.GmrfError:
        pass            # a step that stops at its caps still linearises at the returned point
    assert np.all(np.isfinite(u))
    return u


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [1, 0])
def test_preconditioner_is_the_dense_time_stepping_solve(name, precision):
    (pr, ob), nonlinear = CASES[name]()
    post = gmrf.Posterior(gmrf.Prior(pr), ob)
    N = post.N
    u = _linearisation_point(post, pr, ob) if nonlinear else np.zeros(N)
    Jt, Wr, cond_t = _dense_tsp(pr, ob, u)
    r = np.random.default_rng(11).normal(size=(3, N))
    if precision == 0:
        r = r.astype(np.float32).astype(np.float64)
    z, _, dots = post.stencil_step(5, b=r, precision=precision)
    want = np.linalg.solve(Jt, np.linalg.solve(Wr, np.linalg.solve(Wr, np.linalg.solve(Jt.T, r.T)))).T
    # forward error of the two sweeps and the two solves with T_P: a few dozen
    # roundings times the condition number of each (diagonal weights scale
    # without amplifying errors)
    tol = 64 * (2.0 ** -53 if precision == 1 else 2.0 ** -24) * (np.linalg.cond(Jt) + 2 * cond_t)
    for i in range(r.shape[0]):
        err = np.max(np.abs(z[i] - want[i])) / np.max(np.abs(want[i]))
        assert err <= tol, (i, err)
        assert dots[i] == pytest.approx(float(r[i] @ want[i]), rel=10 * tol)
