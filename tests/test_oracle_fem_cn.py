"""Pins of the oracle's FEM (Galerkin-tested) Crank-Nicolson PDE rows.

The oracle integrates the rows by Gauss-Legendre quadrature element by
element.  Independently, the integrals have closed forms on the uniform P1
mesh (hat phi_i on [x_(i-1), x_(i+1)], width h), worked out by hand:

  int phi_i phi_j         = h/6 [1 4 1]          (consistent mass)
  int phi_i' phi_j'       = 1/h [-1 2 -1]
  int phi_i c phi_j'      = c/2 [-1 0 1]
  int phi_i v v_x         = (v_(i+1) - v_(i-1)) (v_(i+1) + v_i + v_(i-1)) / 6
                            (v piecewise linear; per element the integrand is
                            phi_i times a linear function times a constant)

so F_ik = (h/6dt)[1 4 1](u^k - u^(k-1)) + 1/2 sum over the two levels of
(convection + nu [-1 2 -1]/h).  Pins: the rows equal that closed form; the
Jacobian equals central differences of the residual; for a smooth exact
solution of u_t + c u_x = nu u_xx the rows divided by h vanish at second order
in (h, dt) (Crank-Nicolson in time, P1 Galerkin in space).
"""
import math

import numpy as np
import pytest

from oracle import fem, observe
from paper_2503_08343_gb300 import workloads as W


def _closed_form(pr, u, nu, advect):
    nx, _, nt = pr["n"]
    h, _, dt = fem.grid_spacing(pr)
    U = u.reshape(nt, nx)
    i, k = observe.colloc_rows(pr)

    def conv(v, ii):
        if advect is None:
            return (v[ii + 1] - v[ii - 1]) * (v[ii + 1] + v[ii] + v[ii - 1]) / 6.0
        return advect * (v[ii + 1] - v[ii - 1]) / 2.0

    out = np.empty(len(i))
    for r, (ii, kk) in enumerate(zip(i, k)):
        dU = U[kk] - U[kk - 1]
        mass = h / (6.0 * dt) * (dU[ii - 1] + 4.0 * dU[ii] + dU[ii + 1])
        sp_ = sum(conv(U[lev], ii) + nu * (2.0 * U[lev, ii] - U[lev, ii - 1] - U[lev, ii + 1]) / h
                  for lev in (kk, kk - 1))
        out[r] = mass + 0.5 * sp_
    return out


@pytest.mark.parametrize("advect", [None, 0.7])
def test_rows_equal_the_closed_form_integrals(advect):
    pr = W.prior_st1d(11, 7, 0.5, 0.05, x0=-1.0, x1=1.0, t1=0.6)
    u = np.random.default_rng(2).normal(size=11 * 7)
    got = observe.fem_cn_residual(pr, u, 0.03, advect)
    want = _closed_form(pr, u, 0.03, advect)
    assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("advect", [None, 0.7])
def test_jacobian_equals_central_differences(advect):
    pr = W.prior_st1d(9, 6, 0.5, 0.05)
    u = np.random.default_rng(3).normal(size=9 * 6)
    J = observe.fem_cn_jacobian(pr, u, 0.04, advect).toarray()
    eps = 1e-6
    fd = np.empty_like(J)
    for j in range(u.size):
        e = np.zeros_like(u)
        e[j] = eps
        fd[:, j] = (observe.fem_cn_residual(pr, u + e, 0.04, advect) - observe.fem_cn_residual(pr, u - e, 0.04, advect)) / (2 * eps)
    assert np.max(np.abs(J - fd)) <= 1e-7 * max(1.0, np.max(np.abs(J)))
    # each row couples six unknowns: x-1, x, x+1 on its level and on the level before
    assert np.all((np.abs(J) > 0).sum(axis=1) == 6)


def test_rows_vanish_at_second_order_on_a_smooth_solution():
    c, nu, kw = 0.8, 0.05, 2.0 * math.pi

    def exact(x, t):
        return np.exp(-nu * kw * kw * t) * np.sin(kw * (x - c * t))

    errs = []
    for nx, nt in ((33, 17), (65, 33), (129, 65)):
        pr = W.prior_st1d(nx, nt, c, nu, x0=0.0, x1=1.0, t1=0.5)
        h, _, _ = fem.grid_spacing(pr)
        xs = fem.axis_nodes(0.0, 1.0, nx)
        ts = np.linspace(0.0, 0.5, nt)
        u = exact(xs[None, :], ts[:, None]).ravel()
        errs.append(float(np.max(np.abs(observe.fem_cn_residual(pr, u, nu, c))) / h))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs
