"""Observation operators (Sec. 3.1): point data rows A_ij = phi_j(x_i),
collocation rows of linear advection-diffusion, initial-condition rows and
the Burgers residual with its Jacobian (Sec. 3.3).

Test infrastructure (see the package docstring).

Readings:
* With a periodic prior the point data are taken on the full n x n mesh and
  the weight of a node on x = hi or y = hi goes to its mirror on the torus.
* Off-grid point data in space-time use P1 barycentric weights in space
  times linear interpolation in time.  A point on an element edge goes to the
  lower-index cell; inside a cell the lower triangle wins on the diagonal.
* Collocation uses the lumped-P1 finite-difference form of the residual at
  interior spatial nodes and time levels k >= 1:
  (u_i^k - u_i^(k-1))/dt + a_i^k (u_(i+1)^k - u_(i-1)^k)/(2h)
  - nu (u_(i+1)^k - 2 u_i^k + u_(i-1)^k)/h^2, with a = c (linear proxy) or
  a = u (Burgers).
* FEM observations (Sec. 3.1, A_ij = int <phi_i, D phi_j>, b_i = int <phi_i, f>)
  with a Crank-Nicolson discretisation in time (Sec. 5, the Burgers comparison:
  implicit-Euler prior, Crank-Nicolson FEM observations): at the same rows
  (i, k) as the collocation rows, the spatial hat phi_i tests the P1
  interpolant of each time level,
  F_ik = int phi_i (u^k - u^(k-1))/dt + 1/2 [N_i(u^k) + N_i(u^(k-1))],
  N_i(v) = int phi_i a v_x + nu int phi_i' v_x (the diffusion term integrated
  by parts; phi_i vanishes at both ends of its support), with a = c or a = v
  (Burgers).  The integrals are exact (consistent mass): three-point
  Gauss-Legendre per element, exact for the cubic integrands here.
* The observation rows are ordered: point data, then the initial-condition
  rows (every node at t = 0), then the collocation rows (t = 1..nt-1, then
  x = 1..nx-2).  Random draws for the observation part of a sample follow
  this order.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import fem


def _cell(v, lo, hi, n):
    h = (hi - lo) / (n - 1)
    i = np.floor((v - lo) / h).astype(np.int64)
    return np.clip(i, 0, n - 2), h


def _hat_weights_1d(v, lo, hi, n):
    """Cell index and the two hat-function values at v."""
    i, h = _cell(v, lo, hi, n)
    xi = lo + i * h
    w1 = (v - xi) / h
    return i, np.stack([1.0 - w1, w1], axis=1)


def _barycentric(px, py, P):
    """Barycentric coordinates of (px, py) in triangle P [3, 2] by solving
    sum_a lambda_a P_a = p, sum_a lambda_a = 1."""
    Mx = np.array([[P[0, 0], P[1, 0], P[2, 0]],
                   [P[0, 1], P[1, 1], P[2, 1]],
                   [1.0, 1.0, 1.0]])
    return np.linalg.solve(Mx, np.array([px, py, 1.0]))


def _spatial_2d_weights(prior, x, y):
    """(node indices [3], weights [3]) of the P1 interpolant at (x, y)."""
    nx, ny, _ = prior["n"]
    lo, hi = prior["lo"], prior["hi"]
    i, hx = _cell(np.array([x]), lo[0], hi[0], nx)
    j, hy = _cell(np.array([y]), lo[1], hi[1], ny)
    i, j = int(i[0]), int(j[0])
    xi, yj = lo[0] + i * hx, lo[1] + j * hy
    lower = (x - xi) / hx >= (y - yj) / hy
    if lower:
        verts = [(i, j), (i + 1, j), (i + 1, j + 1)]
    else:
        verts = [(i, j), (i + 1, j + 1), (i, j + 1)]
    P = np.array([[lo[0] + a * hx, lo[1] + b * hy] for (a, b) in verts])
    lam = _barycentric(x, y, P)
    idx = [b * nx + a for (a, b) in verts]
    return idx, lam


def point_matrix(prior: dict, coords: np.ndarray) -> sp.csr_matrix:
    """Regression rows A_ij = phi_j(x_i) (Sec. 3.1, "classic regression")."""
    kind = prior["kind"]
    nx, ny, nt = prior["n"]
    lo, hi = prior["lo"], prior["hi"]
    N = nx * ny * nt
    m = coords.shape[0]
    rows, cols, vals = [], [], []
    for r in range(m):
        if kind in ("matern2d", "steady_advdiff2d"):
            idx, lam = _spatial_2d_weights(prior, coords[r, 0], coords[r, 1])
            pairs = list(zip(idx, lam))
        elif kind == "advdiff_st1d":
            i, wx = _hat_weights_1d(np.array([coords[r, 0]]), lo[0], hi[0], nx)
            k, wt = _hat_weights_1d(np.array([coords[r, 1]]), lo[2], hi[2], nt)
            pairs = []
            for a in range(2):
                for b in range(2):
                    pairs.append(((int(k[0]) + b) * nx + int(i[0]) + a, wx[0, a] * wt[0, b]))
        else:
            idx, lam = _spatial_2d_weights(prior, coords[r, 0], coords[r, 1])
            k, wt = _hat_weights_1d(np.array([coords[r, 2]]), lo[2], hi[2], nt)
            pairs = []
            for b in range(2):
                for s_idx, s_w in zip(idx, lam):
                    pairs.append(((int(k[0]) + b) * nx * ny + s_idx, s_w * wt[0, b]))
        for c, v in pairs:
            rows.append(r)
            cols.append(c)
            vals.append(v)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(m, N))
    if fem.is_periodic(prior):
        # weights on a node of x = hi or y = hi belong to its mirror (App. B)
        A = (A @ fem.mirror_matrix(prior)).tocsr()
    return A


def ic_matrix(prior: dict) -> sp.csr_matrix:
    """Rows picking every node at t = 0 (initial condition as direct data,
    Fig. 1 "Direct measurements y, e.g. Initial condition")."""
    nx, ny, nt = prior["n"]
    ns = nx * ny
    return sp.csr_matrix((np.ones(ns), (np.arange(ns), np.arange(ns))), shape=(ns, ns * nt))


def colloc_active(prior: dict, obs: dict) -> np.ndarray:
    """Which collocation rows observe the PDE: with obs["colloc_stride"] =
    (sx, st) only the rows with i % sx == 0 and k % st == 0 (a grid of
    collocation points, coarser than the mesh); all rows by default.  The
    other rows stay in the row numbering with zero weight (no observation),
    so random draws keep their row indices."""
    sx, st = obs.get("colloc_stride", (1, 1))
    i, k = colloc_rows(prior)
    return (i % int(sx) == 0) & (k % int(st) == 0)


def colloc_rows(prior: dict):
    """(i, k) pairs of the collocation rows: interior x, time levels >= 1."""
    nx, ny, nt = prior["n"]
    assert ny == 1, "collocation rows are defined for 1D space-time"
    ks, is_ = np.meshgrid(np.arange(1, nt), np.arange(1, nx - 1), indexing="ij")
    return is_.ravel(), ks.ravel()


def burgers_residual(prior: dict, u: np.ndarray, nu: float, advect=None) -> np.ndarray:
    """Implicit-Euler, centred-difference residual of u_t + a u_x = nu u_xx at
    every collocation node, with a = u (Burgers, advect None) or a = const."""
    nx, _, nt = prior["n"]
    hx, _, dt = fem.grid_spacing(prior)
    U = u.reshape(nt, nx)
    i, k = colloc_rows(prior)
    a = U[k, i] if advect is None else advect
    return ((U[k, i] - U[k - 1, i]) / dt
            + a * (U[k, i + 1] - U[k, i - 1]) / (2.0 * hx)
            - nu * (U[k, i + 1] - 2.0 * U[k, i] + U[k, i - 1]) / hx ** 2)


def burgers_jacobian(prior: dict, u: np.ndarray, nu: float, advect=None) -> sp.csr_matrix:
    """Jacobian of burgers_residual, row by row (Sec. 3.3, J^(k))."""
    nx, _, nt = prior["n"]
    hx, _, dt = fem.grid_spacing(prior)
    U = u.reshape(nt, nx)
    i, k = colloc_rows(prior)
    m = len(i)
    r = np.arange(m)
    node = lambda kk, ii: kk * nx + ii
    if advect is None:
        a = U[k, i]
        da = (U[k, i + 1] - U[k, i - 1]) / (2.0 * hx)   # d(a u_x)/d u_i from a = u_i
    else:
        a = np.full(m, float(advect))
        da = np.zeros(m)
    entries = [
        (node(k, i), 1.0 / dt + da + 2.0 * nu / hx ** 2),
        (node(k - 1, i), np.full(m, -1.0 / dt)),
        (node(k, i + 1), a / (2.0 * hx) - nu / hx ** 2),
        (node(k, i - 1), -a / (2.0 * hx) - nu / hx ** 2),
    ]
    rows = np.concatenate([r for _ in entries])
    cols = np.concatenate([c for c, _ in entries])
    vals = np.concatenate([np.broadcast_to(v, (m,)) for _, v in entries])
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, nx * nt))


# ---------------------------------------------------------------------------
# FEM (Galerkin-tested) Crank-Nicolson rows


_GL_X = np.array([-math.sqrt(0.6), 0.0, math.sqrt(0.6)])
_GL_W = np.array([5.0, 8.0, 5.0]) / 9.0


def _fem_cn_row(xs, U, i, k, nu, dt, advect):
    """Residual F_ik and its derivatives {(level, node): dF/du} for one row,
    by Gauss-Legendre quadrature on the two elements of phi_i's support."""
    F = 0.0
    jac = {}
    for (l, r) in ((i - 1, i), (i, i + 1)):
        h = xs[r] - xs[l]
        for xq, wq in zip(_GL_X, _GL_W):
            x = xs[l] + 0.5 * h * (xq + 1.0)
            w = 0.5 * h * wq
            hat = {l: (xs[r] - x) / h, r: (x - xs[l]) / h}       # the two local hats
            dhat = {l: -1.0 / h, r: 1.0 / h}
            phi_i, dphi_i = hat[i], dhat[i]
            vals, ders = {}, {}
            for lev in (k, k - 1):
                vals[lev] = hat[l] * U[lev, l] + hat[r] * U[lev, r]
                ders[lev] = dhat[l] * U[lev, l] + dhat[r] * U[lev, r]
            F += w * phi_i * (vals[k] - vals[k - 1]) / dt
            for lev, sgn in ((k, 1.0), (k - 1, -1.0)):
                a = vals[lev] if advect is None else advect
                F += w * 0.5 * (phi_i * a * ders[lev] + nu * dphi_i * ders[lev])
                for j in (l, r):
                    da = hat[j] if advect is None else 0.0        # d a / d u_j (Burgers: a = v)
                    d = sgn * phi_i * hat[j] / dt + 0.5 * (phi_i * (da * ders[lev] + a * dhat[j]) + nu * dphi_i * dhat[j])
                    jac[(lev, j)] = jac.get((lev, j), 0.0) + w * d
    return F, jac


def fem_cn_residual(prior: dict, u: np.ndarray, nu: float, advect=None) -> np.ndarray:
    """F_ik of the FEM Crank-Nicolson rows (see the module docstring) at the
    collocation rows, for u_t + a u_x = nu u_xx with a = u (advect None) or
    a = advect."""
    nx, _, nt = prior["n"]
    xs = fem.axis_nodes(prior["lo"][0], prior["hi"][0], nx)
    _, _, dt = fem.grid_spacing(prior)
    U = u.reshape(nt, nx)
    i, k = colloc_rows(prior)
    return np.array([_fem_cn_row(xs, U, int(a), int(b), nu, dt, advect)[0] for a, b in zip(i, k)])


def fem_cn_jacobian(prior: dict, u: np.ndarray, nu: float, advect=None) -> sp.csr_matrix:
    """dF/du of fem_cn_residual (Sec. 3.3, J^(k) of the FEM rows)."""
    nx, _, nt = prior["n"]
    xs = fem.axis_nodes(prior["lo"][0], prior["hi"][0], nx)
    _, _, dt = fem.grid_spacing(prior)
    U = u.reshape(nt, nx)
    i, k = colloc_rows(prior)
    rows, cols, vals = [], [], []
    for r, (a, b) in enumerate(zip(i, k)):
        _, jac = _fem_cn_row(xs, U, int(a), int(b), nu, dt, advect)
        for (lev, j), v in jac.items():
            rows.append(r)
            cols.append(lev * nx + j)
            vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(i), nx * nt))


def pde_rows(prior: dict, obs: dict, u: np.ndarray, nu: float, advect=None):
    """(J, f(u)) of the PDE observation rows in the form obs["colloc_form"]:
    "collocation" (default; burgers_jacobian / burgers_residual) or "fem_cn"."""
    if obs.get("colloc_form", "collocation") == "fem_cn":
        return fem_cn_jacobian(prior, u, nu, advect), fem_cn_residual(prior, u, nu, advect)
    return burgers_jacobian(prior, u, nu, advect), burgers_residual(prior, u, nu, advect)
