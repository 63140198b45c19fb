"""P1 FEM assembly and the SPDE prior precision, written as element loops.

Test infrastructure (see the package docstring): float64, slow, explicit.

Readings of the paper used here (where it is silent or ambiguous):

* n nodes per axis include the boundary; h = (hi - lo) / (n - 1).  Time
  levels include t = 0, dt = T / (nt - 1).
* 2D meshes split every cell (i, j) along the diagonal (i, j) -> (i+1, j+1).
* Mass lumping everywhere (Sec. 2.2): Ml_ii = row sum of the consistent mass.
* Homogeneous Dirichlet boundary (App. B, N_k = 0): rows and columns of the
  constrained matrices are zeroed and the diagonal set to 1; the boundary
  DOF is given variance eps2 (App. B "M_kk = eps_k^2"), independent of tau.
* Periodic boundary (App. B, N_k = 1, c_1 = 1, h(1) = mirror(k)), for the
  spatial kinds with prior["bc"] == "periodic": the nodes on x = hi and on
  y = hi are constrained to their mirrors on x = lo and y = lo.  App. B adds
  column k to column mirror(k); for the FEM assembly the test functions are
  periodic too, so row k is added to row mirror(k) (without it the rows of
  the mirror nodes would hold half an element ring and the operator would
  not be translation invariant).  The constrained rows become e_k with
  M_kk = eps_k^2, and we take App. B's hard limit eps_k -> 0: u_k = 0, the
  field at k equals the field at mirror(k), and the unknowns are the
  (n - 1)^2 nodes of the torus.  In matrix form K_t = T^T K T and
  ml_t = T^T ml with T the n^2 x (n - 1)^2 mirror map.
* Matern transition noise (App. A: "we choose W_s as spatial Matern noise"),
  when prior["noise_kappa"] > 0: the spatial noise W_s is the unit-variance
  alpha = 2 Matern field with inverse range kappa_s, Dirichlet on the same
  boundary, so the FEM-tested noise w = int phi W_s of the interior has
  covariance tau^2 dt Ml Sigma_s Ml with Sigma_s^-1 = tau_s^2 K_s Ml^-1 K_s
  (K_s = kappa_s^2 Ml + S on the interior, tau_s = matern_tau_unit(kappa_s)).
  The root of its precision is (tau_s / (tau sqrt dt)) Ml^-1/2 K_s Ml^-1, so
  the interior rows of the level blocks are T_K times the white-noise rows,
  T_K = tau_s Ml^-1/2 K_s Ml^-1/2 (symmetric; identity on the boundary rows
  and on the initial level).  prior["decay"] (default 0) scales the previous
  level by rho = 1 - decay: G u^k = rho Ml u^(k-1) + w (an AR(1) in time).
* Space-time noise is otherwise white in space and lumped, w ~ N(0, tau^2 dt Ml)
  (App. A with Sigma = M^-1), so the whole prior scales as tau^-2.  The
  initial block is a Matern alpha = 2 precision with kappa0, normalised to
  unit marginal variance (tau0).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def axis_nodes(lo: float, hi: float, n: int) -> np.ndarray:
    return np.linspace(lo, hi, n)


# ---------------------------------------------------------------------------
# 1D P1 elements (segments)


def p1_1d(x: np.ndarray, c: float = 0.0):
    """Stiffness S_ij = int phi_i' phi_j', lumped mass ml_i = int phi_i and
    advection Badv_ij = int phi_i c phi_j' on the segment mesh x (element
    loop; Sec. 2.2, FEM discretisation of the SPDE)."""
    n = len(x)
    rows, cols, vs, va = [], [], [], []
    ml = np.zeros(n)
    for e in range(n - 1):
        loc = (e, e + 1)
        h = x[e + 1] - x[e]
        grad = (-1.0 / h, 1.0 / h)          # derivatives of the two hats
        for a in range(2):
            ml[loc[a]] += 0.5 * h           # int phi_a over the segment
            for b in range(2):
                rows.append(loc[a])
                cols.append(loc[b])
                vs.append(h * grad[a] * grad[b])
                va.append(0.5 * h * c * grad[b])   # int phi_a = h/2, phi_b' const
    S = sp.csr_matrix((vs, (rows, cols)), shape=(n, n))
    Badv = sp.csr_matrix((va, (rows, cols)), shape=(n, n))
    return S, ml, Badv


# ---------------------------------------------------------------------------
# 2D P1 elements (triangles of a structured grid)


def triangles(nx: int, ny: int):
    """Vertex index triples; node (i, j) has index j * nx + i.  Each cell is
    split along (i,j)->(i+1,j+1): lower (i,j),(i+1,j),(i+1,j+1) and upper
    (i,j),(i+1,j+1),(i,j+1)."""
    tris = []
    for j in range(ny - 1):
        for i in range(nx - 1):
            a, b = j * nx + i, j * nx + i + 1
            c, d = (j + 1) * nx + i + 1, (j + 1) * nx + i
            tris.append((a, b, c))
            tris.append((a, c, d))
    return np.array(tris, dtype=np.int64)


def p1_2d(xs: np.ndarray, ys: np.ndarray, vx: float = 0.0, vy: float = 0.0):
    """Stiffness S_ab = int grad phi_a . grad phi_b, lumped mass ml_a =
    int phi_a and advection Badv_ab = int phi_a (v . grad phi_b), assembled
    triangle by triangle from barycentric gradients."""
    nx, ny = len(xs), len(ys)
    X = np.tile(xs, ny)
    Y = np.repeat(ys, nx)
    tris = triangles(nx, ny)
    P = np.stack([X[tris], Y[tris]], axis=-1)          # [T, 3, 2]
    x1, x2, x3 = P[:, 0, 0], P[:, 1, 0], P[:, 2, 0]
    y1, y2, y3 = P[:, 0, 1], P[:, 1, 1], P[:, 2, 1]
    det = (x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1)  # 2 * signed area
    area = 0.5 * np.abs(det)
    # gradient of barycentric coordinate lambda_a: (y_b - y_c, x_c - x_b) / det
    gx = np.stack([y2 - y3, y3 - y1, y1 - y2], axis=1) / det[:, None]
    gy = np.stack([x3 - x2, x1 - x3, x2 - x1], axis=1) / det[:, None]
    rows, cols, vs, va = [], [], [], []
    ml = np.zeros(nx * ny)
    for a in range(3):
        np.add.at(ml, tris[:, a], area / 3.0)
        for b in range(3):
            rows.append(tris[:, a])
            cols.append(tris[:, b])
            vs.append(area * (gx[:, a] * gx[:, b] + gy[:, a] * gy[:, b]))
            va.append(area / 3.0 * (vx * gx[:, b] + vy * gy[:, b]))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    N = nx * ny
    S = sp.csr_matrix((np.concatenate(vs), (rows, cols)), shape=(N, N))
    Badv = sp.csr_matrix((np.concatenate(va), (rows, cols)), shape=(N, N))
    return S, ml, Badv


# ---------------------------------------------------------------------------
# Dirichlet constraint (App. B)


def is_periodic(prior: dict) -> bool:
    return prior.get("bc", "dirichlet") == "periodic"


def mirror_matrix(prior: dict) -> sp.csr_matrix:
    """T: the n_x n_y mesh nodes -> the (n_x - 1)(n_y - 1) torus nodes,
    T[(i, j), (i mod (n_x - 1), j mod (n_y - 1))] = 1 (App. B periodic
    boundary: a node on x = hi or y = hi is its mirror on x = lo or y = lo)."""
    nx, ny, _ = prior["n"]
    mx, my = nx - 1, ny - 1
    rows, cols = [], []
    for j in range(ny):
        for i in range(nx):
            rows.append(j * nx + i)
            cols.append((j % my) * mx + (i % mx))
    return sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(nx * ny, mx * my))


def num_unknowns(prior: dict) -> int:
    nx, ny, nt = prior["n"]
    if is_periodic(prior):
        return (nx - 1) * (ny - 1)
    return nx * ny * nt


def spatial_boundary(prior: dict) -> np.ndarray:
    """Boolean mask over the spatial nodes of the Dirichlet boundary (none on
    the torus of a periodic prior)."""
    nx, ny, _ = prior["n"]
    if is_periodic(prior):
        return np.zeros((nx - 1) * (ny - 1), dtype=bool)
    i = np.tile(np.arange(nx), ny)
    j = np.repeat(np.arange(ny), nx)
    bnd = (i == 0) | (i == nx - 1)
    if ny > 1:
        bnd |= (j == 0) | (j == ny - 1)
    return bnd


def boundary_mask(prior: dict) -> np.ndarray:
    """Dirichlet mask over all unknowns (the spatial boundary at every time
    level)."""
    _, _, nt = prior["n"]
    return np.tile(spatial_boundary(prior), nt)


def constrain(X: sp.spmatrix, bnd: np.ndarray) -> sp.csr_matrix:
    """App. B with N_k = 0: zero column k, zero row k, set X_kk = 1."""
    keep = sp.diags((~bnd).astype(float))
    X = keep @ X @ keep
    return (X + sp.diags(bnd.astype(float))).tocsr()


# ---------------------------------------------------------------------------
# spatial operators of each prior kind


def spatial_mesh(prior: dict):
    """Returns (S, ml, Badv, dim) on the spatial mesh of the prior, where
    Badv already carries the velocity (cx, cy)."""
    nx, ny, _ = prior["n"]
    lo, hi = prior["lo"], prior["hi"]
    xs = axis_nodes(lo[0], hi[0], nx)
    if ny == 1:
        S, ml, Badv = p1_1d(xs, prior["cx"])
        return S, ml, Badv, 1
    ys = axis_nodes(lo[1], hi[1], ny)
    S, ml, Badv = p1_2d(xs, ys, prior["cx"], prior["cy"])
    return S, ml, Badv, 2


def matern_tau_unit(kappa: float, dim: int) -> float:
    """tau giving unit marginal variance for the alpha = 2 Matern field,
    sigma^2 = Gamma(nu)/(Gamma(nu + d/2) (4 pi)^(d/2) kappa^(2 nu) tau^2) with
    nu = 2 - d/2 (Lindgren et al. 2011, the SPDE prior of Sec. 2.2):
    1D: 1/(4 kappa^3 tau^2), 2D: 1/(4 pi kappa^2 tau^2)."""
    if dim == 1:
        return 1.0 / math.sqrt(4.0 * kappa ** 3)
    return 1.0 / math.sqrt(4.0 * math.pi * kappa ** 2)


def prior_root(prior: dict) -> sp.csr_matrix:
    """Square sparse root B with Q = B^T B.

    Spatial priors (Sec. 2.2): B = tau Ml^-1/2 Kc, Kc the constrained
    K = kappa^2 Ml + S (Matern) or kappa^2 Ml + nu S + Badv (steady
    advection-diffusion); boundary rows are e_k / eps.

    Space-time (Sec. 2.4, App. A), block rows in time:
      t = 0:  (tau0 / tau) Ml^-1/2 K0c, K0 = kappa0^2 Ml + S
      t >= 1: (tau sqrt(dt))^-1 Ml^-1/2 (Gc u^k - Mlc u^(k-1)),
              G = Ml + dt (nu S + Badv)
    where Mlc is Ml with boundary rows removed; boundary rows e_k / eps.
    """
    kind = prior["kind"]
    if is_periodic(prior):
        # App. B periodic constraint on rows and columns, hard limit (see the
        # module docstring): B = tau ml_t^-1/2 T^T K T
        assert kind in ("matern2d", "steady_advdiff2d"), "periodic boundary: spatial priors only"
        T = mirror_matrix(prior)
        ml = spatial_mesh(prior)[1]
        Kt = T.T @ prior_root_K(prior) @ T
        mlt = T.T @ ml
        return (sp.diags(prior["tau"] / np.sqrt(mlt)) @ Kt).tocsr()
    S, ml, Badv, dim = spatial_mesh(prior)
    Ns = len(ml)
    sbnd = spatial_boundary(prior)
    inv_eps = 1.0 / math.sqrt(prior["eps2"])
    if kind in ("matern2d", "steady_advdiff2d"):
        if kind == "matern2d":      # (kappa^2 - Laplacian): no diffusion or advection coefficient
            K = prior["kappa"] ** 2 * sp.diags(ml) + S
        else:
            K = prior["kappa"] ** 2 * sp.diags(ml) + prior["nu"] * S + Badv
        Kc = constrain(K, sbnd)
        d = np.where(sbnd, inv_eps, prior["tau"] / np.sqrt(ml))
        return (sp.diags(d) @ Kc).tocsr()
    assert kind in ("advdiff_st1d", "advdiff_st2d")
    nt = prior["n"][2]
    dt = (prior["hi"][2] - prior["lo"][2]) / (nt - 1)
    tau = prior["tau"]
    tau0 = matern_tau_unit(prior["kappa0"], dim)
    K0c = constrain(prior["kappa0"] ** 2 * sp.diags(ml) + S, sbnd)
    Gc = constrain(sp.diags(ml) + dt * (prior["nu"] * S + Badv), sbnd)
    rho = 1.0 - prior.get("decay", 0.0)
    Mlc = sp.diags(np.where(sbnd, 0.0, ml))
    d0 = np.where(sbnd, inv_eps, (tau0 / tau) / np.sqrt(ml))
    dk = np.where(sbnd, inv_eps, 1.0 / (tau * math.sqrt(dt) * np.sqrt(ml)))
    TK = noise_transform(prior)
    blocks = [[None] * nt for _ in range(nt)]
    blocks[0][0] = sp.diags(d0) @ K0c
    for k in range(1, nt):
        blocks[k][k] = TK @ sp.diags(dk) @ Gc
        blocks[k][k - 1] = -rho * (TK @ sp.diags(dk) @ Mlc)
    for k in range(nt):
        for l in range(nt):
            if blocks[k][l] is None and abs(k - l) > 1:
                continue
            if blocks[k][l] is None:
                blocks[k][l] = sp.csr_matrix((Ns, Ns))
    B = sp.bmat(blocks, format="csr")
    return B


def noise_transform(prior: dict) -> sp.csr_matrix:
    """T_K of the Matern transition noise (see the module docstring) on one
    time level: tau_s Ml^-1/2 K_s Ml^-1/2 on the interior nodes, identity on
    the boundary; the identity for white noise."""
    S, ml, _, dim = spatial_mesh(prior)
    ks = prior.get("noise_kappa", 0.0)
    if not ks > 0.0:
        return sp.identity(len(ml), format="csr")
    sbnd = spatial_boundary(prior)
    keep = sp.diags((~sbnd).astype(float))
    Ks = keep @ (ks ** 2 * sp.diags(ml) + S) @ keep            # K_s on the interior block
    r = 1.0 / np.sqrt(ml)
    return (matern_tau_unit(ks, dim) * sp.diags(r) @ Ks @ sp.diags(r) + sp.diags(sbnd.astype(float))).tocsr()


def _zero_boundary(X: sp.spmatrix, bnd: np.ndarray) -> sp.csr_matrix:
    """keep X keep: the derivative of constrain(X) (the unit diagonal it adds
    on the boundary does not depend on any parameter)."""
    keep = sp.diags((~bnd).astype(float))
    return (keep @ X @ keep).tocsr()


def prior_root_derivative(prior: dict, name: str) -> sp.csr_matrix:
    """dB/dtheta of the root of prior_root, exactly, for theta in
    (log_kappa, log_tau, c, nu) (c: the x velocity).  B is affine in
    kappa^2, c and nu inside K or G, carries tau as a row scale (tau for the
    spatial priors, 1/tau for space-time), and in the space-time t = 0 block
    the unit-variance scale tau0(kappa0) as well; boundary rows e_k / eps do
    not depend on any parameter.  The Matern kind has no c or nu.
    Space-time priors: kappa means kappa0 (the initial block)."""
    kind = prior["kind"]
    S, ml, _, dim = spatial_mesh(prior)
    nx, ny, _ = prior["n"]
    if is_periodic(prior):
        T = mirror_matrix(prior)
        d = prior["tau"] / np.sqrt(T.T @ ml)
        if name == "log_tau":
            dK = prior_root_K(prior)
        elif name == "log_kappa":
            dK = 2.0 * prior["kappa"] ** 2 * sp.diags(ml)
        elif kind == "matern2d":
            return sp.csr_matrix((len(d), len(d)))
        elif name == "c":
            dK = p1_2d(axis_nodes(prior["lo"][0], prior["hi"][0], nx),
                       axis_nodes(prior["lo"][1], prior["hi"][1], ny), 1.0, 0.0)[2]
        else:
            dK = S
        return (sp.diags(d) @ (T.T @ dK @ T)).tocsr()
    sbnd = spatial_boundary(prior)
    xs = axis_nodes(prior["lo"][0], prior["hi"][0], nx)
    if dim == 1:
        Bx = p1_1d(xs, 1.0)[2]
    else:
        Bx = p1_2d(xs, axis_nodes(prior["lo"][1], prior["hi"][1], ny), 1.0, 0.0)[2]
    Ml = sp.diags(ml)
    if kind in ("matern2d", "steady_advdiff2d"):
        d = np.where(sbnd, 0.0, prior["tau"] / np.sqrt(ml))      # interior row scale
        if name == "log_tau":
            return (sp.diags(d) @ constrain(prior_root_K(prior), sbnd)).tocsr()
        if name == "log_kappa":
            dK = 2.0 * prior["kappa"] ** 2 * Ml
        elif kind == "matern2d":
            return sp.csr_matrix((len(ml), len(ml)))
        elif name == "c":
            dK = Bx
        else:
            dK = S
        return (sp.diags(d) @ _zero_boundary(dK, sbnd)).tocsr()
    nt = prior["n"][2]
    Ns = len(ml)
    dt = (prior["hi"][2] - prior["lo"][2]) / (nt - 1)
    tau, k0 = prior["tau"], prior["kappa0"]
    tau0 = matern_tau_unit(k0, dim)
    d0 = np.where(sbnd, 0.0, (tau0 / tau) / np.sqrt(ml))
    dk = np.where(sbnd, 0.0, 1.0 / (tau * math.sqrt(dt) * np.sqrt(ml)))
    zero = sp.csr_matrix((Ns, Ns))
    blocks = [[None] * nt for _ in range(nt)]
    if name == "log_tau":
        # every interior row scales as 1/tau
        K0c = constrain(k0 ** 2 * Ml + S, sbnd)
        Gc = constrain(Ml + dt * (prior["nu"] * S + spatial_mesh(prior)[2]), sbnd)
        Mlc = sp.diags(np.where(sbnd, 0.0, ml))
        blocks[0][0] = -(sp.diags(d0) @ K0c)
        for k in range(1, nt):
            blocks[k][k] = -(sp.diags(dk) @ Gc)
            blocks[k][k - 1] = sp.diags(dk) @ Mlc
    elif name == "log_kappa":
        # d/dlog kappa0 of diag(d0) K0c: d0 ~ tau0(kappa0) with the exponent
        # of matern_tau_unit (tau0 ~ kappa0^-3/2 in 1D, kappa0^-1 in 2D), and
        # K0 = kappa0^2 Ml + S
        dlog_tau0 = -1.5 if dim == 1 else -1.0
        K0c = constrain(k0 ** 2 * Ml + S, sbnd)
        blocks[0][0] = dlog_tau0 * (sp.diags(d0) @ K0c) + sp.diags(d0) @ _zero_boundary(2.0 * k0 ** 2 * Ml, sbnd)
    else:
        dG = dt * (Bx if name == "c" else S)
        for k in range(1, nt):
            blocks[k][k] = sp.diags(dk) @ _zero_boundary(dG, sbnd)
    TK = noise_transform(prior)
    rho = 1.0 - prior.get("decay", 0.0)
    for k in range(1, nt):          # the transition rows carry T_K (and the decay on the previous level)
        if blocks[k][k] is not None:
            blocks[k][k] = TK @ blocks[k][k]
        if blocks[k][k - 1] is not None:
            blocks[k][k - 1] = rho * (TK @ blocks[k][k - 1])
    for k in range(nt):
        for l in range(nt):
            if blocks[k][l] is None and (k == l or k == l + 1):
                blocks[k][l] = zero
    return sp.bmat(blocks, format="csr")


def prior_root_K(prior: dict) -> sp.spmatrix:
    """The unconstrained operator K of a spatial prior (Matern:
    kappa^2 Ml + S; steady advection-diffusion: kappa^2 Ml + nu S + Badv)."""
    S, ml, Badv, _ = spatial_mesh(prior)
    if prior["kind"] == "matern2d":
        return prior["kappa"] ** 2 * sp.diags(ml) + S
    return prior["kappa"] ** 2 * sp.diags(ml) + prior["nu"] * S + Badv


def prior_precision(prior: dict) -> sp.csr_matrix:
    """Q = B^T B (Sec. 2.2 eq. sparse-prec-matrix; App. A eq.
    block-tridiag-prec)."""
    B = prior_root(prior)
    return (B.T @ B).tocsr()


def grid_spacing(prior: dict):
    nx, ny, nt = prior["n"]
    lo, hi = prior["lo"], prior["hi"]
    hx = (hi[0] - lo[0]) / (nx - 1)
    hy = (hi[1] - lo[1]) / (ny - 1) if ny > 1 else 0.0
    dt = (hi[2] - lo[2]) / (nt - 1) if nt > 1 else 0.0
    return hx, hy, dt
