"""Seeded synthetic workloads shaped like the paper's problems.

This module only draws inputs: grid sizes, parameters, observation locations
and observed values (a known truth function plus Gaussian noise).  It holds
none of the method's arithmetic (no FEM, no precision matrices, no solves), so
that both the CUDA path and the FP64 oracle can take their inputs from it.

A prior description is a plain dict:

    kind    "matern2d"          Whittle-Matern SPDE, alpha = 2 (Sec. 2.2)
            "advdiff_st1d"      implicit-Euler advection-diffusion in 1D space
                                 x time (Sec. 2.4, App. A)
            "advdiff_st2d"      the same in 2D space x time
            "steady_advdiff2d"  (kappa^2 - nu Lap + c d/dx) u = W in 2D
    n       (nx, ny, nt) nodes per axis, boundary nodes included (ny = 1 in
            1D space, nt = 1 for purely spatial priors)
    lo, hi  (x0, y0, t0), (x1, y1, t1) domain corners
    kappa, tau, nu, cx, cy, kappa0, eps2   SPDE parameters (see the oracle
            and the C header for their exact role)
    bc      optional: "dirichlet" (default) or "periodic" (spatial kinds)

An observation description is a dict with "coords" [m, d] (space, then time),
"y" [m], "sigma" [m] and optional collocation settings for Burgers.
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# priors


def prior_matern2d(n: int, kappa: float, eps2: float = 1e-8) -> dict:
    """2D Matern alpha=2 prior on [0,1]^2, tau set for unit marginal variance
    in the continuum limit, 1/tau^2 = 4 pi kappa^2 (Lindgren et al. 2011)."""
    return dict(kind="matern2d", n=(n, n, 1), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 0.0),
                kappa=float(kappa), tau=1.0 / math.sqrt(4.0 * math.pi * kappa * kappa),
                nu=1.0, cx=0.0, cy=0.0, kappa0=0.0, eps2=float(eps2))


def prior_steady_advdiff2d(n: int, kappa: float, nu: float, c: float, eps2: float = 1e-8) -> dict:
    return dict(kind="steady_advdiff2d", n=(n, n, 1), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 0.0),
                kappa=float(kappa), tau=1.0 / math.sqrt(4.0 * math.pi * nu * kappa * kappa),
                nu=float(nu), cx=float(c), cy=0.0, kappa0=0.0, eps2=float(eps2))


def prior_st1d(nx: int, nt: int, c: float, nu: float, tau: float = 1.0, kappa0: float = 10.0,
               x0: float = 0.0, x1: float = 1.0, t1: float = 1.0, eps2: float = 1e-8) -> dict:
    return dict(kind="advdiff_st1d", n=(nx, 1, nt), lo=(x0, 0.0, 0.0), hi=(x1, 0.0, t1),
                kappa=kappa0, tau=float(tau), nu=float(nu), cx=float(c), cy=0.0,
                kappa0=float(kappa0), eps2=float(eps2))


def prior_st2d(n: int, nt: int, cx: float, cy: float, nu: float, kappa: float, tau: float = 1.0,
               t1: float = 1.0, eps2: float = 1e-8) -> dict:
    return dict(kind="advdiff_st2d", n=(n, n, nt), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, t1),
                kappa=float(kappa), tau=float(tau), nu=float(nu), cx=float(cx), cy=float(cy),
                kappa0=float(kappa), eps2=float(eps2))


def periodic(prior: dict) -> dict:
    """The same spatial prior with the periodic boundary of App. B (N_k = 1):
    the nodes on x = hi and y = hi are the mirrors of those on x = lo and
    y = lo, so the unknowns are the (n - 1)^2 nodes of the torus."""
    assert prior["kind"] in ("matern2d", "steady_advdiff2d")
    return dict(prior, bc="periodic")


def n_nodes(prior: dict) -> int:
    nx, ny, nt = prior["n"]
    if prior.get("bc", "dirichlet") == "periodic":
        return (nx - 1) * (ny - 1)
    return nx * ny * nt


def obs_dim(prior: dict) -> int:
    """Coordinates per observation: spatial dims, plus time for space-time."""
    return {"matern2d": 2, "steady_advdiff2d": 2, "advdiff_st1d": 2, "advdiff_st2d": 3}[prior["kind"]]


# ---------------------------------------------------------------------------
# truth functions (data generators only)


def fourier_modes(rng: np.random.Generator, k: int = 20, dim: int = 2, wmax: int = 8):
    """Random sum of k sine modes with integer frequencies in [1, wmax]^dim,
    amplitudes N(0, 1/k) and phases U[0, 2 pi)."""
    a = rng.normal(0.0, math.sqrt(1.0 / k), size=k)
    w = rng.integers(1, wmax + 1, size=(k, dim))
    ph = rng.uniform(0.0, 2.0 * math.pi, size=k)

    def f(x):
        x = np.atleast_2d(x)
        return (a[None, :] * np.sin(2.0 * math.pi * (x @ w.T) + ph[None, :])).sum(axis=1)
    return f


def decaying_sine(x, t):
    """u*(x, t) = exp(-t) sin(pi x)."""
    return np.exp(-t) * np.sin(math.pi * x)


def cole_hopf_burgers(x, t, nu: float, npts: int = 4001):
    """Viscous Burgers on (-1, 1), u(x,0) = -sin(pi x), u(+-1,t) = 0, through
    the Cole-Hopf transform (the 2-periodic odd extension of the initial
    condition keeps u(+-1, t) = 0): u = -2 nu phi_x / phi with
    phi(x,t) = int exp(-(x-y)^2/(4 nu t) + (1 - cos(pi y)) / (2 pi nu)) dy.
    Written as u = (r / t) E[s], s = (x - y) / r, r = sqrt(4 nu t), under the
    weight exp(-s^2 + (1 - cos(pi y)) / (2 pi nu)); the expectation is taken
    by the trapezoid rule on s in [-12, 12]."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    xb, tb = np.broadcast_arrays(x, t)
    xf, tf = xb.ravel(), tb.ravel()
    out = np.empty(xf.shape)
    s = np.linspace(-12.0, 12.0, npts)
    for lo in range(0, xf.size, 256):
        xs, ts = xf[lo:lo + 256], tf[lo:lo + 256]
        pos = ts > 0.0
        r = np.sqrt(4.0 * nu * np.where(pos, ts, 1.0))
        y = xs[:, None] - r[:, None] * s[None, :]
        e = -s[None, :] ** 2 + (1.0 - np.cos(np.pi * y)) / (2.0 * np.pi * nu)
        e -= e.max(axis=1, keepdims=True)
        g = np.exp(e)
        val = (r / np.where(pos, ts, 1.0)) * (g * s[None, :]).sum(axis=1) / g.sum(axis=1)
        out[lo:lo + 256] = np.where(pos, val, -np.sin(np.pi * xs))
    return out.reshape(xb.shape)


# ---------------------------------------------------------------------------
# observation sets


def point_obs(prior: dict, m: int, sigma: float, truth, seed: int) -> dict:
    """m points uniform over the (space[, time]) domain, y = truth + N(0, sigma^2)."""
    rng = np.random.default_rng(seed)
    d = obs_dim(prior)
    lo, hi = prior["lo"], prior["hi"]
    kind = prior["kind"]
    if kind in ("matern2d", "steady_advdiff2d"):
        axes = [(lo[0], hi[0]), (lo[1], hi[1])]
    elif kind == "advdiff_st1d":
        axes = [(lo[0], hi[0]), (lo[2], hi[2])]
    else:
        axes = [(lo[0], hi[0]), (lo[1], hi[1]), (lo[2], hi[2])]
    coords = np.stack([rng.uniform(a, b, size=m) for (a, b) in axes], axis=1)
    assert coords.shape == (m, d)
    y = truth(coords) + rng.normal(0.0, sigma, size=m)
    return dict(coords=coords, y=y, sigma=np.full(m, float(sigma)))


def node_obs(prior: dict, frac: float, sigma: float, truth, seed: int) -> dict:
    """Observations at a random subset of grid nodes (distinct nodes)."""
    rng = np.random.default_rng(seed)
    nx, ny, _ = prior["n"]
    lo, hi = prior["lo"], prior["hi"]
    nn = nx * ny
    m = max(1, int(round(frac * nn)))
    pick = rng.choice(nn, size=m, replace=False)
    ix, iy = pick % nx, pick // nx
    xs = lo[0] + (hi[0] - lo[0]) * ix / (nx - 1)
    ys = lo[1] + (hi[1] - lo[1]) * iy / (ny - 1)
    coords = np.stack([xs, ys], axis=1)
    y = truth(coords) + rng.normal(0.0, sigma, size=m)
    return dict(coords=coords, y=y, sigma=np.full(m, float(sigma)))


def torus_node_obs(prior: dict, sigma: float, truth, seed: int) -> dict:
    """One observation at every node of a periodic prior's torus (x = lo + i h,
    i < n - 1), y = truth + N(0, sigma^2)."""
    rng = np.random.default_rng(seed)
    nx, ny, _ = prior["n"]
    lo, hi = prior["lo"], prior["hi"]
    ix = np.tile(np.arange(nx - 1), ny - 1)
    iy = np.repeat(np.arange(ny - 1), nx - 1)
    xs = lo[0] + (hi[0] - lo[0]) * ix / (nx - 1)
    ys = lo[1] + (hi[1] - lo[1]) * iy / (ny - 1)
    coords = np.stack([xs, ys], axis=1)
    y = truth(coords) + rng.normal(0.0, sigma, size=len(xs))
    return dict(coords=coords, y=y, sigma=np.full(len(xs), float(sigma)))


def periodic_fourier(rng: np.random.Generator, k: int = 20, wmax: int = 8):
    """Sum of k random Fourier modes of period one in x and y (a smooth
    periodic truth)."""
    kx = rng.integers(-wmax, wmax + 1, size=k)
    ky = rng.integers(-wmax, wmax + 1, size=k)
    amp = rng.normal(size=k) / np.sqrt(k)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=k)

    def f(z):
        z = np.atleast_2d(z)
        return np.sum(amp * np.cos(2.0 * np.pi * (np.outer(z[:, 0], kx) + np.outer(z[:, 1], ky)) + ph), axis=1)
    return f


def c2_matern_periodic(n: int = 513, m: int = 10000, seed: int = 2, kappa: float = 20.0, all_nodes: bool = False,
                       sigma: float = 0.1):
    """The 2D Matern workload on the unit torus (periodic boundary, (n-1)^2
    unknowns): m uniform point observations of a periodic 20-mode Fourier sum
    plus N(0, sigma^2), or with all_nodes one observation at every node."""
    pr = periodic(prior_matern2d(n, kappa))
    rng = np.random.default_rng(seed + 200)
    f = periodic_fourier(rng, 20, 8)
    if all_nodes:
        return pr, torus_node_obs(pr, sigma, f, seed)
    return pr, point_obs(pr, m, sigma, f, seed)


# ---------------------------------------------------------------------------
# the five workloads (full size) and their small replicas


def c1_st1d(nx: int = 64, nt: int = 64, m: int = 50, seed: int = 1):
    """1D advection-diffusion space-time prior, 50 point observations of
    exp(-t) sin(pi x) + N(0, 1e-4)."""
    pr = prior_st1d(nx, nt, c=0.5, nu=0.01, tau=1.0, kappa0=10.0)
    ob = point_obs(pr, m, 1e-2, lambda z: decaying_sine(z[:, 0], z[:, 1]), seed)
    return pr, ob


def c2_matern(n: int = 512, m: int = 10000, seed: int = 2, kappa: float = 20.0):
    """2D Matern, kappa = 20, m point observations of a 20-mode Fourier sum
    plus N(0, 1e-2)."""
    pr = prior_matern2d(n, kappa)
    rng = np.random.default_rng(seed + 100)
    f = fourier_modes(rng, 20, 2, 8)
    ob = point_obs(pr, m, 0.1, f, seed)
    return pr, ob


def c3_burgers(nx: int = 1024, nt: int = 1024, m: int = 200, seed: int = 3, nu: float = 0.01):
    """Burgers on (-1,1) x (0,1): advection-diffusion proxy prior (c = 1),
    collocation of the Burgers residual at interior nodes (sigma 1e-6), the
    initial condition -sin(pi x) at t = 0 (sigma 1e-6), and m data points
    of the Cole-Hopf truth plus N(0, 1e-4)."""
    pr = prior_st1d(nx, nt, c=1.0, nu=nu, tau=1.0, kappa0=10.0, x0=-1.0, x1=1.0, t1=1.0)
    rng = np.random.default_rng(seed)
    xs = rng.uniform(-1.0, 1.0, size=m)
    ts = rng.uniform(0.0, 1.0, size=m)
    y = cole_hopf_burgers(xs, ts, nu) + rng.normal(0.0, 1e-2, size=m)
    ob = dict(coords=np.stack([xs, ts], axis=1), y=y, sigma=np.full(m, 1e-2),
              colloc_sigma=1e-6, ic_sigma=1e-6, burgers_nu=nu)
    return pr, ob


def c4_instances(count: int = 256, seed: int = 4, smin: int = 64, smax: int = 512):
    """Independent 2D instances: sides log-uniform in [smin, smax], Matern or
    steady advection-diffusion (50/50), kappa U[5,40], c U[0,2],
    nu U[1e-3, 1e-1], 1-5 % of nodes observed with sigma U[1e-3, 1e-1]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        kappa = rng.uniform(5.0, 40.0)
        if rng.uniform() < 0.5:
            pr = prior_matern2d(n, kappa)
        else:
            pr = prior_steady_advdiff2d(n, kappa, nu=rng.uniform(1e-3, 1e-1), c=rng.uniform(0.0, 2.0))
        frac = rng.uniform(0.01, 0.05)
        sigma = rng.uniform(1e-3, 1e-1)
        f = fourier_modes(np.random.default_rng(seed * 1000 + i), 10, 2, 6)
        ob = node_obs(pr, frac, sigma, f, seed * 1000 + i + 7)
        out.append((pr, ob))
    return out


def c5_st2d(n: int = 256, nt: int = 256, m: int = 50000, seed: int = 5):
    """2D advection-diffusion space-time prior, velocity (0.5, 0), nu 0.01,
    kappa 10, tau 1; m points of a smooth space-time Fourier truth plus
    N(0, 0.01)."""
    pr = prior_st2d(n, nt, cx=0.5, cy=0.0, nu=0.01, kappa=10.0, tau=1.0)
    f = fourier_modes(np.random.default_rng(seed + 100), 12, 3, 4)
    ob = point_obs(pr, m, 0.1, f, seed)
    return pr, ob


#: random-draw seeds for the Philox streams (samples, probes), per workload
DRAW_SEED = {"c1": 1001, "c2": 1002, "c3": 1003, "c4": 1004, "c5": 1005}


# ---------------------------------------------------------------------------
# physics-informed vs generic prior on Burgers (the Sec. 5 prior comparison,
# on synthetic data): the initial condition as data, nonlinear collocation
# at a grid of points coarser than the mesh


STUDY_PRIORS = ("advdiff", "product_matern")


def burgers_prior_study(prior: str, stride, nx: int = 257, nt: int = 101, nu: float = 0.01,
                        noise_kappa: float = 35.0, colloc_sigma: float = 1e-2, ic_sigma: float = 1e-3):
    """Burgers on (-1, 1) x (0, 1) with u(x, 0) = -sin(pi x) observed at every
    t = 0 node (noise ic_sigma) and the collocation rows on the points
    x % sx == 0, k % st == 0 (stride (sx, st); None: no collocation).
    prior "advdiff": the advection-diffusion proxy with the bulk advection of
    the initial condition (its mean, zero for -sin(pi x)) and the diffusion of
    the equation, with Matern transition noise of inverse range noise_kappa;
    "product_matern": no dynamics (c = nu = 0), the same Matern noise and an
    AR(1) decay with temporal range 3 (a separable Matern prior with
    nu_t = 1/2 in time).  Returns (prior, obs)."""
    if prior == "advdiff":
        xs = np.linspace(-1.0, 1.0, nx)
        c = float(np.round(np.mean(-np.sin(np.pi * xs)), 12)) + 0.0   # bulk advection of the initial condition
        pr = prior_st1d(nx, nt, c=c, nu=nu, tau=1.0, kappa0=10.0, x0=-1.0, x1=1.0, t1=1.0)
        pr = dict(pr, noise_kappa=float(noise_kappa))
    else:
        dt = 1.0 / (nt - 1)
        decay = 1.0 - math.exp(-dt / 3.0)
        # stationary variance tau^2 dt / (1 - rho^2) of about one
        tau = math.sqrt((1.0 - (1.0 - decay) ** 2) / dt)
        pr = prior_st1d(nx, nt, c=0.0, nu=0.0, tau=tau, kappa0=float(noise_kappa), x0=-1.0, x1=1.0, t1=1.0)
        pr = dict(pr, noise_kappa=float(noise_kappa), decay=decay)
    ob = dict(coords=np.zeros((0, 2)), y=np.zeros(0), sigma=np.zeros(0), ic_sigma=float(ic_sigma), burgers_nu=nu)
    if stride is not None:
        ob = dict(ob, colloc_sigma=float(colloc_sigma), colloc_stride=(int(stride[0]), int(stride[1])))
    return pr, ob
