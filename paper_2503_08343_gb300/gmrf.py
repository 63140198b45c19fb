"""Thin Python binding of the C ABI in include/gmrf.h (ctypes).

Argument marshalling only: every step of the computation runs in libgmrf.so.
Arrays may be numpy arrays (host memory) or CUDA torch tensors (device
memory); float64, C-contiguous.  The library fails loudly when it is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

KIND = {"matern2d": 0, "advdiff_st1d": 1, "advdiff_st2d": 2, "steady_advdiff2d": 3}
STATUS = {0: "ok", 1: "invalid argument", 2: "not positive definite", 3: "no convergence",
          4: "CUDA error", 5: "out of device memory", 6: "timeout"}


class PriorDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nt", C.c_int32),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("kappa", C.c_double), ("tau", C.c_double), ("nu", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("kappa0", C.c_double), ("eps2", C.c_double),
                ("bc", C.c_int32), ("noise_kappa", C.c_double), ("decay", C.c_double)]


class ObsDesc(C.Structure):
    _fields_ = [("m", C.c_int64), ("coords", C.POINTER(C.c_double)), ("y", C.POINTER(C.c_double)),
                ("sigma", C.POINTER(C.c_double)), ("sigma_all", C.c_double),
                ("ic", C.c_int32), ("ic_sigma", C.c_double), ("ic_values", C.POINTER(C.c_double)),
                ("colloc", C.c_int32), ("colloc_sigma", C.c_double), ("colloc_c", C.c_double),
                ("colloc_nu", C.c_double), ("colloc_f", C.POINTER(C.c_double)),
                ("colloc_stride_x", C.c_int32), ("colloc_stride_t", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_refine", C.c_int32), ("max_inner", C.c_int32),
                ("inner_rtol", C.c_double), ("precision", C.c_int32), ("batched", C.c_int32),
                ("timeout_s", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("nrhs", C.c_int32), ("refinements", C.c_int32), ("inner_iterations", C.c_int32),
                ("converged", C.c_int32), ("max_rel_residual", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LoglikInfo(C.Structure):
    _fields_ = [("loglik_stderr", C.c_double), ("logdet_prior", C.c_double), ("logdet_post", C.c_double),
                ("lanczos_steps", C.c_int32), ("lanczos_converged", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GmrfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libgmrf.so (built in-tree by paper_2503_08343_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libgmrf.so not built at {path}: run __graft_entry__.build() first")
        _build.build()
    lib = C.CDLL(path)
    P, I32, I64, U64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    DP = C.POINTER(C.c_double)
    sig = {
        "gmrf_default_opts": (None, [C.POINTER(SolveOpts)]),
        "gmrf_build_prior": (I32, [C.POINTER(PriorDesc), P, C.POINTER(P)]),
        "gmrf_condition": (I32, [P, C.POINTER(ObsDesc), C.POINTER(P)]),
        "gmrf_update_data": (I32, [P, P]),
        "gmrf_solve_mean": (I32, [P, P, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
        "gmrf_reserve": (I32, [P, I32, C.POINTER(SolveOpts)]),
        "gmrf_sample": (I32, [P, I32, U64, P, P, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
        "gmrf_marginal_var": (I32, [P, I32, U64, P, P, P, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
        "gmrf_gauss_newton_step": (I32, [P, P, P, DP, DP, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
        "gmrf_loglik_grad": (I32, [P, I32, U64, DP, DP, DP, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
        "gmrf_loglik_grad_ex": (I32, [P, I32, U64, I32, DP, C.POINTER(LoglikInfo), DP, DP, C.POINTER(SolveOpts),
                                      C.POINTER(SolveInfo)]),
        "gmrf_apply_posterior": (I32, [P, I32, P, P]),
        "gmrf_marginal_var_batch": (I32, [C.POINTER(P), I32, I32, U64, C.POINTER(P), C.POINTER(P),
                                          C.POINTER(SolveOpts), C.POINTER(SolveInfo), I32]),
        "gmrf_normals": (I32, [U64, I32, I32, I32, I64, P]),
        "gmrf_time_stencil": (I32, [P, I32, I32, I32, DP]),
        "gmrf_stencil_step": (I32, [P, I32, I32, I32, I32, P, P, P, D, D, D, P, P, DP]),
        "gmrf_level_info": (I32, [P, I32, C.POINTER(C.c_int32), DP]),
        "gmrf_prior_logdet": (I32, [C.POINTER(PriorDesc), DP, DP]),
        "gmrf_transfer_info": (I32, [P, C.POINTER(C.c_int32), DP]),
        "gmrf_test_set_wait_cap": (None, [I32]),
        "gmrf_launch_count": (U64, []),
        "gmrf_autotune_mode": (I32, [I32]),
        "gmrf_autotune_log": (I64, [C.c_char_p, I64]),
        "gmrf_num_unknowns": (I64, [P]),
        "gmrf_num_levels": (I32, [P]),
        "gmrf_prior_destroy": (None, [P]),
        "gmrf_posterior_destroy": (None, [P]),
        "gmrf_status_string": (C.c_char_p, [I32]),
        "gmrf_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st):
    if st != 0:
        raise GmrfError(st, load().gmrf_last_error().decode())


def _ptr(a):
    """Raw pointer of a float64 numpy array or CUDA tensor (or None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        assert a.dtype == torch.float64 and a.is_contiguous(), "tensors must be contiguous float64"
        return C.c_void_p(a.data_ptr())
    assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return C.c_void_p(a.ctypes.data)


def _dptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def default_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    load().gmrf_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def prior_desc(prior: dict) -> PriorDesc:
    d = PriorDesc()
    d.kind = KIND[prior["kind"]]
    d.nx, d.ny, d.nt = (int(v) for v in prior["n"])
    for i in range(3):
        d.lo[i] = float(prior["lo"][i])
        d.hi[i] = float(prior["hi"][i])
    for k in ("kappa", "tau", "nu", "cx", "cy", "kappa0", "eps2"):
        setattr(d, k, float(prior[k]))
    d.bc = {"dirichlet": 0, "periodic": 1}[prior.get("bc", "dirichlet")]
    d.noise_kappa = float(prior.get("noise_kappa", 0.0))
    d.decay = float(prior.get("decay", 0.0))
    return d


def prior_logdet(prior: dict):
    """Exact log det Q and 1/2 tr(Q^-1 dQ/dtheta) for theta = (log kappa,
    log tau, c, nu) of a prior (host computation, gmrf_prior_logdet)."""
    d = prior_desc(prior)
    ld = C.c_double()
    tr = np.zeros(4)
    _check(load().gmrf_prior_logdet(C.byref(d), C.byref(ld), _dptr(tr)))
    return ld.value, tr


class Prior:
    def __init__(self, prior: dict, stream=None):
        lib = load()
        self._desc = prior_desc(prior)
        self.spec = prior
        h = C.c_void_p()
        s = C.c_void_p(stream.cuda_stream if stream is not None else 0)
        _check(lib.gmrf_build_prior(C.byref(self._desc), s, C.byref(h)))
        self.h = h

    @property
    def N(self) -> int:
        return int(load().gmrf_num_unknowns(self.h))

    @property
    def levels(self) -> int:
        return int(load().gmrf_num_levels(self.h))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gmrf_prior_destroy(self.h)
            self.h = None


class Posterior:
    def __init__(self, prior: Prior, obs: dict):
        lib = load()
        self.prior = prior
        self._keep = []
        o = ObsDesc()
        coords = np.ascontiguousarray(obs["coords"], dtype=np.float64)
        y = np.ascontiguousarray(obs["y"], dtype=np.float64)
        sigma = np.ascontiguousarray(obs["sigma"], dtype=np.float64)
        o.m = len(y)
        o.coords, o.y, o.sigma = _dptr(coords), _dptr(y), _dptr(sigma)
        self._keep += [coords, y, sigma]
        if obs.get("ic_sigma") is not None:
            o.ic = 1
            o.ic_sigma = float(obs["ic_sigma"])
            if obs.get("ic_values") is not None:
                icv = np.ascontiguousarray(obs["ic_values"], dtype=np.float64)
                self._keep.append(icv)
                o.ic_values = _dptr(icv)
        if obs.get("colloc_sigma") is not None:
            o.colloc = 1 if obs.get("colloc_c") is not None else 2
            if obs.get("colloc_form", "collocation") == "fem_cn":
                o.colloc += 2          # FEM Crank-Nicolson rows: 3 linear, 4 Burgers
            o.colloc_stride_x, o.colloc_stride_t = (int(v) for v in obs.get("colloc_stride", (1, 1)))
            o.colloc_sigma = float(obs["colloc_sigma"])
            o.colloc_c = float(obs.get("colloc_c") or 0.0)
            o.colloc_nu = float(obs.get("burgers_nu", prior.spec["nu"]))
            if obs.get("colloc_f") is not None:
                f = np.ascontiguousarray(obs["colloc_f"], dtype=np.float64)
                self._keep.append(f)
                o.colloc_f = _dptr(f)
        h = C.c_void_p()
        _check(lib.gmrf_condition(prior.h, C.byref(o), C.byref(h)))
        self.h = h
        self.m = len(y)

    @property
    def N(self) -> int:
        return self.prior.N

    def update_data(self, y):
        _check(load().gmrf_update_data(self.h, _ptr(y)))

    def reserve(self, nrhs, opts=None):
        """Pre-creates the scratch and graphs of a batch of nrhs right-hand
        sides (gmrf_reserve)."""
        _check(load().gmrf_reserve(self.h, nrhs, C.byref(opts or default_opts())))

    def solve_mean(self, out=None, opts=None):
        out = np.empty(self.N) if out is None else out
        info = SolveInfo()
        _check(load().gmrf_solve_mean(self.h, _ptr(out), C.byref(opts or default_opts()), C.byref(info)))
        return out, info.as_dict()

    def sample(self, ns, seed, mean=True, out=None, mean_out=None, opts=None):
        x = np.empty((ns, self.N)) if out is None else out
        mu = (np.empty(self.N) if mean_out is None else mean_out) if mean else None
        info = SolveInfo()
        _check(load().gmrf_sample(self.h, ns, seed, _ptr(mu), _ptr(x), C.byref(opts or default_opts()), C.byref(info)))
        return mu, x, info.as_dict()

    def marginal_var(self, ns, seed, mean=True, stderr=True, out=None, opts=None):
        var = np.empty(self.N) if out is None else out
        mu = np.empty(self.N) if mean else None
        se = np.empty(self.N) if stderr else None
        info = SolveInfo()
        _check(load().gmrf_marginal_var(self.h, ns, seed, _ptr(mu), _ptr(var), _ptr(se),
                                        C.byref(opts or default_opts()), C.byref(info)))
        return mu, var, se, info.as_dict()

    def gauss_newton_step(self, mu_k, delta_prev, opts=None):
        dec = C.c_double()
        alpha = C.c_double()
        info = SolveInfo()
        _check(load().gmrf_gauss_newton_step(self.h, _ptr(mu_k), _ptr(delta_prev), C.byref(dec), C.byref(alpha),
                                             C.byref(opts or default_opts()), C.byref(info)))
        return dec.value, alpha.value, info.as_dict()

    def loglik_grad(self, nprobes, seed, opts=None, value=True, max_lanczos=0):
        """(log marginal likelihood or None, gradient [5], gradient stderr [5],
        solve info); info["loglik"] holds the value's standard error and the
        log-determinant parts (gmrf_loglik_grad_ex).  value=False skips the
        Lanczos quadrature of the value."""
        ll = C.c_double()
        li = LoglikInfo()
        g = np.zeros(5)
        se = np.zeros(5)
        info = SolveInfo()
        _check(load().gmrf_loglik_grad_ex(self.h, nprobes, seed, max_lanczos, C.byref(ll) if value else None,
                                          C.byref(li) if value else None, _dptr(g), _dptr(se),
                                          C.byref(opts or default_opts()), C.byref(info)))
        d = info.as_dict()
        if value:
            d["loglik"] = li.as_dict()
        return (ll.value if value else None), g, se, d

    def apply(self, x):
        x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
        y = np.empty_like(x)
        _check(load().gmrf_apply_posterior(self.h, x.shape[0], _ptr(x), _ptr(y)))
        return y

    def stencil_step(self, mode, x=None, b=None, d=None, level=0, precision=0, c0=0.0, c1=0.0, c2=0.0):
        """One launch of the fused stencil kernel (gmrf_stencil_step): mode 0
        apply, 1 residual, 2 Chebyshev step, 3 Chebyshev from zero, 4 PCG
        iteration (x previous direction, b iterate, d preconditioned residual,
        c1 alpha, c2 beta), 5 the solve's preconditioner z = M b (level 0);
        inputs [k][N_level].  Returns (out, out2 or None, dots), and for mode 4
        (q, p', dots, updated iterate)."""
        ref = next(v for v in (x, b) if v is not None)
        k, n = np.atleast_2d(ref).shape
        prep = lambda v: None if v is None else np.ascontiguousarray(np.atleast_2d(v), dtype=np.float64)
        x, b, d = prep(x), prep(b), prep(d)
        out = np.empty((k, n))
        out2 = np.empty((2 * k if mode == 4 else k, n)) if 2 <= mode <= 4 else None
        dots = np.empty(k)
        _check(load().gmrf_stencil_step(self.h, level, precision, mode, k, _ptr(x), _ptr(b), _ptr(d),
                                        c0, c1, c2, _ptr(out), _ptr(out2), _dptr(dots)))
        if mode == 4:
            return out, out2[:k], dots, out2[k:]
        return out, out2, dots

    def level_info(self):
        """[(nx, ny, nt, chebyshev lambda_max bound)] from finest to coarsest."""
        out = []
        for l in range(self.prior.levels):
            dims = (C.c_int32 * 3)()
            lm = C.c_double()
            _check(load().gmrf_level_info(self.h, l, dims, C.byref(lm)))
            out.append((dims[0], dims[1], dims[2], lm.value))
        return out

    def transfer_info(self):
        """(True for P1 space-plane grid transfers / False for bilinear,
        largest observation share of a fine-level diagonal entry)."""
        p1 = C.c_int32()
        share = C.c_double()
        _check(load().gmrf_transfer_info(self.h, C.byref(p1), C.byref(share)))
        return bool(p1.value), share.value

    def time_stencil(self, kernel, k, iters=20) -> float:
        """kernel: 0 apply, 1 residual, 2 Chebyshev step (finest level, FP32)."""
        ms = C.c_double()
        _check(load().gmrf_time_stencil(self.h, kernel, k, iters, C.byref(ms)))
        return ms.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gmrf_posterior_destroy(self.h)
            self.h = None


def marginal_var_batch(posts, ns, seed, means=True, opts=None, nthreads=1):
    """gmrf_marginal_var over independent posteriors, concurrently across
    priors (posteriors of one prior run in list order); instance i uses
    seed + i.  Returns (means, vars, infos)."""
    k = len(posts)
    vs = [np.empty(p.N) for p in posts]
    ms = [np.empty(p.N) for p in posts] if means else None
    hp = (C.c_void_p * k)(*[p.h.value for p in posts])
    vp = (C.c_void_p * k)(*[v.ctypes.data for v in vs])
    mp = (C.c_void_p * k)(*[m.ctypes.data for m in ms]) if means else None
    infos = (SolveInfo * k)()
    _check(load().gmrf_marginal_var_batch(hp, k, ns, seed, mp, vp, C.byref(opts or default_opts()), infos, nthreads))
    return ms, vs, [i.as_dict() for i in infos]


def autotune_mode(mode=None) -> int:
    """Launch-shape autotuner: sets the mode (0 off, 1 on) and returns the
    previous one; with no argument only returns the current mode."""
    return int(load().gmrf_autotune_mode(-1 if mode is None else int(mode)))


def autotune_log() -> list[dict]:
    """Every launch shape the autotuner has chosen in this process: key,
    CTAs per SM, time-chunk multiplier, milliseconds per candidate."""
    import json
    lib = load()
    n = lib.gmrf_autotune_log(None, 0)
    if n < 0:
        raise RuntimeError("gmrf_autotune_log failed")
    buf = C.create_string_buffer(n + 1)
    lib.gmrf_autotune_log(buf, n + 1)
    return [json.loads(line) for line in buf.value.decode().splitlines() if line.strip()]


def normals(seed, stream, sample0, count, n):
    out = np.empty((count, n))
    _check(load().gmrf_normals(seed, stream, sample0, count, n, _ptr(out)))
    return out


# ---------------------------------------------------------------------------
# Log marginal likelihood as a differentiable torch function of the
# hyper-parameters theta = (log kappa, log tau, log sigma_obs, c, nu).

HYPER = ("log_kappa", "log_tau", "log_sigma", "c", "nu")


def with_hyper(prior: dict, obs: dict, theta) -> tuple[dict, dict]:
    """Copies of (prior, obs) at hyper-parameters theta (sequence in HYPER
    order).  kappa is the initial-block kappa0 of the space-time priors,
    sigma_obs is one noise level for all point observations and c the x
    velocity; the Matern kind ignores c and nu."""
    lk, lt, ls, c, nu = (float(v) for v in theta)
    pr, ob = dict(prior), dict(obs)
    pr["kappa"] = float(np.exp(lk))
    if pr["kind"].startswith("advdiff_st"):
        pr["kappa0"] = pr["kappa"]
    pr["tau"] = float(np.exp(lt))
    pr["cx"], pr["nu"] = c, nu
    ob["sigma"] = np.full(len(obs["y"]), float(np.exp(ls)))
    return pr, ob


def hyper_of(prior: dict, obs: dict) -> np.ndarray:
    """theta of (prior, obs) in HYPER order (inverse of with_hyper)."""
    k = prior["kappa0"] if prior["kind"].startswith("advdiff_st") else prior["kappa"]
    return np.array([np.log(k), np.log(prior["tau"]), np.log(float(np.asarray(obs["sigma"])[0])),
                     prior.get("cx", 0.0), prior.get("nu", 0.0)])


def _loglik_function():
    import torch

    class LogMarginalLikelihood(torch.autograd.Function):
        """Forward: the log marginal likelihood at theta (exact prior log
        determinant, Lanczos-quadrature estimate of the posterior one; its
        standard error is in ctx.info).  Backward: its gradient, with the
        posterior trace terms estimated by Hutchinson probes from the same
        batched solve and the prior trace terms exact (gmrf_loglik_grad_ex);
        no graph through the solver is recorded."""

        @staticmethod
        def forward(ctx, theta, prior, obs, nprobes, seed, opts):
            pr, ob = with_hyper(prior, obs, theta.detach().cpu().tolist())
            post = Posterior(Prior(pr), ob)
            ll, g, se, info = post.loglik_grad(nprobes, seed, opts=opts)
            ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
            ctx.info = dict(info, grad_stderr=se.tolist())
            return theta.new_tensor(ll)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g, None, None, None, None, None

    return LogMarginalLikelihood


_LOGLIK = None


def log_marginal_likelihood(theta, prior: dict, obs: dict, nprobes: int = 32, seed: int = 0, opts=None):
    """Differentiable in theta (a float64 torch tensor of 5 entries in HYPER
    order); see LogMarginalLikelihood for what the value and the gradient are."""
    global _LOGLIK
    if _LOGLIK is None:
        _LOGLIK = _loglik_function()
    return _LOGLIK.apply(theta, prior, obs, nprobes, seed, opts)
