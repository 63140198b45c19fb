/*
 * gmrf.h -- C ABI of the GB300 GMRF probabilistic PDE solver.
 *
 * Conditions an SPDE-discretised Gaussian Markov random field prior
 * u ~ N(0, Q^-1) (P1 FEM in space, implicit Euler in time, lumped mass) on
 * noisy point data and on linear or linearised PDE collocation, then
 * computes posterior means, perturbation samples, marginal variances,
 * Gauss-Newton steps and log-likelihood gradients.  The posterior precision
 * Q_u|y = Q + A^T Q_eps A (Sec. 3.1, eq. posterior-mean) is applied
 * matrix-free by fused stencil kernels and solved by multi-RHS conjugate
 * gradients preconditioned by a geometric multigrid V-cycle, with FP32 inner
 * iterations inside FP64 iterative refinement.
 *
 * Conventions for every entry point:
 *  - Nothing aborts or prints.  A non-zero gmrf_status is returned and
 *    gmrf_last_error() (thread-local) describes it.
 *  - Work is ordered on the stream given to gmrf_build_prior; every call
 *    returns after that stream has finished the call's work (scalars and
 *    host outputs are valid on return).
 *  - Array outputs are caller-owned.  A pointer may be host memory or device
 *    memory (detected with cudaPointerGetAttributes); host buffers are
 *    copied inside the call.  Device pointers must be on the handle's device.
 *  - Vectors over the unknowns are ordered lexicographically,
 *    index ((t * ny + y) * nx + x), FP64.  Batches of vectors are
 *    [count][N], row-major.
 *  - Handles may be destroyed in any order: a prior stays alive until its
 *    own handle and every posterior built on it are destroyed.
 *  - Handles own all device scratch.  Scratch for a batch of k right-hand
 *    sides is allocated at the first call that needs k (or by gmrf_reserve)
 *    and reused after.
 *  - The first call in a process that draws normals (gmrf_sample,
 *    gmrf_marginal_var, gmrf_normals, gmrf_condition's eigenvalue bound)
 *    fills a 6 KB device table of the Box-Muller transform: one kernel and a
 *    device synchronisation, once.  The library drives one GPU per process.
 */
#ifndef GMRF_H
#define GMRF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gmrf_status {
    GMRF_OK = 0,
    GMRF_E_INVALID = 1,        /* bad argument or descriptor */
    GMRF_E_NOT_SPD = 2,        /* CG breakdown: p^T Q p <= 0 or non-finite */
    GMRF_E_NO_CONVERGENCE = 3, /* iteration caps reached; info holds the residual */
    GMRF_E_CUDA = 4,           /* a CUDA runtime call failed */
    GMRF_E_OOM = 5,            /* device allocation failed */
    GMRF_E_TIMEOUT = 6         /* wall-clock limit of gmrf_solve_opts reached */
} gmrf_status;

/* Prior families (Sec. 2.2, 2.3, 2.4 and App. A):
 *  GMRF_MATERN2_2D        (kappa^2 - Lap) u = W / tau on [lo, hi]^2, alpha = 2:
 *                         Q = tau^2 K Ml^-1 K, K = kappa^2 Ml + S.
 *  GMRF_STEADY_ADVDIFF_2D Q = tau^2 K^T Ml^-1 K, K = kappa^2 Ml + nu S + cx Bx + cy By.
 *  GMRF_ADVDIFF_ST_1D     u_t + c u_x - nu u_xx = tau W on [x0,x1] x [0,T]
 *  GMRF_ADVDIFF_ST_2D     u_t + c . grad u - nu Lap u = tau W on [lo,hi]^2 x [0,T]:
 *                         implicit Euler (App. A): G u^k = Ml u^(k-1) + w,
 *                         G = Ml + dt (nu S + B_c), w ~ N(0, tau^2 dt Ml); the
 *                         initial level is a unit-variance Matern (kappa0).
 * Every prior is applied in the stacked form Q = B^T B with B a short stencil.
 * Boundary (gmrf_prior_desc.bc):
 *  GMRF_BC_DIRICHLET  boundary nodes carry a homogeneous Dirichlet condition
 *                     (App. B, N_k = 0): decoupled, variance eps2.
 *  GMRF_BC_PERIODIC   spatial kinds (GMRF_MATERN2_2D, GMRF_STEADY_ADVDIFF_2D)
 *                     only: App. B with N_k = 1, c_1 = 1, h(1) = mirror(k),
 *                     in its hard limit.  The nodes on x = hi and y = hi are
 *                     the nodes on x = lo and y = lo; columns and rows of the
 *                     constrained nodes are added to those of their mirrors
 *                     (test and trial functions periodic), so the unknowns
 *                     are the (nx - 1) x (ny - 1) nodes of the torus, node
 *                     (i, j) at (lo + i h_x, lo + j h_y), h = (hi - lo) / (n - 1).
 *                     Every field the library reads or writes has that size.
 *                     The multigrid hierarchy halves nx - 1 and ny - 1 while
 *                     they are even and at least 8; a coarsest level above
 *                     1024 unknowns is rejected (GMRF_E_INVALID). */
typedef enum gmrf_prior_kind {
    GMRF_MATERN2_2D = 0,
    GMRF_ADVDIFF_ST_1D = 1,
    GMRF_ADVDIFF_ST_2D = 2,
    GMRF_STEADY_ADVDIFF_2D = 3
} gmrf_prior_kind;

typedef enum gmrf_boundary {
    GMRF_BC_DIRICHLET = 0,
    GMRF_BC_PERIODIC = 1
} gmrf_boundary;

typedef struct gmrf_prior_desc {
    int32_t kind;              /* gmrf_prior_kind */
    int32_t nx, ny, nt;        /* nodes per axis incl. boundary; ny = 1 in 1D space, nt = 1 if spatial */
    double lo[3], hi[3];       /* domain corners (x, y, t) */
    double kappa;              /* Matern / steady: inverse range; space-time: unused */
    double tau;                /* scale: Matern/steady Q ~ tau^2, space-time Q ~ tau^-2 */
    double nu;                 /* diffusion (Matern: 1) */
    double cx, cy;             /* advection velocity */
    double kappa0;             /* space-time: Matern kappa of the initial level */
    double eps2;               /* Dirichlet boundary variance (App. B "M_kk = eps^2") */
    int32_t bc;                /* gmrf_boundary (0: Dirichlet) */
    /* Space-time priors (App. A): transition G u^k = (1 - decay) Ml u^(k-1) + w.
     * noise_kappa > 0 (GMRF_ADVDIFF_ST_1D only): the spatial noise W_s is the
     * unit-variance alpha = 2 Matern field of inverse range noise_kappa
     * (Dirichlet on the same boundary), so w ~ N(0, tau^2 dt Ml Sigma_s Ml),
     * Sigma_s^-1 = tau_s^2 K_s Ml^-1 K_s, K_s = noise_kappa^2 Ml + S; B's
     * transition rows become T_K B_w, T_K = tau_s Ml^-1/2 K_s Ml^-1/2 on the
     * interior.  noise_kappa = 0: white spatial noise, w ~ N(0, tau^2 dt Ml).
     * decay in [0, 1) (both space-time kinds): an AR(1) in time (0: none). */
    double noise_kappa;
    double decay;
} gmrf_prior_desc;

/* Observations (Sec. 3.1).  All pointers are host memory, read during the call.
 *  point data: y_k = phi(x_k) . u + e_k, e_k ~ N(0, sigma_k^2), with P1
 *    barycentric weights in space times linear weights in time; coords are
 *    [m][d], d = 2 (x, y) for spatial priors, 2 (x, t) for 1D space-time,
 *    3 (x, y, t) for 2D space-time.
 *  ic: the initial condition as data at every t = 0 node, values ic_values
 *    [nx * ny] (NULL: -sin(pi x)), noise ic_sigma.
 *  colloc: 1 = linear advection-diffusion residual with speed colloc_c and
 *    right-hand side colloc_f (NULL: 0) at interior nodes of levels k >= 1;
 *    3, 4 = the same rows as 1, 2 in FEM form (Sec. 3.1, A_ij =
 *    int phi_i D phi_j, exact integrals of the P1 interpolant, consistent
 *    mass) with Crank-Nicolson in time (Sec. 5: FEM observations in
 *    Crank-Nicolson form on an implicit-Euler prior): row (x, k) is
 *    int phi_x (u^k - u^(k-1))/dt + 1/2 sum over levels k, k-1 of
 *    (int phi_x a u_x + nu int phi_x' u_x), a = colloc_c (3) or a = u (4,
 *    Burgers, linearised like 2); colloc_f gives int phi_x f per row (3).
 *    2 = Burgers residual (Sec. 3.3), linearised at the point given to
 *    gmrf_gauss_newton_step.  Diffusion colloc_nu, noise colloc_sigma.
 *    Defined for GMRF_ADVDIFF_ST_1D only. */
typedef struct gmrf_obs_desc {
    int64_t m;
    const double* coords;
    const double* y;
    const double* sigma;       /* [m], or NULL to use sigma_all */
    double sigma_all;
    int32_t ic;
    double ic_sigma;
    const double* ic_values;
    int32_t colloc;
    double colloc_sigma;
    double colloc_c;
    double colloc_nu;
    const double* colloc_f;
    /* collocation points: only the rows with x % colloc_stride_x == 0 and
     * k % colloc_stride_t == 0 observe the PDE (0 or 1: every row); the
     * others keep their row index (random draws) with zero weight */
    int32_t colloc_stride_x;
    int32_t colloc_stride_t;
} gmrf_obs_desc;

typedef struct gmrf_solve_opts {
    double rtol;               /* per-RHS FP64 residual target ||b - Q_u|y x||_D / ||b - Q_u|y x0||_D,
                                  ||v||_D^2 = sum_i v_i^2 / (Q_u|y)_ii (default 1e-10) */
    int32_t max_refine;        /* FP64 refinement steps (default 12) */
    int32_t max_inner;         /* inner PCG iterations per refinement step; 0 (default): 60 with the
                                  multigrid preconditioner, 200 with the time-stepping one */
    double inner_rtol;         /* inner reduction of the preconditioned residual norm (default 1e-5) */
    int32_t precision;         /* 0: FP32 inner + FP64 refinement; 1: plain FP64 PCG.  1D space-time
                                  posteriors whose time-stepping preconditioner mixes PDE rows with the
                                  prior's rows (collocation points on a coarser grid than the mesh, or
                                  no observed initial condition) always take 1: FP32 cannot resolve
                                  their weights (1 / colloc_sigma^2 against one) */
    int32_t batched;           /* 1: all right-hand sides in one batch; 0: one at a time */
    double timeout_s;          /* wall-clock limit, 0 = none */
} gmrf_solve_opts;

typedef struct gmrf_solve_info {
    int32_t nrhs;
    int32_t refinements;       /* FP64 residual evaluations */
    int32_t inner_iterations;  /* total PCG iterations (batched: per batch) */
    int32_t converged;         /* 1 if every RHS reached rtol */
    double max_rel_residual;   /* max over RHS of the final FP64 relative residual (D-weighted) */
    double seconds;
} gmrf_solve_info;

typedef struct gmrf_prior gmrf_prior;          /* opaque, library-owned */
typedef struct gmrf_posterior gmrf_posterior;  /* opaque, library-owned */

/* Fill opts with the defaults listed above. */
void gmrf_default_opts(gmrf_solve_opts* opts);

/* Builds the stencil description of Q = B^T B on every multigrid level
 * (Sec. 2.2 eq. sparse-prec-matrix; App. A eq. block-tridiag-prec; App. B).
 * stream: a cudaStream_t other than the legacy default stream, used for all
 * work of this prior and its posteriors; NULL: the handle creates and owns a
 * non-blocking stream.  *out receives the handle. */
gmrf_status gmrf_build_prior(const gmrf_prior_desc* desc, void* stream, gmrf_prior** out);

/* Conditions the prior on observations: builds the observation lists on every
 * level and the right-hand side A^T Q_eps y (Sec. 3.1).  The prior must
 * outlive the posterior. */
gmrf_status gmrf_condition(gmrf_prior* prior, const gmrf_obs_desc* obs, gmrf_posterior** out);

/* Replaces the point-data values y (length m of the descriptor; host or
 * device memory) without rebuilding the observation operator. */
gmrf_status gmrf_update_data(gmrf_posterior* post, const double* y);

/* Creates the device scratch and CUDA graphs of a batch of nrhs right-hand
 * sides (the mean and nrhs - 1 samples) for the options opts (precision,
 * batched; NULL: defaults) by running that batch once (results discarded).
 * Later calls of gmrf_solve_mean (nrhs = 1), gmrf_sample and
 * gmrf_marginal_var with the same batch size and options allocate no device
 * memory, so they can run where allocation is unwelcome (inside a memory
 * budget, next to other work).  The paper has no counterpart: it is serving
 * plumbing. */
gmrf_status gmrf_reserve(gmrf_posterior* post, int32_t nrhs, const gmrf_solve_opts* opts);

/* Posterior mean mu = Q_u|y^-1 A^T Q_eps y (eq. posterior-mean, prior mean 0).
 * mu: [N]. */
gmrf_status gmrf_solve_mean(gmrf_posterior* post, double* mu, const gmrf_solve_opts* opts,
                            gmrf_solve_info* info);

/* Perturbation samples x_s = Q_u|y^-1 L z_s ~ N(0, Q_u|y^-1) (Sec. 3.2) with
 * the left root L = [B^T, A^T Q_eps^1/2] and z_s from Philox4x32-10 keyed by
 * seed (sample s uses counter words (j, s, stream, 0)).  x: [ns][N]
 * zero-mean perturbations.  mean: [N] or NULL; when given, the posterior mean
 * is solved in the same batch. */
gmrf_status gmrf_sample(gmrf_posterior* post, int32_t ns, uint64_t seed, double* mean, double* x,
                        const gmrf_solve_opts* opts, gmrf_solve_info* info);

/* Rao-Blackwellised Monte Carlo marginal variances (Sec. 3.2; Siden et al.
 * 2018) from ns perturbation samples:
 * var_i = 1/Q_ii + (1/ns) sum_s (sum_{j != i} Q_ij x_s,j / Q_ii)^2.
 * var: [N]; stderr_: [N] or NULL (standard error of the Monte Carlo term);
 * mean: [N] or NULL (posterior mean solved in the same batch). */
gmrf_status gmrf_marginal_var(gmrf_posterior* post, int32_t ns, uint64_t seed, double* mean,
                              double* var, double* stderr_, const gmrf_solve_opts* opts,
                              gmrf_solve_info* info);

/* Batched serving of independent posteriors (not in the paper, which solves
 * one problem at a time; a serving workload of many uneven instances):
 * gmrf_marginal_var for
 * posts[0..count), instance i with seed + i, means[i] (NULL array or NULL
 * entry: no mean) and vars[i] (non-NULL, [N_i]) outputs as in
 * gmrf_marginal_var.  Instances whose posteriors share a prior handle run in
 * list order on that prior's stream.  nthreads <= 1 with the FP32
 * refinement path (precision 0, batched, no timeout): one host thread
 * enqueues every instance (each solve is one CUDA graph whose refinement and
 * PCG loops run on the device, so nothing is waited for until all are
 * enqueued), then collects them; instances of different priors run
 * concurrently on their streams.  nthreads > 1 (or other options): instances
 * of different priors run from min(nthreads, number of priors) host threads.
 * Results equal those of calling gmrf_marginal_var on each instance alone.
 * No posterior or prior in the list may be used elsewhere during the call.
 * infos: [count] or NULL.  Returns GMRF_E_INVALID for a NULL entry before any
 * work, else the status of the first instance in list order that failed
 * (gmrf_last_error names it); the other instances still complete. */
gmrf_status gmrf_marginal_var_batch(gmrf_posterior* const* posts, int32_t count, int32_t ns, uint64_t seed,
                                    double* const* means, double* const* vars, const gmrf_solve_opts* opts,
                                    gmrf_solve_info* infos, int32_t nthreads);

/* One Gauss-Newton step on -log pi(u) (Sec. 3.3, eq. nonlinear-mode) for
 * Burgers collocation: H = Q + J^T Q_eps J + A^T R^-1 A at mu_k, solve
 * H d = -grad, warm-started from delta_prev when that gives a smaller
 * starting residual than zero (the solve's rtol is relative to it), then Armijo backtracking
 * (halving from 1, c1 = 1e-4, at most 20 halvings).  mu_k [N] (in/out, host
 * or device), delta_prev [N] (in/out, may be all zero).  newton_decrement
 * (host) receives d^T H d, alpha (host, may be NULL) the step length. */
gmrf_status gmrf_gauss_newton_step(gmrf_posterior* post, double* mu_k, double* delta_prev,
                                   double* newton_decrement, double* alpha,
                                   const gmrf_solve_opts* opts, gmrf_solve_info* info);

/* Log marginal likelihood l = log N(y; 0, A Q^-1 A^T + R) of the point
 * data and its gradient with respect to (log kappa, log tau, log sigma, cx,
 * nu) (not in the paper, which fixes its hyper-parameters; Gaussian
 * identities with b = A^T R^-1 y, mu = Q_u|y^-1 b):
 *   l = 1/2 log det Q - 1/2 log det Q_u|y - 1/2 log det R - 1/2 y^T R^-1 y
 *       + 1/2 b^T mu - (M/2) log 2 pi.
 * One batched solve of the posterior system for the mean and nprobes
 * Rademacher probes (Philox stream 2, seed).  The prior terms are exact
 * (log det Q and 1/2 tr(Q^-1 dQ), as gmrf_prior_logdet, computed on host
 * threads while the GPU solves and cached in the prior handle); the
 * posterior trace 1/2 tr(Q_u|y^-1 dQ_u|y) is the Hutchinson estimate over
 * the probes, log det Q_u|y the stochastic Lanczos quadrature estimate over
 * the same probes (Jacobi-scaled operator, at most max_lanczos steps, <= 0:
 * 400).  loglik (host, may be NULL: then no Lanczos run) receives l;
 * li (may be NULL) its standard error and parts; grad[5], grad_stderr[5]
 * (host; stderr of the Hutchinson part, the exact parts have none). */
typedef struct gmrf_loglik_info {
    double loglik_stderr;      /* standard error of loglik (half that of the log det Q_u|y estimate) */
    double logdet_prior;       /* log det Q, exact */
    double logdet_post;        /* estimate of log det Q_u|y */
    int32_t lanczos_steps;     /* Lanczos steps run for every probe */
    int32_t lanczos_converged; /* 1 if every probe's quadrature settled before max_lanczos */
} gmrf_loglik_info;

gmrf_status gmrf_loglik_grad_ex(gmrf_posterior* post, int32_t nprobes, uint64_t seed, int32_t max_lanczos,
                                double* loglik, gmrf_loglik_info* li, double* grad, double* grad_stderr,
                                const gmrf_solve_opts* opts, gmrf_solve_info* info);

/* gmrf_loglik_grad_ex with the default Lanczos cap and no gmrf_loglik_info. */
gmrf_status gmrf_loglik_grad(gmrf_posterior* post, int32_t nprobes, uint64_t seed, double* loglik,
                             double* grad, double* grad_stderr, const gmrf_solve_opts* opts,
                             gmrf_solve_info* info);

/* Exact log det Q of the prior and the prior trace terms of the
 * log-likelihood gradient, trace[p] = 1/2 tr(Q^-1 dQ/dtheta_p) for
 * theta = (log kappa, log tau, cx, nu) (kappa: kappa0 of the initial level
 * for space-time priors).  Not in the paper (hyper-parameter learning;
 * Gaussian identities).  Q = B^T B with B block lower bidiagonal in time, so
 * log det Q = 2 sum_k log|det B_kk| and 1/2 tr(Q^-1 dQ) = sum_k
 * tr(B_kk^-1 dB_kk) over the diagonal blocks: at most two distinct interior
 * operators (the spatial / initial block and the transition block), by the
 * sine-transform closed form when symmetric, else by banded LU and the band of
 * the inverse, O(N_s (n_x)^2) host work for N_s spatial nodes.  Runs on the
 * host only (no GPU, no handle).  logdet or trace may be NULL. */
gmrf_status gmrf_prior_logdet(const gmrf_prior_desc* desc, double* logdet, double* trace);

/* y = Q_u|y x in FP64 for a batch of k vectors x, y: [k][N].  Test hook for
 * the fused stencil.  GMRF_E_CUDA if a stencil CTA gave up its bounded wait
 * for a staged input tile. */
gmrf_status gmrf_apply_posterior(gmrf_posterior* post, int32_t k, const double* x, double* y);

/* Allocation-free y = Q_u|y x for one vector (FP64), with x^T Q_u|y x.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they need the product -- code running
 * inside a custom allocator or memory-pool callback, loops that must not take
 * cudaMalloc's implicit device synchronisation, processes whose device memory
 * is fully reserved by a pool.  It makes no cudaMalloc/cudaFree call and uses
 * no allocating library routine: its scratch is one fixed device array of
 * 16.1 MB inside the library, held by every GPU that loads the library until
 * the process exits.
 *  x, y: device memory, [N], N <= 262144 unknowns (a 512 x 512 grid); larger
 *        posteriors are rejected with GMRF_E_INVALID and a message naming the
 *        limit.  xQx: host or device, may be NULL.
 *  Set-up happens in gmrf_condition, on the posterior's device, for every
 *  posterior within the limit: it looks up the scratch address
 *  (cudaGetSymbolAddress), which loads the library module that holds the
 *  array, and loads the kernels this call launches.  The call itself then
 *  loads and allocates nothing.
 *  All calls share the one scratch array: calls that overlap on the GPU (other
 *  host threads, other streams) race and must be serialised by the caller.
 *  Runs on the posterior's stream and returns after it has finished.  If a
 *  stencil CTA gave up its bounded wait for a staged input tile, the call
 *  returns GMRF_E_CUDA (y and xQx are then incomplete). */
gmrf_status gmrf_apply_posterior_noalloc(gmrf_posterior* post, const double* x, double* y, double* xQx);

/* Normal draws of the sample stream: out[s][i] = z(seed, stream, sample0 + s, i)
 * for s < count, i < n.  Test hook for the in-kernel generator. */
gmrf_status gmrf_normals(uint64_t seed, int32_t stream, int32_t sample0, int32_t count, int64_t n,
                         double* out);

/* Average duration in milliseconds of one launch of the fused FP32 stencil
 * kernel on the finest level, over `iters` launches on the handle's stream
 * (CUDA events around the launches), for a batch of k right-hand sides of
 * random data.  kernel: 0 = apply (y = Q_u|y x), 1 = residual
 * (r = b - Q_u|y x), 2 = Chebyshev smoothing step
 * (d' = c1 d + c2 D^-1 (b - Q_u|y x), x' = x + d'), 3 = the conjugate-gradient
 * iteration's fused apply (p' = z + beta p, q = Q_u|y p', x += alpha p). */
gmrf_status gmrf_time_stencil(gmrf_posterior* post, int32_t kernel, int32_t k, int32_t iters, double* ms);

/* One launch of the fused stencil kernel on multigrid level `level`
 * (0 = finest) in FP32 (precision 0) or FP64 (1), for k right-hand sides.
 * Test hook for the kernel modes the solver uses (the FP32 ones only
 * precondition, so wrong arithmetic there would show as slower convergence,
 * not as wrong results).  Inputs x, b, d and outputs out, out2 are [k][N_l]
 * FP64, host or device (inputs are rounded to the kernel precision); N_l the
 * level's unknowns; D the diagonal of the level's operator Q_l:
 *  mode 0 apply:      out = Q_l x,                        dots = x^T out
 *  mode 1 residual:   out = b - Q_l x,                    dots = |out|^2
 *  mode 2 Chebyshev:  out2 = c1 d + c2 D^-1 (b - Q_l x),  out = x + out2,
 *                     dots = b^T out (d may be NULL: taken as 0)
 *  mode 3 Chebyshev from zero: x1 = c0 D^-1 b, then mode 2 with x = d = x1.
 *  mode 4 PCG (one conjugate-gradient iteration's vector work around the
 *                     apply): p' = d + c2 x (x the previous direction, d the
 *                     preconditioned residual, c2 = beta), out = Q_l p',
 *                     dots = p'^T out; out2 holds [2][k][N_l]: p', then the
 *                     iterate update b + c1 x (b the iterate, c1 = alpha).
 *  mode 5 preconditioner (level 0 only): out = M b with M the preconditioner
 *                     of the posterior's solves (a multigrid V-cycle, or the
 *                     time-stepping preconditioner J~^-1 W^-1 J~^-T where it
 *                     applies), dots = b^T out; x, d and out2 are unused.
 * dots: [k] host.  Allocates its own scratch. */
gmrf_status gmrf_stencil_step(gmrf_posterior* post, int32_t level, int32_t precision, int32_t mode, int32_t k,
                              const double* x, const double* b, const double* d, double c0, double c1, double c2,
                              double* out, double* out2, double* dots);

/* Test hook for the failure path of the stencil kernels: the number of
 * polls each CTA spends on a bounded wait for a staged input tile before it
 * gives up (0 restores the default, 2^22; a negative cap gives up without
 * polling, so every CTA fails its first wait).  A poll may itself block for
 * a short hardware-defined time.  A CTA that gives up records a device flag,
 * still waits (with the default cap) for its copies in flight, and returns;
 * the solver turns the flag into GMRF_E_CUDA and clears it, so the handle
 * stays usable.  Process-wide; not for production use. */
void gmrf_test_set_wait_cap(int32_t cap);

/* Number of kernels this library has launched in the process so far
 * (kernels inside replayed CUDA graphs included). */
uint64_t gmrf_launch_count(void);

/* Launch-shape autotuner of the persistent stencil kernels.  Nothing in the
 * method depends on the grid a persistent kernel runs on: it decides only
 * how the work units (tiles x right-hand-side blocks, and time chunks of the
 * marching space-time kernel) are shared among CTAs, and in which order the
 * per-CTA dot partials are summed.  The first launch of a kernel on a new
 * (instantiation, right-hand-side blocks, size bucket, observation-table
 * bucket) key times every candidate shape (CTAs per SM; time-chunk length)
 * on zero-filled scratch copies of its vectors, outside any graph capture,
 * and keeps the fastest for the rest of the process.  Environment:
 * GMRF_AUTOTUNE=0 disables measuring (default shapes); GMRF_AUTOTUNE_FILE
 * names a file the choices are read from at first use and appended to.
 *
 * gmrf_autotune_mode: mode 0 off, 1 on, negative only queries; returns the
 * mode before the call.  Process-wide.
 * gmrf_autotune_log: copies every recorded choice (one JSON object per line:
 * key, chosen CTAs per SM and time-chunk multiplier, measured milliseconds
 * per launch of each candidate) into buf (NUL-terminated, truncated to
 * cap - 1 bytes; buf may be NULL) and returns the full length in bytes, or
 * -1 on an internal error. */
int32_t gmrf_autotune_mode(int32_t mode);
int64_t gmrf_autotune_log(char* buf, int64_t cap);

/* Multigrid hierarchy of a posterior: grid dimensions (nx, ny, nt) of level
 * `level` (0 = finest) and the bound on the spectrum of D^-1 Q_u|y used by
 * its Chebyshev smoother (0 on the coarsest level, which is solved directly). */
gmrf_status gmrf_level_info(const gmrf_posterior* post, int32_t level, int32_t* dims, double* lmax);

/* Grid transfer of the multigrid hierarchy in the space plane: *p1 = 1 for
 * P1 interpolation on the triangulation (chosen when the observation rows
 * contribute at least half of some fine-level diagonal entry of Q_u|y),
 * 0 for bilinear; *data_share (may be NULL) receives that largest share.
 * Both transfers reduce to linear interpolation along a single axis. */
gmrf_status gmrf_transfer_info(const gmrf_posterior* post, int32_t* p1, double* data_share);

int64_t gmrf_num_unknowns(const gmrf_prior* prior);
int32_t gmrf_num_levels(const gmrf_prior* prior);
void gmrf_prior_destroy(gmrf_prior* prior);
void gmrf_posterior_destroy(gmrf_posterior* post);
const char* gmrf_status_string(gmrf_status s);
const char* gmrf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GMRF_H */
