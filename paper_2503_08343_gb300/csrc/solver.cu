// Multi-RHS multigrid-preconditioned conjugate gradients inside FP64
// iterative refinement (CG: Sec. 3.2 "Conjugate gradient method").
//
// Outer loop (FP64): r = b - Q_u|y x with the FP64 stencil, per-RHS norms,
// stop at ||r|| <= rtol ||b||.  Inner solve (FP32): PCG on r / ||r|| to a
// relative reduction inner_rtol, preconditioned by one V(2,2)-cycle with a
// Chebyshev(2) smoother on D^-1 Q (D the diagonal of Q_u|y) over levels
// rediscretised on coarser grids, and a dense inverse on the coarsest level.
// One PCG iteration is captured into a CUDA graph and replayed.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "autotune.h"
#include "host.h"

namespace gmrf {

struct Cheb {
    double c1[2], c2[2];
};

// Chebyshev iteration on [lmax/10, lmax]: x <- x + d_k, d_0 = r/theta,
// d_k = rho_k rho_(k-1) d_(k-1) + (2 rho_k / delta) r, rho_k = 1/(2 sigma - rho_(k-1)).
static Cheb cheb_coeffs(double lmax) {
    const double lmin = lmax / 10.0;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    const double sigma = theta / delta, rho0 = 1.0 / sigma;
    const double rho1 = 1.0 / (2.0 * sigma - rho0);
    Cheb c;
    c.c1[0] = 0.0;
    c.c2[0] = 1.0 / theta;
    c.c1[1] = rho1 * rho0;
    c.c2[1] = 2.0 * rho1 / delta;
    return c;
}

template <typename T> static const T* dinv_of(const Level& L);
template <> const float* dinv_of<float>(const Level& L) { return L.d_dinv32; }
template <> const double* dinv_of<double>(const Level& L) { return L.d_dinv64; }
template <typename T> static const T* dense_of(const Level& L);
template <> const float* dense_of<float>(const Level& L) { return L.d_dense32; }
template <> const double* dense_of<double>(const Level& L) { return L.d_dense64; }
template <typename T> static const T* pw_of(const Level& L, int a);
template <> const float* pw_of<float>(const Level& L, int a) { return L.d_pw[a]; }
template <> const double* pw_of<double>(const Level& L, int a) { return L.d_pwd[a]; }

void level_free(Level& L) {
    dev_free(L.d_obs); dev_free(L.d_tile_ptr); dev_free(L.d_tile_idx);
    dev_free(L.d_omap); dev_free(L.d_oent32); dev_free(L.d_oent64);
    dev_free(L.d_mu32); dev_free(L.d_mu64);
    dev_free(L.d_dinv32); dev_free(L.d_dinv64); dev_free(L.d_diag64);
    for (int a = 0; a < 3; ++a) {
        dev_free(L.d_pj[a]); dev_free(L.d_pw[a]); dev_free(L.d_pwd[a]); dev_free(L.d_rs[a]); dev_free(L.d_rc[a]);
    }
    dev_free(L.d_dense32); dev_free(L.d_dense64);
    dev_free(L.d_tsp32); dev_free(L.d_tsp64);
    dev_free(L.d_tspc32); dev_free(L.d_tspc64);
    L = Level();
}

static size_t partial_slots(const Posterior& P, int nblk) {
    long long m = 1;
    for (const Level& L : P.levels) m = std::max(m, std::max(L.ntiles(), (long long)elem_parts(L.N)));
    m = std::max<long long>(m, stencil_max_grid());
    return (size_t)m * nblk * 8;
}

// ---------------------------------------------------------------------------
// operator-dependent setup: Jacobi diagonal, Chebyshev bound, dense inverse

static double power_lmax(Posterior& P, Level& L, cudaStream_t s) {
    const long long N = L.N;
    float* v = dev_alloc<float>((size_t)N * 4);
    float* q = dev_alloc<float>((size_t)N * 4);
    const long long nt = L.ntiles();
    const int np = elem_parts(N);
    double* part = dev_alloc<double>((size_t)std::max<long long>(std::max<long long>(nt, np), stencil_max_grid()) * 4);
    double* red = dev_alloc<double>(4);
    // Start from D^-1/2 g: every node then carries the same weight in the
    // D-norm.  A plain normal start would be dominated by the Dirichlet rows
    // (D = 1/eps^2, eigenvalue exactly 1) and, when lambda_max is close to 1
    // (mass-dominated operators, kappa^2 h^2 >> nu), 24 steps could not lift
    // the interior modes above them.
    launch_fill_random(v, N, 0x5eed, s, L.d_dinv32);
    StencilArgs<float> a{};
    a.L = L.view<float>();
    a.x = v;
    a.out = q;
    a.nblk = 1;
    double lam = 0.0;
    double h[4];
    const int iters = 24;
    for (int it = 0; it < iters; ++it) {
        launch_stencil<float>(L.geo, M_APPLY, a, s);
        launch_power_scale(q, L.d_dinv32, N, part, np, s);
        launch_reduce(part, np, 1, red, s);
        launch_scale_comp(v, q, red, N, s);
        GCK(cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, s));
        GCK(cudaStreamSynchronize(s));
        if (it >= 2) {
            double m = 0.0;
            for (int c = 0; c < 4; ++c) m = std::max(m, std::sqrt(h[c]));
            lam = std::max(lam, m);
        }
    }
    dev_free(v); dev_free(q); dev_free(part); dev_free(red);
    (void)P;
    return lam;
}

// Jacobi diagonal of level L; with share != nullptr also the largest share of
// a node's diagonal that the observation rows contribute (dinv64 holds the
// prior diagonal until the final step overwrites it).
static void setup_diag(Level& L, cudaStream_t s, double* share = nullptr) {
    if (!L.d_diag64) L.d_diag64 = dev_alloc<double>((size_t)L.N);
    if (!L.d_dinv32) L.d_dinv32 = dev_alloc<float>((size_t)L.N);
    if (!L.d_dinv64) L.d_dinv64 = dev_alloc<double>((size_t)L.N);
    launch_diag<double>(L.geo, L.view<double>(), L.d_diag64, s);
    unsigned long long* d_share = nullptr;
    if (share) {
        d_share = dev_alloc<unsigned long long>(1);
        GCK(cudaMemsetAsync(d_share, 0, sizeof(unsigned long long), s));
        GCK(cudaMemcpyAsync(L.d_dinv64, L.d_diag64, (size_t)L.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    launch_obs_diag(L, L.d_diag64, s);
    if (share) {
        launch_max_share(L.d_dinv64, L.d_diag64, L.N, d_share, s);
        unsigned long long bits = 0;
        GCK(cudaMemcpyAsync(&bits, d_share, sizeof(bits), cudaMemcpyDeviceToHost, s));
        GCK(cudaStreamSynchronize(s));
        std::memcpy(share, &bits, sizeof(double));
        dev_free(d_share);
    }
    launch_finish_diag(L.d_diag64, L.d_dinv32, L.d_dinv64, L.N, s);
}

static void setup_dense(Level& L, cudaStream_t s) {
    std::vector<double> mu;
    if ((L.col.kind == 2 || L.col.kind == 4) && L.d_mu64) {
        mu.resize((size_t)L.N);
        GCK(cudaMemcpyAsync(mu.data(), L.d_mu64, mu.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        GCK(cudaStreamSynchronize(s));
    }
    std::vector<double> A = dense_operator(L, mu.empty() ? nullptr : mu.data());
    if (!spd_inverse(A, (int)L.N)) throw Error(GMRF_E_NOT_SPD, "coarsest-level operator is not positive definite");
    const int n = (int)L.N;            // store the inverse exactly symmetric (the solve kernel reads columns)
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const double v = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
            A[(size_t)i * n + j] = v;
            A[(size_t)j * n + i] = v;
        }
    std::vector<float> A32(A.size());
    for (size_t i = 0; i < A.size(); ++i) A32[i] = (float)A[i];
    dev_upload(&L.d_dense64, A);
    dev_upload(&L.d_dense32, A32);
}

void posterior_refresh_operator(Posterior& P, cudaStream_t s) {
    const int nl = (int)P.levels.size();
    double share = 0.0;
    for (int l = 0; l < nl; ++l) setup_diag(P.levels[l], s, l == 0 ? &share : nullptr);
    P.data_share = share;
    P.transfer_p1 = share >= kP1DataShare;
    for (int l = 0; l < nl - 1; ++l) P.levels[l].lmax = 1.1 * power_lmax(P, P.levels[l], s);
    setup_dense(P.levels[nl - 1], s);
    GCK(cudaStreamSynchronize(s));
}

void posterior_setup_levels(Posterior& P, cudaStream_t s) {
    const int nl = (int)P.levels.size();
    for (int l = 0; l + 1 < nl; ++l) build_transfer(P.levels[l], P.levels[l + 1]);
    posterior_refresh_operator(P, s);
}

// ---------------------------------------------------------------------------
// workspace

template <typename T> static void alloc_vecs(Posterior& P, Workspace& W, Workspace::Vecs& V) {
    if (V.ready) return;
    const int nblk = W.nblk;
    const long long N0 = P.levels[0].N;
    for (int i = 0; i < 6; ++i) V.pcg[i] = dev_alloc<T>((size_t)nblk * N0 * 4);
    const size_t nl = P.levels.size();
    V.xa.assign(nl, nullptr); V.xb.assign(nl, nullptr); V.d.assign(nl, nullptr); V.res.assign(nl, nullptr);
    V.b.assign(nl, nullptr); V.t1.assign(nl, nullptr); V.t2.assign(nl, nullptr);
    for (size_t l = 0; l < nl; ++l) {
        const size_t n = (size_t)nblk * P.levels[l].N * 4;
        V.xa[l] = dev_alloc<T>(n);
        V.d[l] = dev_alloc<T>(n);
        V.res[l] = dev_alloc<T>(n);
        V.t1[l] = dev_alloc<T>(n);
        V.t2[l] = dev_alloc<T>(n);
        if (l > 0) {
            V.b[l] = dev_alloc<T>(n);
            V.xb[l] = dev_alloc<T>(n);
        }
    }
    V.ready = true;
}

static void free_vecs(Workspace::Vecs& V) {
    for (void* p : V.pcg) dev_free(p);
    for (auto* vec : {&V.xa, &V.xb, &V.d, &V.res, &V.b, &V.t1, &V.t2})
        for (void* p : *vec) dev_free(p);
    if (V.exec) cudaGraphExecDestroy(V.exec);
    if (V.graph) cudaGraphDestroy(V.graph);
    V = Workspace::Vecs();
}

void workspace_free(Workspace* w) {
    if (!w) return;
    dev_free(w->b64); dev_free(w->x64); dev_free(w->r64); dev_free(w->t64); dev_free(w->z2);
    dev_free(w->partial); dev_free(w->red); dev_free(w->red2); dev_free(w->norms); dev_free(w->sc32); dev_free(w->sc64);
    dev_free(w->slot_a); dev_free(w->slot_b);
    if (w->h_red) cudaFreeHost(w->h_red);
    if (w->h_active) cudaFreeHost(w->h_active);
    if (w->h_abort) cudaFreeHost(w->h_abort);
    solve_graph_free(w->sgraph);
    w->sgraph = nullptr;
    free_vecs(w->v32);
    free_vecs(w->v64);
    delete w;
}

Workspace& workspace(Posterior& P, int nblk) {
    auto it = P.ws.find(nblk);
    if (it != P.ws.end()) return *it->second;
    Workspace* W = new Workspace();
    W->nblk = nblk;
    const size_t n = (size_t)nblk * P.levels[0].N * 4;
    W->b64 = dev_alloc<double>(n);
    W->x64 = dev_alloc<double>(n);
    W->r64 = dev_alloc<double>(n);
    W->t64 = dev_alloc<double>(n);
    W->npartial = partial_slots(P, nblk);
    W->partial = dev_alloc<double>(W->npartial);
    W->red = dev_alloc<double>((size_t)nblk * 4);
    W->red2 = dev_alloc<double>((size_t)nblk * 4);
    W->norms = dev_alloc<double>((size_t)nblk * 4);
    W->sc32 = dev_alloc<double>((size_t)nblk * 4 * 8);
    W->sc64 = dev_alloc<double>((size_t)nblk * 4 * 8);
    W->slot_a = dev_alloc<int32_t>((size_t)nblk * 4);
    W->slot_b = dev_alloc<int32_t>((size_t)nblk * 4);
    GCK(cudaMallocHost((void**)&W->h_red, sizeof(double) * nblk * 8));
    GCK(cudaMallocHost((void**)&W->h_active, sizeof(double) * nblk * 4));
    GCK(cudaMallocHost((void**)&W->h_abort, sizeof(int32_t) * 2));
    P.ws[nblk] = W;
    return *W;
}

// ---------------------------------------------------------------------------
// V-cycle

// One V-cycle x = M b on level l.  With rz_partial, the partial sums of
// b . x are written there; the return value is their count per block.
template <typename T>
static int vcycle(Posterior& P, Workspace& W, Workspace::Vecs& V, int l, const T* b, T* x, double* rz_partial,
                  cudaStream_t s) {
    const int nl = (int)P.levels.size();
    Level& L = P.levels[l];
    const int nblk = W.nblk;
    if (l == 0 && P.use_tsp && tsp_fits<T>(L)) {
        launch_tsp<T>(L, P.ic_rinv, L.inv_eps2, b, (T*)V.t1[0], x, nblk, s);
        if (rz_partial) {
            launch_dot<T>(b, x, L.N, nblk, rz_partial, elem_parts(L.N), s);
            return elem_parts(L.N);
        }
        return 0;
    }
    if (l == nl - 1) {
        launch_dense_solve<T>(dense_of<T>(L), b, x, (int)L.N, nblk, s);
        if (rz_partial) {
            launch_dot<T>(b, x, L.N, nblk, rz_partial, elem_parts(L.N), s);
            return elem_parts(L.N);
        }
        return 0;
    }
    const Cheb ch = cheb_coeffs(L.lmax);
    T* X0 = (T*)V.xa[l];
    T* D = (T*)V.d[l];
    T* R = (T*)V.res[l];
    const T* dinv = dinv_of<T>(L);
    // pre-smoothing from x = 0: both Chebyshev steps in one pass (the first,
    // x1 = c2[0] D^-1 b, is pointwise and formed in shared memory)
    StencilArgs<T> a{};
    a.L = L.view<T>();
    a.nblk = nblk;
    a.x = nullptr; a.b = b; a.d = nullptr; a.dinv = dinv; a.out = x; a.out2 = D;
    a.c0 = (T)ch.c2[0]; a.c1 = (T)ch.c1[1]; a.c2 = (T)ch.c2[1];
    launch_stencil<T>(L.geo, M_CHEB0, a, s);
    // residual and restriction (transpose of the interpolation): one pass
    // over the space plane when both space axes coarsen (P1 or bilinear),
    // then linear per remaining axis
    StencilArgs<T> r = a;
    r.x = x; r.b = b; r.d = nullptr; r.out = R; r.out2 = nullptr;
    launch_stencil<T>(L.geo, M_RESID, r, s);
    Level& C = P.levels[l + 1];
    int dims[3] = {L.nx, L.ny, L.nt};
    const int cdims[3] = {C.nx, C.ny, C.nt};
    int last = -1;
    for (int ax = 0; ax < 3; ++ax)
        if (L.coarsen[ax]) last = ax;
    const T* src = R;
    bool use_t1 = true;
    const bool plane = L.coarsen[0] && L.coarsen[1];
    if (L.periodic) {                // torus levels halve x and y together
        launch_restrict_torus<T>(src, (T*)V.b[l + 1], L, C, P.transfer_p1, nblk, s);
        last = -2;
    } else if (plane) {
        T* dst = last == 1 ? (T*)V.b[l + 1] : (T*)V.t1[l];
        use_t1 = false;
        const int32_t* const rs[2] = {L.d_rs[0], L.d_rs[1]};
        const int32_t* const rc[2] = {L.d_rc[0], L.d_rc[1]};
        const int32_t* const pj[2] = {L.d_pj[0], L.d_pj[1]};
        const T* const pw[2] = {pw_of<T>(L, 0), pw_of<T>(L, 1)};
        launch_restrict_xy<T>(src, dst, dims[0], dims[1], dims[2], cdims[0], cdims[1], rs, rc, pj, pw, P.transfer_p1,
                              L.rspan, nblk, s);
        dims[0] = cdims[0];
        dims[1] = cdims[1];
        src = dst;
    }
    for (int ax = plane ? 2 : 0; ax < 3 && last != -2; ++ax) {
        if (!L.coarsen[ax]) continue;
        T* dst = ax == last ? (T*)V.b[l + 1] : (use_t1 ? (T*)V.t1[l] : (T*)V.t2[l]);
        use_t1 = !use_t1;
        launch_restrict_axis<T>(src, dst, dims[0], dims[1], dims[2], ax, cdims[ax], L.d_rs[ax], L.d_rc[ax], L.d_pj[ax],
                                pw_of<T>(L, ax), nblk, s);
        dims[ax] = cdims[ax];
        src = dst;
    }
    vcycle<T>(P, W, V, l + 1, (const T*)V.b[l + 1], (T*)V.xb[l + 1], nullptr, s);
    launch_prolong_add<T>(x, (const T*)V.xb[l + 1], L, C, P.transfer_p1, nblk, s);
    // post-smoothing: a fresh Chebyshev(2) sweep
    StencilArgs<T> p1 = a;
    p1.x = x; p1.d = nullptr; p1.out = X0; p1.out2 = D; p1.c1 = T(0); p1.c2 = (T)ch.c2[0];
    launch_stencil<T>(L.geo, M_CHEB, p1, s);
    StencilArgs<T> p2 = a;
    p2.x = X0; p2.d = D; p2.out = x; p2.out2 = D; p2.partial = rz_partial;
    return launch_stencil<T>(L.geo, M_CHEB, p2, s);
}

// ---------------------------------------------------------------------------
// PCG

template <typename T> static Workspace::Vecs& vecs(Workspace& W);
template <> Workspace::Vecs& vecs<float>(Workspace& W) { return W.v32; }
template <> Workspace::Vecs& vecs<double>(Workspace& W) { return W.v64; }
template <typename T> static double* scal(Workspace& W);
template <> double* scal<float>(Workspace& W) { return W.sc32; }
template <> double* scal<double>(Workspace& W) { return W.sc64; }

// The tiled stencil kernels carry the vector work of one iteration in their
// PCG mode (the marching space-time kernel does not); GMRF_PCG_FUSED=0 selects
// the separate passes.
static bool pcg_fused(const Level& L) {
    static const bool on = [] {
        const char* v = std::getenv("GMRF_PCG_FUSED");
        return !(v && v[0] == '0');
    }();
    return on && L.geo != GEO_XYT;
}

// One PCG iteration.  Separate passes: q = Q p, alpha, r -= alpha q, z = M r,
// beta, then x += alpha p and p = z + beta p in one pass.  Fused: the last
// pass moves into the next iteration's apply, which stages the previous
// direction and z with their halos and forms x += alpha p, p' = z + beta p
// and q = Q p' in one kernel; p and p' alternate between two buffers (a
// neighbouring CTA still reads the old direction's halo), so iteration
// `parity` reads V.pcg[parity ? 5 : 2] and writes the other one, and after
// the last iteration pcg_finish adds the pending alpha p to x.
template <typename T>
static void pcg_iteration(Posterior& P, Workspace& W, Workspace::Vecs& V, double tol2, cudaStream_t s, int parity) {
    Level& L = P.levels[0];
    const int nblk = W.nblk;
    T *x = (T*)V.pcg[0], *r = (T*)V.pcg[1], *p = (T*)V.pcg[2], *q = (T*)V.pcg[3], *z = (T*)V.pcg[4];
    double* sc = scal<T>(W);
    const int P4 = nblk * 4;
    StencilArgs<T> a{};
    a.L = L.view<T>();
    a.nblk = nblk;
    a.partial = W.partial;
    const bool fused = pcg_fused(L);
    if (fused) {
        T* pc = (T*)V.pcg[parity ? 5 : 2];
        T* pn = (T*)V.pcg[parity ? 2 : 5];
        a.x = pc; a.d = z; a.b = x;
        a.out = q; a.out2 = pn; a.out3 = x;
        a.alpha = sc + 2 * P4; a.beta = sc + 3 * P4;
        const int ng = launch_stencil<T>(L.geo, M_PCG, a, s);
        launch_reduce_scalar(0, W.partial, ng, nblk, W.red, sc, tol2, s);
    } else {
        a.x = p; a.out = q;
        const int ng = launch_stencil<T>(L.geo, M_APPLY, a, s);
        launch_reduce_scalar(0, W.partial, ng, nblk, W.red, sc, tol2, s);
    }
    launch_pcg_update_r<T>(r, q, sc, L.N, nblk, s);
    const int nz = vcycle<T>(P, W, V, 0, r, z, W.partial, s);
    launch_reduce_scalar(2, W.partial, nz, nblk, W.red, sc, tol2, s);
    if (!fused) launch_pcg_update_xp<T>(x, p, z, sc, L.N, nblk, s);     // x += alpha p with this iteration's p
}

// After `iters` iterations: the fused form still owes x += alpha p with the
// direction of the last iteration (written to V.pcg[2] after an even count).
template <typename T>
static void pcg_finish(Posterior& P, Workspace& W, Workspace::Vecs& V, int iters, cudaStream_t s) {
    Level& L = P.levels[0];
    if (!pcg_fused(L) || iters <= 0) return;
    const T* pl = (const T*)V.pcg[(iters % 2 == 0) ? 2 : 5];
    launch_pcg_update_x<T>((T*)V.pcg[0], pl, scal<T>(W), L.N, W.nblk, s);
}

static const int kItersPerGraph = 2;

// the device-driven solve graph (on by default; GMRF_DEVICE_LOOP=0 selects the
// host-driven loop, which also serves the plain FP64 path and timeouts)
static bool device_loop_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("GMRF_DEVICE_LOOP");
        return !(v && v[0] == '0');
    }();
    return on;
}

// x = 0, rz = r^T M r with z = M r, p = z: the start of a PCG solve on the
// right-hand side already in V.pcg[1]
template <typename T>
static void pcg_prologue(Posterior& P, Workspace& W, double tol2, cudaStream_t s) {
    Level& L = P.levels[0];
    Workspace::Vecs& V = vecs<T>(W);
    const int nblk = W.nblk;
    T *x = (T*)V.pcg[0], *r = (T*)V.pcg[1], *p = (T*)V.pcg[2], *z = (T*)V.pcg[4];
    double* sc = scal<T>(W);
    const int ne = elem_parts(L.N);
    const size_t bytes = (size_t)nblk * L.N * 4 * sizeof(T);
    GCK(cudaMemsetAsync(x, 0, bytes, s));
    launch_norm2<T>(r, L.N, nblk, W.partial, ne, s);
    launch_reduce_scalar(4, W.partial, ne, nblk, W.red, sc, tol2, s);
    const int nz = vcycle<T>(P, W, V, 0, r, z, W.partial, s);
    launch_reduce_scalar(3, W.partial, nz, nblk, W.red, sc, tol2, s);
    GCK(cudaMemcpyAsync(p, z, bytes, cudaMemcpyDeviceToDevice, s));
}

// Solves Q x = r (r already in V.pcg[1]) into V.pcg[0]; returns iterations.
template <typename T>
static int pcg(Posterior& P, Workspace& W, double tol, int maxit, cudaStream_t s, bool use_graph, bool* breakdown,
               const std::chrono::steady_clock::time_point* deadline) {
    Level& L = P.levels[0];
    Workspace::Vecs& V = vecs<T>(W);
    const int nblk = W.nblk;
    T *x = (T*)V.pcg[0], *r = (T*)V.pcg[1], *p = (T*)V.pcg[2], *z = (T*)V.pcg[4];
    double* sc = scal<T>(W);
    const int nt = (int)L.ntiles(), ne = elem_parts(L.N);
    const double tol2 = tol * tol;
    pcg_prologue<T>(P, W, tol2, s);
    const int P4 = nblk * 4;
    (void)x; (void)r; (void)p; (void)z; (void)nt; (void)ne;
    if (use_graph && V.graph == nullptr) {
        // a second capture when launch shapes were measured after the first
        for (int pass = 0; pass < 2; ++pass) {
            GCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            capture_begin();
            for (int k = 0; k < kItersPerGraph; ++k) pcg_iteration<T>(P, W, V, tol2, s, k & 1);
            V.graph_kernels = capture_end();
            cudaMemcpyAsync(W.h_active, sc + 6 * P4, sizeof(double) * P4, cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(W.h_red, sc + 7 * P4, sizeof(double) * P4, cudaMemcpyDeviceToHost, s);
            GCK(cudaStreamEndCapture(s, &V.graph));
            if (pass == 1 || !tune_flush(s)) break;
            GCK(cudaGraphDestroy(V.graph));
            V.graph = nullptr;
        }
        GCK(cudaGraphInstantiate(&V.exec, V.graph, 0));
    }
    int it = 0;
    *breakdown = false;
    while (it < maxit) {
        if (use_graph) {
            GCK(cudaGraphLaunch(V.exec, s));
            note_graph_launch(V.graph_kernels);
            it += kItersPerGraph;
        } else {
            pcg_iteration<T>(P, W, V, tol2, s, it & 1);
            GCK(cudaMemcpyAsync(W.h_active, sc + 6 * P4, sizeof(double) * P4, cudaMemcpyDeviceToHost, s));
            GCK(cudaMemcpyAsync(W.h_red, sc + 7 * P4, sizeof(double) * P4, cudaMemcpyDeviceToHost, s));
            it += 1;
        }
        GCK(cudaStreamSynchronize(s));
        bool any = false;
        for (int i = 0; i < P4; ++i) {
            any |= W.h_active[i] != 0.0;
            *breakdown |= W.h_red[i] != 0.0;
        }
        if (!any) break;
        if (deadline && std::chrono::steady_clock::now() > *deadline) throw Error(GMRF_E_TIMEOUT, "solve exceeded timeout_s");
    }
    pcg_finish<T>(P, W, V, it, s);
    return it;
}

// The graph bakes in the tolerance; re-capture when it changes.
template <typename T> static void invalidate_graph(Workspace::Vecs& V) {
    if (V.exec) cudaGraphExecDestroy(V.exec);
    if (V.graph) cudaGraphDestroy(V.graph);
    V.exec = nullptr;
    V.graph = nullptr;
}


// ---------------------------------------------------------------------------
// FP64 iterative refinement

void apply64(Posterior& P, int nblk, const double* x64, double* y64, cudaStream_t s) {
    Level& L = P.levels[0];
    StencilArgs<double> a{};
    a.L = L.view<double>();
    a.nblk = nblk;
    a.x = x64;
    a.out = y64;
    launch_stencil<double>(L.geo, M_APPLY, a, s);
}

// ---------------------------------------------------------------------------
// Device-driven solve: the FP64 refinement loop and each PCG loop run as
// conditional while nodes of one CUDA graph, so a whole solve is one graph
// launch with no host round trip; kernels decide convergence on the device.
// The controller reproduces the host loop of solve_blocked: per right-hand
// side, the D^-1-weighted residual relative to the first one, the forward
// error estimate rho/(1-rho) |dx| of the last correction, and the unweighted
// residual norm that scales the FP32 inner right-hand side.

namespace {

// controller state: doubles [bn | dxn | dxp | xn] x P4 then max_rel;
// ints: 0 residual evaluations, 1 inner iterations, 2 iterations of the
// current PCG loop, 3 converged, 4 breakdown, 5 non-finite residual
enum { IS_REF = 0, IS_INNER = 1, IS_PCG = 2, IS_CONV = 3, IS_BRK = 4, IS_NONFIN = 5, IS_N = 8 };

__global__ void k_ctrl_reset(double* __restrict__ ds, int* __restrict__ is, int P4) {
    for (int i = threadIdx.x; i < P4; i += blockDim.x) {
        ds[0 * P4 + i] = 0.0;
        ds[1 * P4 + i] = -1.0;
        ds[2 * P4 + i] = -1.0;
        ds[3 * P4 + i] = 0.0;
    }
    if (threadIdx.x == 0) {
        ds[4 * P4] = 0.0;
        for (int k = 0; k < IS_N; ++k) is[k] = 0;
    }
}

// after a residual: red = |r|_D^2, red2 = |r|^2 per right-hand side
__global__ void k_ctrl(const double* __restrict__ red, const double* __restrict__ red2, double* __restrict__ norms,
                       double* __restrict__ ds, int* __restrict__ is, int P4, double rtol, double xtol, int max_refine,
                       cudaGraphConditionalHandle h) {
    __shared__ int s_open, s_bad;
    __shared__ double s_max;
    if (threadIdx.x == 0) { s_open = 0; s_bad = 0; s_max = 0.0; }
    __syncthreads();
    const bool first = is[IS_REF] == 0;
    double mx = 0.0;
    int open = 0, bad = 0;
    for (int i = threadIdx.x; i < P4; i += blockDim.x) {
        const double v = red[i];
        if (!isfinite(v)) bad = 1;
        const double rn = sqrt(fmax(v, 0.0));
        if (first) ds[0 * P4 + i] = rn;
        const double bn = ds[0 * P4 + i];
        const double rel = bn > 0.0 ? rn / bn : 0.0;
        mx = fmax(mx, rel);
        bool done = rel <= rtol;
        const double dxn = ds[1 * P4 + i], dxp = ds[2 * P4 + i];
        if (done && dxn >= 0.0) {
            double est = dxn;
            if (dxp > 0.0) {
                const double rho = dxn / dxp;
                est = rho < 0.5 ? dxn * rho / (1.0 - rho) : dxn;
            }
            done = est <= xtol * ds[3 * P4 + i];
        }
        norms[i] = done ? 0.0 : sqrt(fmax(red2[i], 0.0));
        open |= done ? 0 : 1;
    }
    if (open) atomicOr(&s_open, 1);
    if (bad) atomicOr(&s_bad, 1);
    // max of the relative residuals (non-negative: the bit patterns order like the values)
    atomicMax(reinterpret_cast<unsigned long long*>(&s_max), (unsigned long long)__double_as_longlong(mx));
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nref = ++is[IS_REF];
        ds[4 * P4] = s_max;
        is[IS_CONV] = s_open ? 0 : 1;
        if (s_bad) is[IS_NONFIN] = 1;
        const bool more = s_open && !s_bad && nref - 1 < max_refine;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}

// after a correction: red = |d|^2, red2 = |x|^2 of the FP32 correction and the iterate
__global__ void k_ctrl_dx(const double* __restrict__ red, const double* __restrict__ red2, const double* __restrict__ norms,
                          double* __restrict__ ds, int P4) {
    for (int i = threadIdx.x; i < P4; i += blockDim.x) {
        if (norms[i] == 0.0) continue;
        ds[2 * P4 + i] = ds[1 * P4 + i];
        ds[1 * P4 + i] = norms[i] * sqrt(fmax(red[i], 0.0));
        ds[3 * P4 + i] = sqrt(fmax(red2[i], 0.0));
    }
}

// PCG loop control: run while a right-hand side is active and below max_inner
__global__ void k_pcg_start(const double* __restrict__ sc, int P4, int* __restrict__ is, int max_inner,
                            cudaGraphConditionalHandle h) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < P4; i += blockDim.x)
        if (sc[6 * P4 + i] != 0.0) atomicOr(&any, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        is[IS_PCG] = 0;
        cudaGraphSetConditional(h, (any && max_inner > 0) ? 1u : 0u);
    }
}

__global__ void k_pcg_cond(const double* __restrict__ sc, int P4, int* __restrict__ is, int max_inner, int step,
                           cudaGraphConditionalHandle h) {
    __shared__ int any, brk;
    if (threadIdx.x == 0) { any = 0; brk = 0; }
    __syncthreads();
    for (int i = threadIdx.x; i < P4; i += blockDim.x) {
        if (sc[6 * P4 + i] != 0.0) atomicOr(&any, 1);
        if (sc[7 * P4 + i] != 0.0) atomicOr(&brk, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        is[IS_PCG] += step;
        is[IS_INNER] += step;
        if (brk) is[IS_BRK] = 1;
        cudaGraphSetConditional(h, (any && is[IS_PCG] < max_inner) ? 1u : 0u);
    }
}

}  // namespace

struct SolveGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap2 = nullptr, cap3 = nullptr;      // capture streams of the loop bodies
    double* ds = nullptr;                             // controller state (device)
    int* is = nullptr;
    double* h_ds = nullptr;                           // pinned mirrors
    int* h_is = nullptr;
    // what the graph bakes in
    const double* b64 = nullptr;
    double* x64 = nullptr;
    double rtol = -1, inner_tol = -1;
    int max_refine = -1, max_inner = -1;
    unsigned long long k_init = 0, k_pre = 0, k_pcg = 0, k_post = 0;    // kernels per segment
};

void solve_graph_free(SolveGraph* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->cap2) cudaStreamDestroy(g->cap2);
    if (g->cap3) cudaStreamDestroy(g->cap3);
    dev_free(g->ds);
    dev_free(g->is);
    if (g->h_ds) cudaFreeHost(g->h_ds);
    if (g->h_is) cudaFreeHost(g->h_is);
    delete g;
}

// the residual of the current iterate into W.r64 with red = |r|_D^2, red2 = |r|^2
// (double-float pairs where the level allows them)
static bool refinement_residual(Posterior& P, Workspace& W, int nblk, const double* x64, const double* b64, cudaStream_t s) {
    Level& L = P.levels[0];
    const int ne = elem_parts(L.N);
    bool pairs = false;
    if (resid_df_applicable(L)) {
        const int ng = launch_resid_df(L, x64, b64, W.r64, L.d_dinv64, W.partial, nblk, s);
        launch_reduce(W.partial, ng, nblk, W.red, s);
        launch_norm2_df(W.r64, L.N, nblk, W.partial, ne, s);
        pairs = true;
    } else {
        StencilArgs<double> a{};
        a.L = L.view<double>();
        a.nblk = nblk;
        a.x = x64; a.b = b64; a.out = W.r64; a.partial = W.partial;
        a.rweight = L.d_dinv64;
        const int ng = launch_stencil<double>(L.geo, M_RESID, a, s);
        launch_reduce(W.partial, ng, nblk, W.red, s);
        launch_norm2<double>(W.r64, L.N, nblk, W.partial, ne, s);
    }
    launch_reduce(W.partial, ne, nblk, W.red2, s);
    return pairs;
}

// appends a while node with handle h after the work captured so far on s;
// returns its body graph
static cudaGraph_t add_while(cudaStream_t s, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    GCK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams prm = {cudaGraphNodeTypeConditional};
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    GCK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &prm));
    GCK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return prm.conditional.phGraph_out[0];
}

static void build_solve_graph(Posterior& P, Workspace& W, SolveGraph& G, const double* b64, double* x64,
                              const gmrf_solve_opts& o, double inner_tol, cudaStream_t s) {
    Level& L = P.levels[0];
    const int nblk = W.nblk, P4 = nblk * 4;
    Workspace::Vecs& V = W.v32;
    const double tol2 = inner_tol * inner_tol;
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G.exec = nullptr;
    G.graph = nullptr;
    if (!G.cap2) GCK(cudaStreamCreateWithFlags(&G.cap2, cudaStreamNonBlocking));
    if (!G.cap3) GCK(cudaStreamCreateWithFlags(&G.cap3, cudaStreamNonBlocking));
    if (!G.ds) G.ds = dev_alloc<double>((size_t)5 * P4);
    if (!G.is) G.is = dev_alloc<int>(IS_N);
    if (!G.h_ds) GCK(cudaMallocHost((void**)&G.h_ds, sizeof(double) * 5 * P4));
    if (!G.h_is) GCK(cudaMallocHost((void**)&G.h_is, sizeof(int) * IS_N));
    const double xtol = 100.0 * o.rtol;
    cudaGraph_t g = nullptr;
    GCK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h_ref, h_pcg;
    GCK(cudaGraphConditionalHandleCreate(&h_ref, g, 0, 0));
    // initial residual and test
    GCK(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    capture_begin();
    k_ctrl_reset<<<1, 256, 0, s>>>(G.ds, G.is, P4);
    note_launch();
    refinement_residual(P, W, nblk, x64, b64, s);
    k_ctrl<<<1, 256, 0, s>>>(W.red, W.red2, W.norms, G.ds, G.is, P4, o.rtol, xtol, o.max_refine, h_ref);
    note_launch();
    G.k_init = capture_end();
    cudaGraph_t body = add_while(s, h_ref);
    GCK(cudaStreamEndCapture(s, &g));
    // refinement step: scaled FP32 correction by PCG, update, new residual, test
    GCK(cudaGraphConditionalHandleCreate(&h_pcg, body, 0, 0));
    GCK(cudaStreamBeginCaptureToGraph(G.cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    capture_begin();
    if (resid_df_applicable(L)) launch_scale_cast_df(W.r64, W.norms, (float*)V.pcg[1], L.N, nblk, G.cap2);
    else launch_scale_cast(W.r64, W.norms, (float*)V.pcg[1], L.N, nblk, G.cap2);
    pcg_prologue<float>(P, W, tol2, G.cap2);
    k_pcg_start<<<1, 256, 0, G.cap2>>>(W.sc32, P4, G.is, o.max_inner, h_pcg);
    note_launch();
    G.k_pre = capture_end();
    cudaGraph_t pbody = add_while(G.cap2, h_pcg);
    capture_begin();
    pcg_finish<float>(P, W, V, kItersPerGraph, G.cap2);     // the body runs whole pairs of iterations
    const int ne = elem_parts(L.N);
    launch_axpy_mixed(x64, W.norms, (const float*)V.pcg[0], L.N, nblk, W.partial, G.cap2);
    launch_reduce(W.partial, ne, nblk, W.red, G.cap2);
    launch_reduce(W.partial + (size_t)nblk * ne * 4, ne, nblk, W.red2, G.cap2);
    k_ctrl_dx<<<1, 256, 0, G.cap2>>>(W.red, W.red2, W.norms, G.ds, P4);
    note_launch();
    refinement_residual(P, W, nblk, x64, b64, G.cap2);
    k_ctrl<<<1, 256, 0, G.cap2>>>(W.red, W.red2, W.norms, G.ds, G.is, P4, o.rtol, xtol, o.max_refine, h_ref);
    note_launch();
    G.k_post = capture_end();
    GCK(cudaStreamEndCapture(G.cap2, &body));
    // PCG body: kItersPerGraph iterations, then the loop test
    GCK(cudaStreamBeginCaptureToGraph(G.cap3, pbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    capture_begin();
    for (int k = 0; k < kItersPerGraph; ++k) pcg_iteration<float>(P, W, V, tol2, G.cap3, k & 1);
    k_pcg_cond<<<1, 256, 0, G.cap3>>>(W.sc32, P4, G.is, o.max_inner, kItersPerGraph, h_pcg);
    note_launch();
    G.k_pcg = capture_end();
    GCK(cudaStreamEndCapture(G.cap3, &pbody));
    GCK(cudaGraphInstantiate(&G.exec, g, 0));
    G.graph = g;
    G.b64 = b64;
    G.x64 = x64;
    G.rtol = o.rtol;
    G.inner_tol = inner_tol;
    G.max_refine = o.max_refine;
    G.max_inner = o.max_inner;
}

bool inner_needs_fp64(const Posterior& P) { return P.use_tsp && tsp_mixed_weights(P.levels[0]); }

gmrf_solve_opts solve_opts_for(const Posterior& P, const gmrf_solve_opts& o_in) {
    gmrf_solve_opts o = o_in;
    // automatic inner cap: the multigrid inner solve is restarted from the
    // FP64 residual after 60 iterations (measured faster than longer FP32
    // runs on the space-time priors); the time-stepping preconditioner
    // leaves one outlying eigenvalue per data point or collocation point and
    // needs the longer Krylov run
    if (o.max_inner <= 0) o.max_inner = P.use_tsp ? 200 : 60;
    if (inner_needs_fp64(P)) o.precision = 1;
    return o;
}

bool device_loop_usable(const gmrf_solve_opts& o) {
    return o.precision != 1 && o.batched != 0 && !(o.timeout_s > 0) && device_loop_enabled();
}

// Enqueues the device-driven solve on s (builds its graph on first use) and
// the copy of the controller state to pinned host memory; nothing waits.
void solve_graph_launch(Posterior& P, int nblk, const double* b64, double* x64, const gmrf_solve_opts& o_in, cudaStream_t s) {
    const gmrf_solve_opts o = solve_opts_for(P, o_in);
    Workspace& W = workspace(P, nblk);
    alloc_vecs<float>(P, W, W.v32);
    const double inner_tol = o.inner_rtol;
    if (!W.sgraph) W.sgraph = new SolveGraph();
    SolveGraph& G = *W.sgraph;
    if (!G.exec || G.b64 != b64 || G.x64 != x64 || G.rtol != o.rtol || G.inner_tol != inner_tol ||
        G.max_refine != o.max_refine || G.max_inner != o.max_inner)
    {
        build_solve_graph(P, W, G, b64, x64, o, inner_tol, s);
        if (tune_flush(s)) build_solve_graph(P, W, G, b64, x64, o, inner_tol, s);   // with the measured launch shapes
    }
    const int P4 = nblk * 4;
    GCK(cudaGraphLaunch(G.exec, s));
    GCK(cudaMemcpyAsync(G.h_ds, G.ds, sizeof(double) * 5 * P4, cudaMemcpyDeviceToHost, s));
    GCK(cudaMemcpyAsync(G.h_is, G.is, sizeof(int) * IS_N, cudaMemcpyDeviceToHost, s));
}

// After s has finished a solve_graph_launch: its statistics (and the checks
// of the stencil abort flags and of a non-finite residual).
SolveStats solve_graph_collect(Posterior& P, int nblk, cudaStream_t s) {
    Workspace& W = workspace(P, nblk);
    SolveGraph& G = *W.sgraph;
    const int P4 = nblk * 4;
    SolveStats st;
    st.refinements = G.h_is[IS_REF];
    st.inner = G.h_is[IS_INNER];
    st.converged = G.h_is[IS_CONV] != 0;
    st.breakdown = G.h_is[IS_BRK] != 0;
    st.max_rel = G.h_ds[4 * P4];
    const unsigned long long corrections = st.refinements > 0 ? (unsigned long long)(st.refinements - 1) : 0;
    note_graph_launch(G.k_init + corrections * (G.k_pre + G.k_post) +
                      (unsigned long long)(st.inner / kItersPerGraph) * G.k_pcg);
    if (stencil_abort_take(s)) throw Error(GMRF_E_CUDA, "stencil kernel: staged input tile did not arrive (bounded wait)");
    if (G.h_is[IS_NONFIN]) throw Error(GMRF_E_NOT_SPD, "non-finite residual in refinement");
    return st;
}

static SolveStats solve_blocked_graph(Posterior& P, int nblk, const double* b64, double* x64, const gmrf_solve_opts& o,
                                      cudaStream_t s) {
    solve_graph_launch(P, nblk, b64, x64, o, s);
    GCK(cudaStreamSynchronize(s));
    return solve_graph_collect(P, nblk, s);
}

SolveStats solve_blocked(Posterior& P, int nblk, const double* b64, double* x64, const gmrf_solve_opts& o_in,
                         cudaStream_t s, bool x_zero) {
    const gmrf_solve_opts o = solve_opts_for(P, o_in);
    if (device_loop_usable(o)) return solve_blocked_graph(P, nblk, b64, x64, o, s);
    (void)x_zero;
    Workspace& W = workspace(P, nblk);
    Level& L = P.levels[0];
    const int P4 = nblk * 4;
    const bool fp64 = o.precision == 1;
    const bool graph = o.batched != 0;
    if (fp64) alloc_vecs<double>(P, W, W.v64);
    else alloc_vecs<float>(P, W, W.v32);
    std::chrono::steady_clock::time_point dl;
    const bool has_dl = o.timeout_s > 0;
    if (has_dl) dl = std::chrono::steady_clock::now() + std::chrono::microseconds((long long)(o.timeout_s * 1e6));
    const double inner_tol = fp64 ? std::min(o.inner_rtol, 0.5 * o.rtol) : o.inner_rtol;
    Workspace::Vecs& V = fp64 ? W.v64 : W.v32;
    if (V.graph_tol != inner_tol) {
        invalidate_graph<float>(V);
        V.graph_tol = inner_tol;
    }
    std::vector<double> bn((size_t)P4, 0.0), rn((size_t)P4, 0.0), nrm((size_t)P4, 0.0);
    // forward-error test: the correction of the last refinement step and the
    // contraction rho between the last two estimate the remaining error as
    // rho / (1 - rho) |dx|; it must be below xtol |x| (xtol = 100 rtol)
    std::vector<double> dxn((size_t)P4, -1.0), dxp((size_t)P4, -1.0), xn((size_t)P4, 0.0);
    const double xtol = 100.0 * o.rtol;
    SolveStats st;
    const int ne = elem_parts(L.N);
    for (int ref = 0; ref <= o.max_refine; ++ref) {
        // r64 holds FP64 values, or (r_pairs) double-float pairs (hi, lo)
        bool r_pairs = false;
        if (ref == 0 && x_zero) {   // r = b
            GCK(cudaMemcpyAsync(W.r64, b64, sizeof(double) * (size_t)nblk * L.N * 4, cudaMemcpyDeviceToDevice, s));
            launch_norm2w(W.r64, L.d_dinv64, L.N, nblk, W.partial, ne, s);
            launch_reduce(W.partial, ne, nblk, W.red, s);
        } else if (!fp64 && resid_df_applicable(L)) {
            // double-float residual: GB300's FP64 rate makes the FP64 stencil compute-bound
            const int ng = launch_resid_df(L, x64, b64, W.r64, L.d_dinv64, W.partial, nblk, s);
            launch_reduce(W.partial, ng, nblk, W.red, s);
            r_pairs = true;
        } else {
            StencilArgs<double> a{};
            a.L = L.view<double>();
            a.nblk = nblk;
            a.x = x64; a.b = b64; a.out = W.r64; a.partial = W.partial;
            a.rweight = L.d_dinv64;     // stop on the D^-1-weighted residual norm
            const int ng = launch_stencil<double>(L.geo, M_RESID, a, s);
            launch_reduce(W.partial, ng, nblk, W.red, s);
        }
        GCK(cudaMemcpyAsync(W.h_red, W.red, sizeof(double) * P4, cudaMemcpyDeviceToHost, s));
        stencil_abort_peek_async(W.h_abort, s);
        GCK(cudaStreamSynchronize(s));
        st.refinements++;
        // a stencil CTA that gave up waiting for a staged tile left this
        // residual (and the solve behind it) incomplete
        if (W.h_abort[0] || W.h_abort[1]) {
            stencil_abort_take(s);
            throw Error(GMRF_E_CUDA, "stencil kernel: staged input tile did not arrive (bounded wait)");
        }
        bool conv = true;
        st.max_rel = 0.0;
        for (int i = 0; i < P4; ++i) {
            rn[(size_t)i] = std::sqrt(std::max(W.h_red[i], 0.0));
            if (!std::isfinite(W.h_red[i])) throw Error(GMRF_E_NOT_SPD, "non-finite residual in refinement");
            if (ref == 0) bn[(size_t)i] = rn[(size_t)i];
            const double rel = bn[(size_t)i] > 0 ? rn[(size_t)i] / bn[(size_t)i] : 0.0;
            st.max_rel = std::max(st.max_rel, rel);
            bool done = rel <= o.rtol;
            if (done && dxn[(size_t)i] >= 0.0) {
                double est = dxn[(size_t)i];
                if (dxp[(size_t)i] > 0.0) {
                    const double rho = dxn[(size_t)i] / dxp[(size_t)i];
                    est = rho < 0.5 ? dxn[(size_t)i] * rho / (1.0 - rho) : dxn[(size_t)i];
                }
                done = est <= xtol * xn[(size_t)i];
            }
            conv &= done;
            nrm[(size_t)i] = done ? 0.0 : rn[(size_t)i];
        }
        if (conv) { st.converged = true; break; }
        if (ref == o.max_refine) break;
        // the inner solve works on r / |r| (unweighted norm keeps FP32 in range)
        if (r_pairs) launch_norm2_df(W.r64, L.N, nblk, W.partial, ne, s);
        else launch_norm2<double>(W.r64, L.N, nblk, W.partial, ne, s);
        launch_reduce(W.partial, ne, nblk, W.red2, s);
        GCK(cudaMemcpyAsync(W.h_red + P4, W.red2, sizeof(double) * P4, cudaMemcpyDeviceToHost, s));
        GCK(cudaStreamSynchronize(s));
        for (int i = 0; i < P4; ++i) nrm[(size_t)i] = nrm[(size_t)i] > 0.0 ? std::sqrt(std::max(W.h_red[P4 + i], 0.0)) : 0.0;
        GCK(cudaMemcpyAsync(W.norms, nrm.data(), sizeof(double) * P4, cudaMemcpyHostToDevice, s));
        bool brk = false;
        if (fp64) {
            launch_scale64(W.r64, W.norms, (double*)W.v64.pcg[1], L.N, nblk, s);
            st.inner += pcg<double>(P, W, inner_tol, o.max_inner, s, graph, &brk, has_dl ? &dl : nullptr);
            launch_axpy_scaled64(x64, W.norms, (const double*)W.v64.pcg[0], L.N, nblk, W.partial, s);
        } else {
            if (r_pairs) launch_scale_cast_df(W.r64, W.norms, (float*)W.v32.pcg[1], L.N, nblk, s);
            else launch_scale_cast(W.r64, W.norms, (float*)W.v32.pcg[1], L.N, nblk, s);
            st.inner += pcg<float>(P, W, inner_tol, o.max_inner, s, graph, &brk, has_dl ? &dl : nullptr);
            launch_axpy_mixed(x64, W.norms, (const float*)W.v32.pcg[0], L.N, nblk, W.partial, s);
        }
        launch_reduce(W.partial, ne, nblk, W.red, s);
        launch_reduce(W.partial + (size_t)nblk * ne * 4, ne, nblk, W.red2, s);
        GCK(cudaMemcpyAsync(W.h_red, W.red, sizeof(double) * P4, cudaMemcpyDeviceToHost, s));
        GCK(cudaMemcpyAsync(W.h_red + P4, W.red2, sizeof(double) * P4, cudaMemcpyDeviceToHost, s));
        GCK(cudaStreamSynchronize(s));
        for (int i = 0; i < P4; ++i) {
            if (nrm[(size_t)i] == 0.0) continue;
            dxp[(size_t)i] = dxn[(size_t)i];
            dxn[(size_t)i] = nrm[(size_t)i] * std::sqrt(std::max(W.h_red[i], 0.0));   // |norm d|
            xn[(size_t)i] = std::sqrt(std::max(W.h_red[P4 + i], 0.0));
        }
        st.breakdown |= brk;
    }
    if (stencil_abort_take(s)) throw Error(GMRF_E_CUDA, "stencil kernel: staged input tile did not arrive (bounded wait)");
    return st;
}

double time_stencil(Posterior& P, int kernel, int nblk, int iters, cudaStream_t s) {
    // kernel ids of gmrf_time_stencil: 0 apply, 1 residual, 2 Chebyshev, 3 PCG
    const int mode = kernel == 3 ? (int)M_PCG : kernel;
    if (mode != M_APPLY && mode != M_RESID && mode != M_CHEB && mode != M_PCG)
        throw Error(GMRF_E_INVALID, "time_stencil: unknown kernel");
    Workspace& W = workspace(P, nblk);
    alloc_vecs<float>(P, W, W.v32);
    Level& L = P.levels[0];
    float* x = (float*)W.v32.pcg[2];
    float* y = (float*)W.v32.pcg[3];
    float* b = (float*)W.v32.pcg[1];
    float* d = (float*)W.v32.d[0];
    float* y2 = (float*)W.v32.xa[0];
    for (int k = 0; k < nblk; ++k) {
        launch_fill_random(x + (size_t)k * L.N * 4, L.N, 99 + k, s);
        launch_fill_random(b + (size_t)k * L.N * 4, L.N, 199 + k, s);
        launch_fill_random(d + (size_t)k * L.N * 4, L.N, 299 + k, s);
    }
    StencilArgs<float> a{};
    a.L = L.view<float>();
    a.nblk = nblk;
    a.x = x; a.out = y; a.partial = W.partial;
    if (mode != M_APPLY) a.b = b;
    if (mode == M_CHEB) { a.d = d; a.dinv = L.d_dinv32; a.out2 = y2; a.c1 = 0.5f; a.c2 = 0.25f; }
    double* ab = nullptr;
    if (mode == M_PCG) {        // the fused iteration: direction, z and iterate in, q, p' and iterate out
        ab = dev_alloc<double>((size_t)nblk * 8);
        GCK(cudaMemsetAsync(ab, 0, sizeof(double) * nblk * 8, s));
        a.d = d; a.out2 = (float*)W.v32.pcg[5]; a.out3 = b; a.alpha = ab; a.beta = ab + nblk * 4;
    }
    launch_stencil<float>(L.geo, mode, a, s);
    cudaEvent_t e0, e1;
    GCK(cudaEventCreate(&e0));
    GCK(cudaEventCreate(&e1));
    GCK(cudaEventRecord(e0, s));
    for (int i = 0; i < iters; ++i) launch_stencil<float>(L.geo, mode, a, s);
    GCK(cudaEventRecord(e1, s));
    GCK(cudaEventSynchronize(e1));
    float ms = 0.f;
    GCK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(ab);
    return ms / iters;
}


template <typename T>
static void stencil_step_t(Posterior& P, int level, int mode, int k, const double* x, const double* b, const double* d,
                           double c0, double c1, double c2, double* out, double* out2, double* out3, double* dots,
                           cudaStream_t s) {
    Level& L = P.levels[(size_t)level];
    const long long N = L.N;
    const int nblk = (k + 3) / 4;
    const size_t nv = (size_t)nblk * N * 4;
    std::vector<int32_t> rows((size_t)nblk * 4, -1);
    for (int i = 0; i < k; ++i) rows[(size_t)i] = i;
    int32_t* drows = dev_alloc<int32_t>(rows.size());
    double* b64 = dev_alloc<double>(nv);
    T* v[6];
    for (int i = 0; i < 6; ++i) v[i] = dev_alloc<T>(nv);   // x, b, d, out, out2, out3 (blocked)
    double* ab = dev_alloc<double>((size_t)nblk * 8);      // PCG: alpha, beta per right-hand side
    {
        std::vector<double> h((size_t)nblk * 8);
        for (int i = 0; i < nblk * 4; ++i) { h[(size_t)i] = c1; h[(size_t)(nblk * 4 + i)] = c2; }
        GCK(cudaMemcpyAsync(ab, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s));
        GCK(cudaStreamSynchronize(s));
    }
    const int parts = std::max(std::max(stencil_max_grid(), march_max_grid()), elem_parts(N));
    double* part = dev_alloc<double>((size_t)nblk * parts * 4);
    double* red = dev_alloc<double>((size_t)nblk * 4);
    GCK(cudaMemcpyAsync(drows, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice, s));
    const double* src[3] = {x, b, d};
    for (int i = 0; i < 3; ++i) {
        GCK(cudaMemsetAsync(v[i], 0, sizeof(T) * nv, s));
        if (!src[i]) continue;
        if (sizeof(T) == 8) {
            launch_pack(src[i], reinterpret_cast<double*>(v[i]), drows, N, nblk, s);
        } else {
            launch_pack(src[i], b64, drows, N, nblk, s);
            launch_cast<T>(b64, v[i], (long long)nv, s);
        }
    }
    StencilArgs<T> a{};
    a.L = L.view<T>();
    a.nblk = nblk;
    a.x = v[0];
    if (mode != M_APPLY) a.b = v[1];
    if ((mode == M_CHEB || mode == M_PCG) && d) a.d = v[2];
    if (mode == M_PCG) {
        a.out3 = v[5];
        a.alpha = ab;
        a.beta = ab + nblk * 4;
    }
    a.dinv = sizeof(T) == 8 ? reinterpret_cast<const T*>(L.d_dinv64) : reinterpret_cast<const T*>(L.d_dinv32);
    a.out = v[3];
    a.out2 = v[4];
    a.c0 = (T)c0;
    a.c1 = (T)c1;
    a.c2 = (T)c2;
    a.partial = part;
    int nparts = 0;
    if (mode == kStepPrecond) {
        // the solve's preconditioner on the finest level: z = M b
        if (level != 0) throw Error(GMRF_E_INVALID, "stencil_step: the preconditioner mode is for level 0");
        Workspace& W = workspace(P, nblk);
        alloc_vecs<T>(P, W, vecs<T>(W));
        nparts = vcycle<T>(P, W, vecs<T>(W), 0, v[1], v[3], part, s);
    } else {
        nparts = launch_stencil<T>(L.geo, mode, a, s);
    }
    launch_reduce(part, nparts, nblk, red, s);
    double* dst[3] = {out, out2, out3};
    for (int i = 0; i < 3; ++i) {
        if (!dst[i]) continue;
        launch_widen<T>(v[3 + i], b64, (long long)nv, s);
        launch_unpack(b64, dst[i], drows, N, nblk, s);
    }
    std::vector<double> h((size_t)nblk * 4);
    GCK(cudaMemcpyAsync(h.data(), red, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    GCK(cudaStreamSynchronize(s));
    const int aborted = stencil_abort_take(s);
    for (int i = 0; i < k; ++i) dots[i] = h[(size_t)i];
    dev_free(drows);
    dev_free(b64);
    for (int i = 0; i < 6; ++i) dev_free(v[i]);
    dev_free(ab);
    dev_free(part);
    dev_free(red);
    if (aborted) throw Error(GMRF_E_CUDA, "stencil kernel: staged input tile did not arrive (bounded wait)");
}

void stencil_step(Posterior& P, int level, int prec, int mode, int k, const double* x, const double* b, const double* d,
                  double c0, double c1, double c2, double* out, double* out2, double* out3, double* dots, cudaStream_t s) {
    if (prec == 1) stencil_step_t<double>(P, level, mode, k, x, b, d, c0, c1, c2, out, out2, out3, dots, s);
    else stencil_step_t<float>(P, level, mode, k, x, b, d, c0, c1, c2, out, out2, out3, dots, s);
}

}  // namespace gmrf
