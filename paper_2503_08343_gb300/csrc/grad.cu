// Gradient of the log marginal likelihood of point data with respect to
// theta = (log kappa, log tau, log sigma, cx, nu).  Not in the paper (which
// fixes its hyper-parameters); Gaussian identities with Q = B^T B,
// Q_u|y = Q + A^T R^-1 A, b = A^T R^-1 y, mu = Q_u|y^-1 b:
//   dl = 1/2 tr(Q^-1 dQ) - 1/2 tr(Q_u|y^-1 dQ_u|y) - 1/2 mu^T dQ_u|y mu
//        + mu^T db - 1/2 y^T d(R^-1) y + 1/2 tr(R d(R^-1)),
// with dQ = dB^T B + B^T dB for the prior parameters and, for log sigma,
// d(R^-1) = -2 R^-1, dQ_u|y = A^T d(R^-1) A, db = A^T d(R^-1) y.  The prior
// trace 1/2 tr(Q^-1 dQ) is exact (prior_det.cu: the block lower-bidiagonal
// root gives it from the diagonal blocks alone); the posterior trace is the
// Hutchinson estimate tr(Q_u|y^-1 dX) ~ mean_s (Q_u|y^-1 v_s)^T dX v_s over
// Rademacher probes v_s (Philox stream 2) from one batched posterior solve
// [mean, probes].  The value
//   l = 1/2 log det Q - 1/2 log det Q_u|y - 1/2 log det R - 1/2 y^T R^-1 y
//       + 1/2 b^T mu - (M/2) log 2 pi
// takes log det Q exactly and log det Q_u|y by stochastic Lanczos quadrature
// on the same probes (slq.cu).
#include <cmath>
#include <cstring>
#include <future>
#include <vector>

#include "handles.h"

namespace gmrf {

namespace {

constexpr int NPAR = 4;   // prior parameters handled by the stencil contraction: log kappa, log tau, cx, nu

// (dB w)^T (B v) + (B w)^T (dB v) summed over rows, per parameter and slot;
// also (B w)^T (B v) for reference.  Rows are nodes; Dirichlet rows have no
// parameter dependence.  One thread per row, gathering w and v at the taps.
__global__ void __launch_bounds__(256) k_probe_contract(const LevelView<double> L, const DerivTaps D,
                                                        const double* __restrict__ Wv, const double* __restrict__ Vv,
                                                        double* __restrict__ part) {
    const int nx = L.nx, ny = L.ny, nt = L.nt;
    const long long N = L.N;
    const int blk = blockIdx.y;
    const long long r = (long long)blockIdx.x * 256 + threadIdx.x;
    double acc[NPAR][4];
#pragma unroll
    for (int p = 0; p < NPAR; ++p) acc[p][0] = acc[p][1] = acc[p][2] = acc[p][3] = 0.0;
    if (r < N) {
        const int x = (int)(r % nx);
        const long long q = r / nx;
        const int y = (int)(q % ny), t = (int)(q / ny);
        const bool per = L.periodic != 0;       // torus: no Dirichlet rows or columns, taps wrap
        const bool dir = !per && (x == 0 || x == nx - 1 || (ny > 1 && (y == 0 || y == ny - 1)));
        if (!dir) {
            const int cls = (nt > 1 && t == 0) ? 1 : 0;
            V4<double> bw = v4zero<double>(), bv = v4zero<double>();
            V4<double> dw[NPAR], dv[NPAR];
#pragma unroll
            for (int p = 0; p < NPAR; ++p) { dw[p] = v4zero<double>(); dv[p] = v4zero<double>(); }
            for (int o = 0; o < NTAP; ++o) {
                int xx = x + tap_dx(o), yy = y + tap_dy(o);
                const int tt = t + tap_dt(o);
                if (per) { xx = wrap_idx(xx, nx); yy = wrap_idx(yy, ny); }
                if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || tt < 0 || tt >= nt) continue;
                if (!per && (xx == 0 || xx == nx - 1 || (ny > 1 && (yy == 0 || yy == ny - 1)))) continue;   // eliminated columns
                const double c = (double)L.cf[cls][o];
                const long long col = ((long long)tt * ny + yy) * nx + xx;
                const V4<double> wv = v4load(Wv + ((size_t)blk * N + col) * RW);
                const V4<double> vv = v4load(Vv + ((size_t)blk * N + col) * RW);
                bw = fma4(c, wv, bw);
                bv = fma4(c, vv, bv);
#pragma unroll
                for (int p = 0; p < NPAR; ++p) {
                    const double dc = D.d[p][cls][o];
                    dw[p] = fma4(dc, wv, dw[p]);
                    dv[p] = fma4(dc, vv, dv[p]);
                }
            }
#pragma unroll
            for (int p = 0; p < NPAR; ++p) {
                acc[p][0] = dw[p].a * bv.a + bw.a * dv[p].a;
                acc[p][1] = dw[p].b * bv.b + bw.b * dv[p].b;
                acc[p][2] = dw[p].c * bv.c + bw.c * dv[p].c;
                acc[p][3] = dw[p].d * bv.d + bw.d * dv[p].d;
            }
        }
    }
    const size_t np = gridDim.x;
#pragma unroll
    for (int p = 0; p < NPAR; ++p)
        block_sum4<256, double>(acc[p], part + (((size_t)p * gridDim.y + blk) * np + blockIdx.x) * 4);
}

// per slot: sum_k dr_k (A w)_k (A v)_k over point-data rows (dr = d(R^-1)),
// and sum_k dr_k (A w)_k y_k
__global__ void __launch_bounds__(256) k_obs_contract(const ObsRow* __restrict__ obs, int m, long long N,
                                                      const double* __restrict__ yv, const double* __restrict__ Wv,
                                                      const double* __restrict__ Vv, double* __restrict__ part) {
    const int blk = blockIdx.y;
    const int k = blockIdx.x * 256 + threadIdx.x;
    double a1[4] = {0, 0, 0, 0}, a2[4] = {0, 0, 0, 0};
    if (k < m) {
        const ObsRow& o = obs[k];
        V4<double> aw = v4zero<double>(), av = v4zero<double>();
        for (int n = 0; n < o.nn; ++n) {
            aw = fma4(o.wd[n], v4load(Wv + ((size_t)blk * N + o.node[n]) * RW), aw);
            av = fma4(o.wd[n], v4load(Vv + ((size_t)blk * N + o.node[n]) * RW), av);
        }
        const double dr = -2.0 * o.rinv;
        a1[0] = dr * aw.a * av.a; a1[1] = dr * aw.b * av.b; a1[2] = dr * aw.c * av.c; a1[3] = dr * aw.d * av.d;
        const double yk = yv[o.row];
        a2[0] = dr * aw.a * yk; a2[1] = dr * aw.b * yk; a2[2] = dr * aw.c * yk; a2[3] = dr * aw.d * yk;
    }
    const size_t np = gridDim.x;
    block_sum4<256, double>(a1, part + ((size_t)blk * np + blockIdx.x) * 4);
    block_sum4<256, double>(a2, part + (((size_t)gridDim.y + blk) * np + blockIdx.x) * 4);
}

__global__ void k_rademacher_slots(uint64_t seed, const int32_t* __restrict__ probe_of_slot, double* __restrict__ b64, long long N) {
    const int blk = blockIdx.y;
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    double* p = b64 + ((size_t)blk * N + n) * RW;
    for (int c = 0; c < 4; ++c) {
        const int id = probe_of_slot[blk * RW + c];
        if (id >= 0) p[c] = philox_rademacher(seed, (uint32_t)id, (uint64_t)n);
        else if (id == -2) p[c] = 0.0;
    }
}

__global__ void k_copy_slot(const double* __restrict__ src, int src_slot, double* __restrict__ dst, long long N, int nblk_dst) {
    // broadcast slot src_slot of a blocked batch into every slot of dst
    const int blk = blockIdx.y;
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    const double v = src[((size_t)(src_slot / 4) * N + n) * RW + (src_slot % 4)];
    double* p = dst + ((size_t)blk * N + n) * RW;
    p[0] = v; p[1] = v; p[2] = v; p[3] = v;
    (void)nblk_dst;
}

unsigned nb256(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// derivative taps of the prior root B for the level (the same closed forms as
// level_coefficients, differentiated)
DerivTaps derivative_taps(const gmrf_prior_desc& d, const Level& L) {
    DerivTaps D;
    std::memset(&D, 0, sizeof(D));
    const bool st = d.kind == GMRF_ADVDIFF_ST_1D || d.kind == GMRF_ADVDIFF_ST_2D;
    const int dim = d.kind == GMRF_ADVDIFF_ST_1D ? 1 : 2;
    auto coeffs = [&](const gmrf_prior_desc& dd, double out[2][NTAP]) {
        Level t2 = L;
        level_coefficients(dd, t2);
        std::memcpy(out, t2.cd, sizeof(t2.cd));
    };
    double base[2][NTAP];
    coeffs(d, base);
    // log tau: Q ~ tau^2 (spatial) or tau^-2 (space-time) on non-Dirichlet rows
    const double stau = st ? -1.0 : 1.0;
    for (int c = 0; c < 2; ++c)
        for (int o = 0; o < NTAP; ++o) D.d[1][c][o] = stau * base[c][o];
    // nu and cx: B is affine in them; difference of two evaluations is exact
    {
        gmrf_prior_desc a = d, b = d;
        a.nu = d.nu + 1.0;
        double ca[2][NTAP];
        coeffs(a, ca);
        for (int c = 0; c < 2; ++c)
            for (int o = 0; o < NTAP; ++o) D.d[3][c][o] = (d.kind == GMRF_MATERN2_2D) ? 0.0 : ca[c][o] - base[c][o];
        b.cx = d.cx + 1.0;
        double cb[2][NTAP];
        coeffs(b, cb);
        for (int c = 0; c < 2; ++c)
            for (int o = 0; o < NTAP; ++o) D.d[2][c][o] = (d.kind == GMRF_MATERN2_2D) ? 0.0 : cb[c][o] - base[c][o];
    }
    // log kappa: spatial priors K = kappa^2 Ml + ..., tau fixed: dB = (tau/sqrt(Ml)) 2 kappa^2 Ml at the centre.
    // space-time: kappa acts on kappa0 of the initial level, whose row scale
    // tau0(kappa0)/tau also changes: tau0 ~ kappa0^-1 (2D), kappa0^-3/2 (1D).
    if (!st) {
        D.d[0][0][0] = (d.tau / std::sqrt(L.hx * L.hy)) * 2.0 * d.kappa * d.kappa * (L.hx * L.hy);
    } else {
        const double M = dim == 1 ? L.hx : L.hx * L.hy;
        const double tau0 = dim == 1 ? 1.0 / std::sqrt(4.0 * d.kappa0 * d.kappa0 * d.kappa0)
                                     : 1.0 / std::sqrt(4.0 * 3.14159265358979323846 * d.kappa0 * d.kappa0);
        const double d0 = (tau0 / d.tau) / std::sqrt(M);
        const double dlog = dim == 1 ? -1.5 : -1.0;
        for (int o = 0; o < NTAP; ++o) D.d[0][1][o] = dlog * base[1][o];
        D.d[0][1][0] += d0 * 2.0 * d.kappa0 * d.kappa0 * M;
    }
    return D;
}


// The prior's exact log det Q and trace terms, computed once per prior on
// host threads (cached in the prior; Q does not change).
static PriorDet cached_prior_det(Prior& pr, const Level& F) {
    std::lock_guard<std::mutex> lock(pr.det_mu);
    if (!pr.det_ready) {
        const PriorDet d = prior_logdet(pr.desc, F);
        pr.det_logdet = d.logdet;
        for (int q = 0; q < 4; ++q) pr.det_tr[q] = d.tr[q];
        pr.det_ready = true;
    }
    PriorDet d;
    d.logdet = pr.det_logdet;
    for (int q = 0; q < 4; ++q) d.tr[q] = pr.det_tr[q];
    return d;
}

// Runs the gradient computation; grad/stderr indexed as (log kappa, log tau, log sigma, cx, nu).
SolveStats loglik_grad(Posterior& P, int S, uint64_t seed, const gmrf_solve_opts& o, int max_lanczos, LoglikOut* ll,
                       double grad[5], double gse[5], cudaStream_t s) {
    Level& F = P.levels[0];
    const long long N = F.N;
    const int m = (int)P.m;
    // 0. the exact prior terms on host threads, while the GPU solves
    std::future<PriorDet> pdet = std::async(std::launch::async, [&P, &F] { return cached_prior_det(*P.prior, F); });
    struct Join {          // the host work reads P and F: finish it before any exit from here
        std::future<PriorDet>& f;
        ~Join() {
            if (f.valid()) f.wait();
        }
    } join{pdet};
    // 1. posterior batch: slot 0 = data right-hand side, slots 1..S = probes 0..S-1
    const int nrhs = S + 1, nblk = (nrhs + 3) / 4;
    Workspace& W = workspace(P, nblk);
    std::vector<int32_t> sid((size_t)nblk * 4, -2), pid((size_t)nblk * 4, -2);
    sid[0] = -1;
    pid[0] = -1;
    for (int i = 1; i < nrhs; ++i) pid[(size_t)i] = i - 1;
    GCK(cudaMemcpyAsync(W.slot_a, sid.data(), sizeof(int32_t) * sid.size(), cudaMemcpyHostToDevice, s));
    launch_sample_rhs(F.geo, F.view<double>(), seed, W.slot_a, P.d_bdata, W.b64, nullptr, nullptr, 0, nblk, s);
    GCK(cudaMemcpyAsync(W.slot_b, pid.data(), sizeof(int32_t) * pid.size(), cudaMemcpyHostToDevice, s));
    k_rademacher_slots<<<dim3(nb256(N), nblk), 256, 0, s>>>(seed, W.slot_b, W.b64, N);
    note_launch();
    GCK(cudaMemsetAsync(W.x64, 0, sizeof(double) * nblk * N * 4, s));
    SolveStats st = solve_blocked(P, nblk, W.b64, W.x64, o, s, true);
    // 2. contractions (probe slots: V = probes (W.b64 holds them), solutions in W.x64)
    const DerivTaps D = derivative_taps(P.prior->desc, F);
    const unsigned nbx = nb256(N);
    const size_t pstride = (size_t)nblk * nbx * 4;   // doubles per parameter
    const size_t need = std::max<size_t>((size_t)NPAR * pstride, (size_t)2 * nblk * nb256(std::max(m, 1)) * 4);
    if (P.grad_part_n < need) {
        dev_free(P.d_grad_part);
        P.d_grad_part = dev_alloc<double>(need);
        P.grad_part_n = need;
    }
    double* part = P.d_grad_part;
    auto contract = [&](const double* Wv, const double* Vv, int nb, std::vector<double>& out) {
        k_probe_contract<<<dim3(nbx, nb), 256, 0, s>>>(F.view<double>(), D, Wv, Vv, part);
        note_launch();
        out.assign((size_t)NPAR * nb * 4, 0.0);
        for (int p = 0; p < NPAR; ++p) {
            launch_reduce(part + (size_t)p * nb * nbx * 4, (int)nbx, nb, W.red, s);
            GCK(cudaMemcpyAsync(out.data() + (size_t)p * nb * 4, W.red, sizeof(double) * nb * 4, cudaMemcpyDeviceToHost, s));
        }
        GCK(cudaStreamSynchronize(s));
    };
    std::vector<double> tpost, quadv;
    contract(W.x64, W.b64, nblk, tpost);    // (Q_u|y^-1 v)^T dQ v per slot (slot 0 unused)
    // mu^T dQ mu: broadcast mu (slot 0) into a one-block batch
    Workspace& W1 = workspace(P, 1);
    k_copy_slot<<<dim3(nb256(N), 1), 256, 0, s>>>(W.x64, 0, W1.t64, N, 1);
    note_launch();
    contract(W1.t64, W1.t64, 1, quadv);
    std::vector<double> quad(NPAR);
    for (int p = 0; p < NPAR; ++p) quad[(size_t)p] = quadv[(size_t)p * 4];
    // observation terms for log sigma
    const unsigned nbo = nb256(std::max(m, 1));
    k_obs_contract<<<dim3(nbo, nblk), 256, 0, s>>>(F.d_obs, m, N, P.d_ypoint, W.x64, W.b64, part);
    note_launch();
    std::vector<double> o1((size_t)nblk * 4), o2((size_t)nblk * 4);
    launch_reduce(part, (int)nbo, nblk, W.red, s);
    GCK(cudaMemcpyAsync(o1.data(), W.red, sizeof(double) * nblk * 4, cudaMemcpyDeviceToHost, s));
    launch_reduce(part + (size_t)nblk * nbo * 4, (int)nbo, nblk, W.red2, s);
    GCK(cudaMemcpyAsync(o2.data(), W.red2, sizeof(double) * nblk * 4, cudaMemcpyDeviceToHost, s));
    // mu^T A^T dR A mu: slot 0 against itself
    k_obs_contract<<<dim3(nbo, 1), 256, 0, s>>>(F.d_obs, m, N, P.d_ypoint, W1.t64, W1.t64, part);
    note_launch();
    launch_reduce(part, (int)nbo, 1, W1.red, s);
    GCK(cudaMemcpyAsync(W1.h_red, W1.red, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    GCK(cudaStreamSynchronize(s));
    const double mu_dR_mu = W1.h_red[0];
    // data-fit part 1/2 b^T mu (needed for the value only)
    double btmu = 0.0;
    if (ll) {
        launch_dot_blocked(W.b64, W.x64, N, nblk, part, elem_parts(N), s);
        launch_reduce(part, elem_parts(N), nblk, W.red, s);
        GCK(cudaMemcpyAsync(W.h_red, W.red, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
        GCK(cudaStreamSynchronize(s));
        btmu = W.h_red[0];
    }
    // 3. log det Q_u|y by Lanczos quadrature on the same probes (value only)
    SlqResult slq;
    if (ll) slq = slq_logdet(P, S, seed, max_lanczos, s);
    const PriorDet pd = pdet.get();
    // host assembly
    double ydRy = 0.0, yRy = 0.0, logrinv = 0.0;
    for (int k = 0; k < m; ++k) {
        const double r = P.levels[0].h_obs[(size_t)k].rinv, yk = P.y_point[(size_t)k];
        ydRy += -2.0 * r * yk * yk;
        yRy += r * yk * yk;
        logrinv += std::log(r);
    }
    const int map[NPAR] = {0, 1, 3, 4};       // stencil parameter -> gradient index
    for (int p = 0; p < NPAR; ++p) {
        std::vector<double> est((size_t)S);
        for (int i = 1; i < nrhs; ++i) est[(size_t)i - 1] = -0.5 * tpost[(size_t)p * nblk * 4 + i];
        double mean = 0.0;
        for (double e : est) mean += e;
        mean /= S;
        double var = 0.0;
        for (double e : est) var += (e - mean) * (e - mean);
        var = S > 1 ? var / (S - 1) : 0.0;
        grad[map[p]] = pd.tr[p] + mean - 0.5 * quad[(size_t)p];
        gse[map[p]] = S > 1 ? std::sqrt(var / S) : INFINITY;
    }
    {
        std::vector<double> est((size_t)S);
        for (int i = 1; i < nrhs; ++i) est[(size_t)i - 1] = -0.5 * o1[(size_t)i];
        double mean = 0.0;
        for (double e : est) mean += e;
        mean /= S;
        double var = 0.0;
        for (double e : est) var += (e - mean) * (e - mean);
        var = S > 1 ? var / (S - 1) : 0.0;
        grad[2] = mean - 0.5 * mu_dR_mu + o2[0] - 0.5 * ydRy - (double)m;
        gse[2] = S > 1 ? std::sqrt(var / S) : INFINITY;
    }
    if (ll) {
        const double log2pi = std::log(2.0 * 3.14159265358979323846);
        ll->logdet_prior = pd.logdet;
        ll->logdet_post = slq.logdet;
        ll->loglik = 0.5 * pd.logdet - 0.5 * slq.logdet + 0.5 * logrinv - 0.5 * yRy + 0.5 * btmu - 0.5 * (double)m * log2pi;
        ll->loglik_se = 0.5 * slq.stderr_;
        ll->lanczos_steps = slq.steps;
        ll->lanczos_converged = slq.converged;
    }
    return st;
}

}  // namespace gmrf
