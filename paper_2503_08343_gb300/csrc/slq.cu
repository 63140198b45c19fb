// log det Q_u|y by stochastic Lanczos quadrature (for the value of the log
// marginal likelihood; not in the paper, which fixes its hyper-parameters).
//
// With D = diag(Q_u|y) and A = D^-1/2 Q_u|y D^-1/2,
//   log det Q_u|y = sum_i log D_ii + tr(log A),
// and tr(log A) is estimated over Rademacher probes v_s (the same Philox
// stream-2 probes as the gradient's trace terms) by v^T log(A) v, each
// evaluated by Gauss quadrature from m Lanczos steps started at v / |v|:
// with T_m = Q^T diag(theta) Q the Lanczos tridiagonal,
//   v^T log(A) v ~ |v|^2 sum_k Q_0k^2 log theta_k
// (Golub and Meurant; Ubaru, Chen and Saad 2017).  The mean over the probes
// is the estimate and its standard error the spread over the probes / sqrt(S).
//
// The Lanczos vectors and the operator apply are FP32 (the fused stencil);
// the alpha / beta dot products are reduced in FP64 and the quadrature runs on
// the host in FP64.  Lanczos runs for all probes as one blocked batch and
// stops when every probe's quadrature value has settled between two checks
// (at steps 16, 32, ... growing by a quarter): a change below 1e-10 of the
// value or below 1 % of the spread of the values over the probes, so that the
// quadrature error is small against the Monte Carlo error; or after max_steps.
#include <algorithm>
#include <cmath>
#include <vector>

#include "host.h"

namespace gmrf {

namespace {

unsigned nb(long long n) { return (unsigned)((n + 255) / 256); }

// D^-1/2 in FP32 and the per-block partial sums of log D_ii
__global__ void k_slq_scale(const double* __restrict__ diag, float* __restrict__ dsq, long long N,
                            double* __restrict__ part) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    double l[4] = {0.0, 0.0, 0.0, 0.0};
    if (n < N) {
        dsq[n] = (float)(1.0 / sqrt(diag[n]));
        l[0] = log(diag[n]);
    }
    block_sum4<256, double>(l, part + (size_t)blockIdx.x * 4);
}

// v_0 = probe / sqrt(N) (Rademacher, Philox stream 2, probe id = slot), vprev = 0,
// u = D^-1/2 v; slots >= S hold zeros
__global__ void k_slq_init(uint64_t seed, int S, const float* __restrict__ dsq, float* __restrict__ v,
                           float* __restrict__ vp, float* __restrict__ u, long long N, float inv_sqrt_n) {
    const int blk = blockIdx.y;
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    float r[4];
    for (int c = 0; c < 4; ++c) {
        const int id = blk * 4 + c;
        r[c] = id < S ? (float)philox_rademacher(seed, (uint32_t)id, (uint64_t)n) * inv_sqrt_n : 0.f;
    }
    const size_t off = ((size_t)blk * N + n) * RW;
    const float d = dsq[n];
    v4store(v + off, V4<float>{r[0], r[1], r[2], r[3]});
    v4store(vp + off, V4<float>{0.f, 0.f, 0.f, 0.f});
    v4store(u + off, V4<float>{d * r[0], d * r[1], d * r[2], d * r[3]});
}

// w = D^-1/2 q - alpha v - beta vprev, written over vprev; |w|^2 partials
__global__ void __launch_bounds__(256) k_slq_update(const float* __restrict__ q, const float* __restrict__ v,
                                                    float* __restrict__ vp, const float* __restrict__ dsq,
                                                    const double* __restrict__ alpha, const double* __restrict__ beta,
                                                    long long N, double* __restrict__ part) {
    const int blk = blockIdx.y;
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (n < N) {
        const size_t off = ((size_t)blk * N + n) * RW;
        const float d = dsq[n];
        const V4<float> qv = v4load(q + off), vv = v4load(v + off), pv = v4load(vp + off);
        float w[4];
        const float qa[4] = {qv.a, qv.b, qv.c, qv.d}, va[4] = {vv.a, vv.b, vv.c, vv.d}, pa[4] = {pv.a, pv.b, pv.c, pv.d};
        for (int c = 0; c < 4; ++c) {
            const float a = (float)alpha[blk * 4 + c], b = (float)beta[blk * 4 + c];
            w[c] = d * qa[c] - a * va[c] - b * pa[c];
            acc[c] = w[c] * w[c];
        }
        v4store(vp + off, V4<float>{w[0], w[1], w[2], w[3]});
    }
    block_sum4<256, float>(acc, part + ((size_t)blk * gridDim.x + blockIdx.x) * 4);
}

// v_next = w / beta (in place in w's buffer), u = D^-1/2 v_next
__global__ void k_slq_next(float* __restrict__ w, float* __restrict__ u, const float* __restrict__ dsq,
                           const double* __restrict__ beta2, long long N) {
    const int blk = blockIdx.y;
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    const size_t off = ((size_t)blk * N + n) * RW;
    const float d = dsq[n];
    V4<float> x = v4load(w + off);
    float s[4];
    for (int c = 0; c < 4; ++c) {
        const double b = sqrt(fmax(beta2[blk * 4 + c], 0.0));
        s[c] = b > 0.0 ? (float)(1.0 / b) : 0.f;
    }
    x = V4<float>{x.a * s[0], x.b * s[1], x.c * s[2], x.d * s[3]};
    v4store(w + off, x);
    v4store(u + off, V4<float>{d * x.a, d * x.b, d * x.c, d * x.d});
}

// beta_j = sqrt(|w|^2) per slot, in place
__global__ void k_slq_sqrt(double* __restrict__ b, int n) {
    const int i = threadIdx.x;
    if (i < n) b[i] = sqrt(fmax(b[i], 0.0));
}

}  // namespace

// e1^T log(T) e1 for the symmetric tridiagonal T (diagonal a[0..m),
// off-diagonal b[0..m-1)): Gauss quadrature with the eigenvalues theta_k of T
// as nodes and the squared first components z_k^2 of its eigenvectors as
// weights (Golub and Welsch 1969).  The eigen-decomposition is the implicit
// symmetric QR iteration with a Wilkinson shift (Golub and Van Loan,
// Matrix Computations, Sec. 8.3): Givens rotations chase the bulge down the
// unreduced block, deflating where an off-diagonal drops below roundoff; only
// the first row of the accumulated rotations is kept.
double gauss_log_quadrature(const std::vector<double>& a, const std::vector<double>& b) {
    const int m = (int)a.size();
    if (m == 0) return 0.0;
    std::vector<double> d(a), e((size_t)std::max(m - 1, 1), 0.0), q((size_t)m, 0.0);
    for (int i = 0; i + 1 < m; ++i) e[(size_t)i] = b[(size_t)i];
    q[0] = 1.0;
    const double eps = 2.2e-16;
    int h = m - 1, sweeps = 0;
    while (h > 0) {
        // deflate negligible off-diagonals at and above the bottom
        for (int i = 0; i < h; ++i)
            if (std::fabs(e[(size_t)i]) <= eps * (std::fabs(d[(size_t)i]) + std::fabs(d[(size_t)i + 1]))) e[(size_t)i] = 0.0;
        if (e[(size_t)h - 1] == 0.0) {
            --h;
            continue;
        }
        int l = h - 1;
        while (l > 0 && e[(size_t)l - 1] != 0.0) --l;
        if (++sweeps > 60 * m) return NAN;
        // Wilkinson shift: the eigenvalue of the trailing 2x2 nearer to d[h]
        const double dd = 0.5 * (d[(size_t)h - 1] - d[(size_t)h]), eh = e[(size_t)h - 1];
        const double den = dd + (dd >= 0 ? 1.0 : -1.0) * std::hypot(dd, eh);
        const double mu = d[(size_t)h] - (den != 0.0 ? eh * eh / den : 0.0);
        double x = d[(size_t)l] - mu, z = e[(size_t)l];
        for (int k = l; k < h; ++k) {
            const double r = std::hypot(x, z);
            const double c = r > 0.0 ? x / r : 1.0, s = r > 0.0 ? z / r : 0.0;
            if (k > l) e[(size_t)k - 1] = r;
            const double ak = d[(size_t)k], bk = e[(size_t)k], ck = d[(size_t)k + 1];
            d[(size_t)k] = c * c * ak + 2.0 * c * s * bk + s * s * ck;
            d[(size_t)k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ck;
            e[(size_t)k] = c * s * (ck - ak) + (c * c - s * s) * bk;
            if (k + 1 < h) {
                x = e[(size_t)k];
                z = s * e[(size_t)k + 1];          // bulge at (k + 2, k)
                e[(size_t)k + 1] *= c;
            }
            const double q0 = q[(size_t)k], q1 = q[(size_t)k + 1];
            q[(size_t)k] = c * q0 + s * q1;
            q[(size_t)k + 1] = -s * q0 + c * q1;
        }
    }
    double out = 0.0;
    for (int k = 0; k < m; ++k) {
        if (!(d[(size_t)k] > 0.0)) return NAN;
        out += q[(size_t)k] * q[(size_t)k] * std::log(d[(size_t)k]);
    }
    return out;
}

SlqResult slq_logdet(Posterior& P, int S, uint64_t seed, int max_steps, cudaStream_t s) {
    Level& F = P.levels[0];
    const long long N = F.N;
    const int nblk = (S + 3) / 4, P4 = nblk * 4;
    const size_t nv = (size_t)nblk * N * 4;
    float* buf = dev_alloc<float>(4 * nv + (size_t)N);
    float *v = buf, *vp = buf + nv, *u = buf + 2 * nv, *q = buf + 3 * nv, *dsq = buf + 4 * nv;
    max_steps = std::max(2, std::min<int>(max_steps, (int)std::min<long long>(N, 100000)));
    double* coef = dev_alloc<double>((size_t)(2 * max_steps + 2) * P4);   // alpha[j][slot], beta2[j][slot]
    double* alpha = coef;
    double* beta = coef + (size_t)(max_steps + 1) * P4;                   // beta[j] = |w_j|, beta[0] = 0
    const int parts = std::max(std::max(stencil_max_grid(), march_max_grid()), (int)nb(N));
    double* part = dev_alloc<double>((size_t)nblk * parts * 4);
    SlqResult res;
    try {
        GCK(cudaMemsetAsync(coef, 0, sizeof(double) * (size_t)(2 * max_steps + 2) * P4, s));
        k_slq_scale<<<nb(N), 256, 0, s>>>(F.d_diag64, dsq, N, part);
        note_launch();
        launch_reduce(part, (int)nb(N), 1, alpha, s);      // alpha[0][0] holds sum log D temporarily
        double sumlog = 0.0;
        GCK(cudaMemcpyAsync(&sumlog, alpha, sizeof(double), cudaMemcpyDeviceToHost, s));
        GCK(cudaStreamSynchronize(s));
        GCK(cudaMemsetAsync(alpha, 0, sizeof(double) * P4, s));
        k_slq_init<<<dim3(nb(N), nblk), 256, 0, s>>>(seed, S, dsq, v, vp, u, N, (float)(1.0 / std::sqrt((double)N)));
        note_launch();
        std::vector<double> ha, hb;
        std::vector<double> prev((size_t)S, 0.0), est((size_t)S, 0.0);
        std::vector<char> open((size_t)S, 1);
        int steps = 0, next_check = 16;
        bool settled = false;
        for (int j = 0; j < max_steps; ++j) {
            StencilArgs<float> a{};
            a.L = F.view<float>();
            a.nblk = nblk;
            a.x = u;
            a.out = q;
            a.partial = part;
            const int ng = launch_stencil<float>(F.geo, M_APPLY, a, s);       // u^T Q u = v^T A v
            launch_reduce(part, ng, nblk, alpha + (size_t)j * P4, s);
            k_slq_update<<<dim3(nb(N), nblk), 256, 0, s>>>(q, v, vp, dsq, alpha + (size_t)j * P4,
                                                           beta + (size_t)j * P4, N, part);
            note_launch();
            launch_reduce(part, (int)nb(N), nblk, beta + (size_t)(j + 1) * P4, s);
            k_slq_next<<<dim3(nb(N), nblk), 256, 0, s>>>(vp, u, dsq, beta + (size_t)(j + 1) * P4, N);
            note_launch();
            k_slq_sqrt<<<1, 256, 0, s>>>(beta + (size_t)(j + 1) * P4, P4);
            note_launch();
            std::swap(v, vp);
            steps = j + 1;
            if (steps == next_check || steps == max_steps) {
                next_check = std::min(max_steps, next_check + std::max(16, next_check / 4));
                ha.assign((size_t)steps * P4, 0.0);
                hb.assign((size_t)(steps + 1) * P4, 0.0);
                GCK(cudaMemcpyAsync(ha.data(), alpha, sizeof(double) * ha.size(), cudaMemcpyDeviceToHost, s));
                GCK(cudaMemcpyAsync(hb.data(), beta, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, s));
                GCK(cudaStreamSynchronize(s));
                double amax = 0.0;
                for (double x : ha) amax = std::max(amax, std::fabs(x));
                for (int k = 0; k < S; ++k) {
                    // the probe's tridiagonal, cut where its Krylov space closed (beta ~ 0)
                    std::vector<double> ta, tb;
                    for (int i = 0; i < steps; ++i) {
                        ta.push_back(ha[(size_t)i * P4 + k]);
                        const double bnext = hb[(size_t)(i + 1) * P4 + k];
                        if (!(bnext > 1e-7 * amax) || i + 1 == steps) break;
                        tb.push_back(bnext);
                    }
                    est[(size_t)k] = (double)N * gauss_log_quadrature(ta, tb);
                    if (!std::isfinite(est[(size_t)k])) throw Error(GMRF_E_NOT_SPD, "Lanczos quadrature met a non-positive node");
                    open[(size_t)k] = (int)ta.size() == steps;
                }
                // settled: no probe's value moved by more than 1e-10 of itself,
                // or by more than 1 % of the spread of the values over the
                // probes (the Monte Carlo error of one probe), since the last check
                double em = 0.0, ev = 0.0;
                for (double e : est) em += e;
                em /= S;
                for (double e : est) ev += (e - em) * (e - em);
                const double spread = S > 1 ? std::sqrt(ev / (S - 1)) : 0.0;
                bool all = true;
                for (int k = 0; k < S; ++k)
                    if (open[(size_t)k] &&
                        std::fabs(est[(size_t)k] - prev[(size_t)k]) > std::max(1e-10 * std::max(1.0, std::fabs(est[(size_t)k])), 0.01 * spread))
                        all = false;
                prev = est;
                if (all && steps >= 32) {
                    settled = true;
                    break;
                }
            }
        }
        double mean = 0.0;
        for (double e : est) mean += e;
        mean /= S;
        double var = 0.0;
        for (double e : est) var += (e - mean) * (e - mean);
        var = S > 1 ? var / (S - 1) : 0.0;
        res.logdet = sumlog + mean;
        res.stderr_ = S > 1 ? std::sqrt(var / S) : INFINITY;
        res.steps = steps;
        res.converged = settled;
        GCK(cudaStreamSynchronize(s));
    } catch (...) {
        cudaStreamSynchronize(s);
        dev_free(buf);
        dev_free(coef);
        dev_free(part);
        throw;
    }
    dev_free(buf);
    dev_free(coef);
    dev_free(part);
    return res;
}

}  // namespace gmrf
