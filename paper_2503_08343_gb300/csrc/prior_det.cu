// Exact log-determinant of the prior precision and the exact prior trace
// terms of the log-likelihood gradient (host code, run once per prior).
//
// Q = B^T B with B square and block lower bidiagonal in time (one block for
// the spatial priors), so
//   log det Q = 2 sum_k log|det B_kk|,
//   1/2 tr(Q^-1 dQ) = tr(B^-1 dB) = sum_k tr(B_kk^-1 dB_kk)
// (B^-1 dB is block lower triangular with diagonal blocks B_kk^-1 dB_kk).
// Every diagonal block is a constant-coefficient stencil: Dirichlet rows
// e_k / eps (App. B) and, on the interior nodes, the 7-point stencil of the
// root's taps (centre, x-1, x+1, y-1, y+1, (x-1,y-1), (x+1,y+1)).  The
// space-time blocks k >= 1 are all the same, so a prior needs at most two
// interior determinants: the spatial block (or the t = 0 block) and the
// transition block.
//
// A periodic prior has one circulant block on the torus and no Dirichlet
// rows: its determinant and traces are sums over the 2D DFT symbol.
// Interior operators are handled two ways:
//  - symmetric and separable (no diagonal taps, equal opposite taps: the
//    Matern blocks, and any block without advection): the operator is a
//    Kronecker sum of tridiagonal Toeplitz matrices, diagonalised by the
//    discrete sine transform, with eigenvalues
//    c0 + 2 cx cos(pi j/(mx+1)) + 2 cy cos(pi k/(my+1)); a derivative
//    operator's symmetric-separable part is diagonal in the same basis and
//    its antisymmetric part has zero trace against a symmetric inverse;
//  - otherwise (advection): banded LU without pivoting (the operators have a
//    positive definite symmetric part, so every leading minor is nonzero),
//    then the band of A^-1 by the Erisman-Tinney recursions
//    (Z = A^-1 = U^-1 L^-1: U Z = L^-1 above the diagonal, Z L = U^-1 below),
//    from which tr(A^-1 X) = sum_n sum_m Z_nm X_mn reads off the entries at
//    the transposed pattern of X.  Cost O(N p^2), N = mx my, p = mx + 1.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "host.h"

namespace gmrf {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int NT7 = 7;   // taps 0..6 of the root stencil (tap 7, t-1, is off the diagonal block)

bool sym_separable(const double a[NT7]) {
    return a[5] == 0.0 && a[6] == 0.0 && a[1] == a[2] && a[3] == a[4];
}

// tr(A^-1 X) and log|det A| for a symmetric separable A (closed form)
void closed_form(int mx, int my, const double a[NT7], const std::vector<Stencil7>& X, InteriorDet& r) {
    std::vector<double> cx((size_t)mx), cy((size_t)my);
    for (int j = 0; j < mx; ++j) cx[(size_t)j] = 2.0 * std::cos(kPi * (j + 1) / (mx + 1));
    for (int k = 0; k < my; ++k) cy[(size_t)k] = my > 1 ? 2.0 * std::cos(kPi * (k + 1) / (my + 1)) : 0.0;
    r.logabsdet = 0.0;
    r.sign = 1;
    r.tr.assign(X.size(), 0.0);
    std::vector<double> xs0(X.size()), xs1(X.size()), xs3(X.size());
    for (size_t p = 0; p < X.size(); ++p) {
        const double* x = X[p].c;
        // symmetric part; its diagonal taps must vanish (separable), the
        // antisymmetric part contributes nothing
        if (0.5 * (x[5] + x[6]) != 0.0) throw Error(GMRF_E_INVALID, "prior trace: non-separable symmetric derivative");
        xs0[p] = x[0];
        xs1[p] = 0.5 * (x[1] + x[2]);
        xs3[p] = 0.5 * (x[3] + x[4]);
    }
    for (int k = 0; k < my; ++k)
        for (int j = 0; j < mx; ++j) {
            const double lam = a[0] + a[1] * cx[(size_t)j] + (my > 1 ? a[3] * cy[(size_t)k] : 0.0);
            if (!(lam != 0.0) || !std::isfinite(lam)) throw Error(GMRF_E_NOT_SPD, "prior block is singular");
            if (lam < 0) r.sign = -r.sign;
            r.logabsdet += std::log(std::fabs(lam));
            for (size_t p = 0; p < X.size(); ++p) {
                const double mu = xs0[p] + xs1[p] * cx[(size_t)j] + (my > 1 ? xs3[p] * cy[(size_t)k] : 0.0);
                r.tr[p] += mu / lam;
            }
        }
}

// tap offsets in the lexicographic interior index n = y mx + x
void tap_geometry(int mx, int o, int& dx, int& dy) {
    static const int DX[NT7] = {0, -1, 1, 0, 0, -1, 1}, DY[NT7] = {0, 0, 0, -1, 1, -1, 1};
    dx = DX[o];
    dy = DY[o];
    (void)mx;
}

// Persistent host threads stepping through a sequence of parallel phases:
// run(nsteps, par, ser) calls par(step, tid, nthreads) on every thread, then
// (after a barrier) ser(step) on the calling thread, then a barrier, for
// step = 0 .. nsteps-1.  The barrier spins on an atomic generation counter
// and yields while it waits long.
class StepPool {
  public:
    explicit StepPool(int n) : n_(std::max(1, n)) {}
    template <typename P, typename S> void run(long long nsteps, P&& par, S&& ser) {
        if (n_ == 1) {
            for (long long k = 0; k < nsteps; ++k) {
                par(k, 0, 1);
                ser(k);
            }
            return;
        }
        std::vector<std::thread> th;
        for (int t = 1; t < n_; ++t)
            th.emplace_back([&, t] {
                for (long long k = 0; k < nsteps; ++k) {
                    par(k, t, n_);
                    barrier();      // parallel phase done
                    barrier();      // serial phase done
                }
            });
        for (long long k = 0; k < nsteps; ++k) {
            par(k, 0, n_);
            barrier();
            ser(k);
            barrier();
        }
        for (auto& x : th) x.join();
    }

  private:
    void barrier() {
        const unsigned g = gen_.load(std::memory_order_acquire);
        if (count_.fetch_add(1, std::memory_order_acq_rel) + 1 == n_) {
            count_.store(0, std::memory_order_relaxed);
            gen_.fetch_add(1, std::memory_order_acq_rel);
            return;
        }
        for (int spin = 0; gen_.load(std::memory_order_acquire) == g; ++spin)
            if (spin > 4000) std::this_thread::yield();
    }
    int n_;
    std::atomic<int> count_{0};
    std::atomic<unsigned> gen_{0};
};

int host_threads(int p) {
    if (p < 48) return 1;
    const unsigned hw = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(hw > 2 ? hw / 2 : 1u, 8u));
}

void chunk(int len, int tid, int nt, int& lo, int& hi) {
    lo = (int)((long long)len * tid / nt);
    hi = (int)((long long)len * (tid + 1) / nt);
}

void band_lu_path(int mx, int my, const double a[NT7], const std::vector<Stencil7>& X, InteriorDet& r) {
    const long long N = (long long)mx * my;
    const int p = my > 1 ? mx + 1 : 1;      // lower = upper bandwidth
    const int W = 2 * p + 1;
    // row-major band: A(i, j) at A[i W + j - i + p]
    std::vector<double> A((size_t)N * W, 0.0);
    for (int y = 0; y < my; ++y)
        for (int x = 0; x < mx; ++x) {
            const long long n = (long long)y * mx + x;
            for (int o = 0; o < NT7; ++o) {
                int dx, dy;
                tap_geometry(mx, o, dx, dy);
                const int xx = x + dx, yy = y + dy;
                if (xx < 0 || xx >= mx || yy < 0 || yy >= my || a[o] == 0.0) continue;
                const long long m = (long long)yy * mx + xx;
                A[(size_t)(n * W + (m - n + p))] += a[o];
            }
        }
    StepPool pool(host_threads(p));
    // LU in place (Doolittle, unit lower L), step k eliminates column k from
    // rows (k, k + p], split over the threads
    bool zero_pivot = false;
    pool.run(
        N,
        [&](long long k, int tid, int nt) {
            const double piv = A[(size_t)(k * W + p)];
            if (!(piv != 0.0) || !std::isfinite(piv)) return;
            const double* rowk = &A[(size_t)(k * W + p)];          // A(k, k + t) at rowk[t]
            const int rows = (int)std::min<long long>(p, N - 1 - k);
            const int tend = rows;
            int lo, hi;
            chunk(rows, tid, nt, lo, hi);
            for (int s = lo + 1; s <= hi; ++s) {
                const long long i = k + s;
                double* rowi = &A[(size_t)(i * W + (k - i + p))];   // A(i, k + t) at rowi[t]
                const double l = rowi[0] / piv;
                rowi[0] = l;
                if (l == 0.0) continue;
                for (int t = 1; t <= tend; ++t) rowi[t] -= l * rowk[t];
            }
        },
        [&](long long k) {
            const double piv = A[(size_t)(k * W + p)];
            if (!(piv != 0.0) || !std::isfinite(piv)) zero_pivot = true;
        });
    if (zero_pivot) throw Error(GMRF_E_NOT_SPD, "prior block: zero pivot in banded LU");
    r.logabsdet = 0.0;
    r.sign = 1;
    for (long long k = 0; k < N; ++k) {
        const double piv = A[(size_t)(k * W + p)];
        if (piv < 0) r.sign = -r.sign;
        r.logabsdet += std::log(std::fabs(piv));
    }
    // columns of L, contiguous: Lc[j p + t - 1] = L(j + t, j), t in [1, p]
    std::vector<double> Lc((size_t)N * p, 0.0);
    for (long long j = 0; j < N; ++j)
        for (int t = 1; t <= p && j + t < N; ++t) Lc[(size_t)(j * p + t - 1)] = A[(size_t)((j + t) * W + (-t + p))];
    // Band of Z = A^-1 in decreasing order of m = min(row, column): step m
    // forms row m above the diagonal, Z(m, m+s) = -(1/U_mm) sum_t U(m, m+t) Z(m+t, m+s)
    // (from U Z = L^-1), and column m below it, Z(m+s, m) = -sum_t Z(m+s, m+t) L(m+t, m)
    // (from Z L = U^-1), both from entries with indices > m only, split over
    // the threads; then the diagonal Z(m, m) = (1 - sum_t U(m, m+t) Z(m+t, m)) / U_mm.
    // Rows live in a ring of p + 2 slots; row n is complete after step n - p.
    const int R = p + 2;
    std::vector<double> zr((size_t)R * W, 0.0);
    auto zrow = [&](long long i) { return &zr[(size_t)((i % R) * W)]; };
    r.tr.assign(X.size(), 0.0);
    auto trace_row = [&](long long n) {      // sum_m Z(n, m) X(m, n), m = n - off(o)
        const double* zn = zrow(n);
        const int x = (int)(n % mx), y = (int)(n / mx);
        for (int o = 0; o < NT7; ++o) {
            int dx, dy;
            tap_geometry(mx, o, dx, dy);
            const int mxp = x - dx, myp = y - dy;
            if (mxp < 0 || mxp >= mx || myp < 0 || myp >= my) continue;
            const long long m = (long long)myp * mx + mxp;
            const double z = zn[m - n + p];
            for (size_t q = 0; q < X.size(); ++q) r.tr[q] += z * X[q].c[o];
        }
    };
    pool.run(
        N,
        [&](long long step, int tid, int nt) {
            const long long m = N - 1 - step;
            const int qn = (int)std::min<long long>(p, N - 1 - m);
            const double* um = &A[(size_t)(m * W + p)];              // U(m, m + t) at um[t]
            double* zm = zrow(m);
            int lo, hi;
            // row m above the diagonal, entries s in (lo, hi]
            chunk(qn, tid, nt, lo, hi);
            if (hi > lo) {
                double acc[1024];
                double* ac = hi - lo <= 1024 ? acc : nullptr;
                std::vector<double> big;
                if (!ac) {
                    big.assign((size_t)(hi - lo), 0.0);
                    ac = big.data();
                } else {
                    std::fill(ac, ac + (hi - lo), 0.0);
                }
                for (int t = 1; t <= qn; ++t) {
                    const double u = um[t];
                    if (u == 0.0) continue;
                    const double* zk = zrow(m + t) + (p - t);         // Z(m+t, m+s) at zk[s]
                    for (int s2 = lo + 1; s2 <= hi; ++s2) ac[s2 - lo - 1] += u * zk[s2];
                }
                const double uinv = 1.0 / um[0];
                for (int s2 = lo + 1; s2 <= hi; ++s2) zm[s2 + p] = -ac[s2 - lo - 1] * uinv;
            }
            // column m below the diagonal, rows m + s, s in (lo, hi]
            chunk(qn, tid, nt, lo, hi);
            const double* lm = &Lc[(size_t)(m * p)];                 // L(m + t, m) at lm[t - 1]
            for (int s2 = lo + 1; s2 <= hi; ++s2) {
                const double* zs = zrow(m + s2) + (p - s2);           // Z(m+s, m+t) at zs[t]
                double acc = 0.0;
                for (int t = 1; t <= qn; ++t) acc += zs[t] * lm[t - 1];
                zrow(m + s2)[p - s2] = -acc;                          // Z(m+s, m)
            }
        },
        [&](long long step) {
            const long long m = N - 1 - step;
            const int qn = (int)std::min<long long>(p, N - 1 - m);
            const double* um = &A[(size_t)(m * W + p)];
            double acc = 0.0;
            for (int t = 1; t <= qn; ++t) acc += um[t] * zrow(m + t)[p - t];    // U(m, m+t) Z(m+t, m)
            zrow(m)[p] = (1.0 - acc) / um[0];
            // row m + p is now complete: take its trace terms, then clear the
            // slot that row m - 1 will use (row m + p + 1, no longer read)
            if (m + p < N) trace_row(m + p);
            if (m > 0) {
                double* z = zrow(m - 1);
                std::fill(z, z + W, 0.0);
            }
        });
    for (long long n = 0; n < std::min<long long>(p, N); ++n) trace_row(n);
}

// Periodic (torus) blocks: B is circulant on the mx x my torus, diagonalised
// by the 2D DFT, with symbol b(w) = sum_o a_o exp(i w.d_o) at the
// frequencies w = 2 pi (j / mx, k / my), so log|det B| = sum_w log|b(w)| and
// tr(B^-1 X) = sum_w x(w) / b(w) (real: the terms of w and -w are conjugate).
void torus_form(int mx, int my, const double a[NT7], const std::vector<Stencil7>& X, InteriorDet& r) {
    static const int DX[NT7] = {0, -1, 1, 0, 0, -1, 1}, DY[NT7] = {0, 0, 0, -1, 1, -1, 1};
    r.logabsdet = 0.0;
    r.sign = 1;
    r.tr.assign(X.size(), 0.0);
    for (int k = 0; k < my; ++k)
        for (int j = 0; j < mx; ++j) {
            const double wx = 2.0 * kPi * j / mx, wy = 2.0 * kPi * k / my;
            double br = 0.0, bi = 0.0;
            double xr[4] = {0, 0, 0, 0}, xi[4] = {0, 0, 0, 0};
            for (int o = 0; o < NT7; ++o) {
                const double ph = wx * DX[o] + wy * DY[o], c = std::cos(ph), sn = std::sin(ph);
                br += a[o] * c;
                bi += a[o] * sn;
                for (size_t p = 0; p < X.size(); ++p) {
                    xr[p] += X[p].c[o] * c;
                    xi[p] += X[p].c[o] * sn;
                }
            }
            const double m2 = br * br + bi * bi;
            if (!(m2 > 0.0) || !std::isfinite(m2)) throw Error(GMRF_E_NOT_SPD, "prior block is singular");
            r.logabsdet += 0.5 * std::log(m2);
            for (size_t p = 0; p < X.size(); ++p) r.tr[p] += (xr[p] * br + xi[p] * bi) / m2;   // Re(x / b)
        }
}

}  // namespace

InteriorDet interior_logdet(int mx, int my, const double a[NT7], const std::vector<Stencil7>& X) {
    InteriorDet r;
    if (mx <= 0 || my <= 0) {
        r.tr.assign(X.size(), 0.0);
        return r;
    }
    if (sym_separable(a)) closed_form(mx, my, a, X, r);
    else band_lu_path(mx, my, a, X, r);
    return r;
}

PriorDet prior_logdet(const gmrf_prior_desc& d, const Level& F) {
    PriorDet out;
    const DerivTaps D = derivative_taps(d, F);
    if (F.periodic) {          // one circulant block on the torus, no Dirichlet rows
        double a[NT7];
        std::vector<Stencil7> X(4);
        for (int o = 0; o < NT7; ++o) {
            a[o] = F.cd[0][o];
            for (int q = 0; q < 4; ++q) X[(size_t)q].c[o] = D.d[q][0][o];
        }
        InteriorDet b;
        torus_form(F.nx, F.ny, a, X, b);
        out.logdet = 2.0 * b.logabsdet;
        for (int q = 0; q < 4; ++q) out.tr[q] = b.tr[(size_t)q];
        return out;
    }
    const bool st = d.kind == GMRF_ADVDIFF_ST_1D || d.kind == GMRF_ADVDIFF_ST_2D;
    const int mx = F.nx - 2, my = F.ny > 1 ? F.ny - 2 : 1;
    const long long ns = (long long)F.nx * F.ny;                 // spatial nodes
    const long long nint = (long long)mx * my;                   // interior spatial nodes
    const long long nbnd = (ns - nint) * (st ? F.nt : 1);        // Dirichlet rows of B
    auto block = [&](int cls) {
        double a[NT7];
        std::vector<Stencil7> X(4);
        for (int o = 0; o < NT7; ++o) {
            a[o] = F.cd[cls][o];
            for (int q = 0; q < 4; ++q) X[(size_t)q].c[o] = D.d[q][cls][o];
        }
        return interior_logdet(mx, my, a, X);
    };
    // Dirichlet rows: B_kk = 1/eps
    double logdetB = (double)nbnd * (-0.5 * std::log(d.eps2));
    double tr[4] = {0, 0, 0, 0};
    if (!st) {
        const InteriorDet b0 = block(0);
        logdetB += b0.logabsdet;
        for (int q = 0; q < 4; ++q) tr[q] = b0.tr[(size_t)q];
    } else {
        const InteriorDet b0 = block(1), b1 = block(0);
        const double nk = (double)(F.nt - 1);
        logdetB += b0.logabsdet + nk * b1.logabsdet;
        for (int q = 0; q < 4; ++q) tr[q] = b0.tr[(size_t)q] + nk * b1.tr[(size_t)q];
        if (F.noise) {
            // B = T_K B_w on the transition levels: + log|det T_K| per level
            // (interior tridiagonal Toeplitz, DST eigenvalues); T_K does not
            // depend on the parameters, so the traces are those of B_w
            double lt = 0.0;
            for (int j = 1; j <= mx; ++j) {
                const double lam = F.tk_c + 2.0 * F.tk_o * std::cos(kPi * j / (mx + 1));
                if (!(lam != 0.0)) throw Error(GMRF_E_NOT_SPD, "noise transform is singular");
                lt += std::log(std::fabs(lam));
            }
            logdetB += nk * lt;
        }
    }
    out.logdet = 2.0 * logdetB;
    for (int q = 0; q < 4; ++q) out.tr[q] = tr[q];
    return out;
}

}  // namespace gmrf
