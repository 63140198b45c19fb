// Gauss-Newton for nonlinear PDE observations (Sec. 3.3), collocation rows
// (below) or FEM Crank-Nicolson rows (colloc = 4; see Colloc).  The Burgers
// collocation residual
//   f_r(u) = (u_r - u_{r-t})/dt + u_r (u_{r+x} - u_{r-x})/(2h) - nu (u_{r+x} - 2 u_r + u_{r-x})/h^2
// at interior nodes of levels k >= 1 is linearised at u_k,
//   f(u) ~ f(u_k) + J (u - u_k),  so the linearised data are J u_k - f(u_k) = u_r (u_{r+x} - u_{r-x})/(2h),
// and H = Q + J^T Q_eps J + A^T R^-1 A is applied by the fused stencil with J
// formed on the fly from u_k.  One step solves H d = -grad(-log pi)(u_k),
// warm-started from the previous direction, and backtracks on -log pi.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "handles.h"

namespace gmrf {

namespace {

// b_J = J^T Q_eps (J u - f(u)) at every node: the collocation rows touching a
// node are its own row (centre), the row at x-1 (its x+1 tap), the row at x+1
// (its x-1 tap) and the row at t+1 (its t-1 tap).
__global__ void k_gn_rhs(const LevelView<double> L, const double* __restrict__ u, const double* __restrict__ bdata,
                         double* __restrict__ b) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= L.N) return;
    const int nx = L.nx, nt = L.nt;
    const int x = (int)(n % nx), t = (int)(n / nx);
    const Colloc& c = L.col;
    auto U = [&](int xx, int tt) { return u[(long long)tt * nx + xx]; };
    auto yJ = [&](int rx, int rt) { return U(rx, rt) * (U(rx + 1, rt) - U(rx - 1, rt)) * c.inv_2h; };
    auto coef = [&](int rx, int rt, int which) {   // 0 centre, 1 x-1 tap, 2 x+1 tap
        const double a = U(rx, rt), da = (U(rx + 1, rt) - U(rx - 1, rt)) * c.inv_2h;
        if (which == 0) return c.inv_dt + da + 2.0 * c.nu_h2;
        if (which == 1) return -a * c.inv_2h - c.nu_h2;
        return a * c.inv_2h - c.nu_h2;
    };
    double acc = 0.0;
    const int rxs[4] = {x, x - 1, x + 1, x};
    const int rts[4] = {t, t, t, t + 1};
    for (int k = 0; k < 4; ++k) {
        const int rx = rxs[k], rt = rts[k];
        if (rx < 1 || rx > nx - 2 || rt < 1 || rt >= nt || !colloc_on(c, rx, rt)) continue;
        const double cf = k == 0 ? coef(rx, rt, 0) : (k == 1 ? coef(rx, rt, 2) : (k == 2 ? coef(rx, rt, 1) : -c.inv_dt));
        acc += cf * yJ(rx, rt);
    }
    b[n] = bdata[n] + c.qeps * acc;
}

// FEM Crank-Nicolson Burgers rows: half the convection of row x on one
// level, int phi_x v v_x / 2 = (v_(x+1) - v_(x-1))(v_(x+1) + v_x + v_(x-1)) / 12
__device__ __forceinline__ double fem_half_conv(const double* lev, int x) {
    return (lev[x + 1] - lev[x - 1]) * (lev[x + 1] + lev[x] + lev[x - 1]) * (1.0 / 12.0);
}

// b_J = J^T Q_eps (J u - f(u)) for the FEM Crank-Nicolson Burgers rows: the
// convection is homogeneous of degree 2, so J u - f(u) of row (x, t) is the
// sum of its two half convections
__global__ void k_gn_rhs_fem(const LevelView<double> L, const double* __restrict__ u, const double* __restrict__ bdata,
                             double* __restrict__ b) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= L.N) return;
    const int nx = L.nx, nt = L.nt;
    const int x = (int)(n % nx), t = (int)(n / nx);
    auto mu_at = [&](int xx, int tt) { return u[(long long)tt * nx + xx]; };
    int rxs[6], rts[6];
    double cfs[6];
    const int nr = fem_cn_column(L.col, nx, nt, x, t, mu_at, rxs, rts, cfs);
    double acc = 0.0;
    for (int k = 0; k < nr; ++k) {
        const double* lk = u + (long long)rts[k] * nx;
        acc += cfs[k] * (fem_half_conv(lk, rxs[k]) + fem_half_conv(lk - nx, rxs[k]));
    }
    b[n] = bdata[n] + L.col.qeps * acc;
}

// sum over collocation rows of f(v)^2 (FP64), per-CTA partials
__global__ void k_colloc_misfit(const LevelView<double> L, double nu, const double* __restrict__ v, double* __restrict__ part) {
    const int nx = L.nx, nt = L.nt;
    const long long nrow = (long long)(nx - 2) * (nt - 1);
    const long long r = (long long)blockIdx.x * 256 + threadIdx.x;
    double s = 0.0;
    if (r < nrow && colloc_on(L.col, 1 + (int)(r % (nx - 2)), 1 + (int)(r / (nx - 2)))) {
        const int x = 1 + (int)(r % (nx - 2)), t = 1 + (int)(r / (nx - 2));
        const long long i = (long long)t * nx + x;
        const double h = 0.5 / L.col.inv_2h;
        double f;
        if (L.col.kind == 4) {
            // int phi_x (v^t - v^(t-1))/dt + 1/2 sum over both levels of (convection + nu stiffness)
            const double* a = v + (long long)t * nx;
            const double* p = a - nx;
            const double m = L.col.m6_dt, k = L.col.nu_2h;
            f = m * ((a[x - 1] - p[x - 1]) + 4.0 * (a[x] - p[x]) + (a[x + 1] - p[x + 1])) + fem_half_conv(a, x) +
                fem_half_conv(p, x) + k * (2.0 * a[x] - a[x - 1] - a[x + 1]) + k * (2.0 * p[x] - p[x - 1] - p[x + 1]);
        } else {
            f = (v[i] - v[i - nx]) * L.col.inv_dt + v[i] * (v[i + 1] - v[i - 1]) * L.col.inv_2h -
                nu * (v[i + 1] - 2.0 * v[i] + v[i - 1]) / (h * h);
        }
        s = f * f;
    }
    double sv[4] = {s, 0.0, 0.0, 0.0};
    block_sum4<256, double>(sv, part + (size_t)blockIdx.x * 4);
}

// sum over observation rows (point data, IC rows) of rinv (y - A v)^2
__global__ void k_obs_misfit(const ObsRow* __restrict__ obs, int nobs, const double* __restrict__ ypoint, int m,
                             const double* __restrict__ yic, const double* __restrict__ v, double* __restrict__ part) {
    const int k = blockIdx.x * 256 + threadIdx.x;
    double s = 0.0;
    if (k < nobs) {
        const ObsRow& o = obs[k];
        double av = 0.0;
        for (int n = 0; n < o.nn; ++n) av += o.wd[n] * v[o.node[n]];
        const double y = o.row < m ? ypoint[o.row] : yic[o.row - m];
        s = o.rinv * (y - av) * (y - av);
    }
    double sv[4] = {s, 0.0, 0.0, 0.0};
    block_sum4<256, double>(sv, part + (size_t)blockIdx.x * 4);
}

__global__ void k_dot1(const double* __restrict__ a, const double* __restrict__ b, long long N, double* __restrict__ part) {
    double s = 0.0;
    for (long long n = (long long)blockIdx.x * 256 + threadIdx.x; n < N; n += (long long)gridDim.x * 256) s += a[n] * b[n];
    double sv[4] = {s, 0.0, 0.0, 0.0};
    block_sum4<256, double>(sv, part + (size_t)blockIdx.x * 4);
}

__global__ void k_axpy1(const double* __restrict__ u, double alpha, const double* __restrict__ d, double* __restrict__ v,
                        long long N) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n < N) v[n] = u[n] + alpha * d[n];
}

// one vector <-> slot 0 of a one-block batch
__global__ void k_to_slot0(const double* __restrict__ v, double* __restrict__ b, long long N) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    b[n * 4] = v[n];
    b[n * 4 + 1] = 0.0;
    b[n * 4 + 2] = 0.0;
    b[n * 4 + 3] = 0.0;
}
__global__ void k_from_slot0(const double* __restrict__ b, double* __restrict__ v, long long N) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n < N) v[n] = b[n * 4];
}
__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out, long long N) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n < N) out[n] = a[n] - b[n];
}

unsigned blocks_of(long long n) { return (unsigned)((n + 255) / 256); }

double reduce_host(Workspace& W, const double* part, int nparts, cudaStream_t s) {
    launch_reduce(part, nparts, 1, W.red, s);
    GCK(cudaMemcpyAsync(W.h_red, W.red, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    GCK(cudaStreamSynchronize(s));
    return W.h_red[0];
}

// linear interpolation of a fine-grid function (nx_f x nt_f, same domain) at the nodes of a coarse grid
void interpolate_level(const std::vector<double>& f, int nxf, int ntf, int nxc, int ntc, std::vector<double>& c) {
    c.assign((size_t)nxc * ntc, 0.0);
    for (int t = 0; t < ntc; ++t) {
        const double st = ntc > 1 ? (double)t * (ntf - 1) / (ntc - 1) : 0.0;
        int kt = std::min((int)std::floor(st), std::max(ntf - 2, 0));
        const double wt = ntf > 1 ? st - kt : 0.0;
        for (int x = 0; x < nxc; ++x) {
            const double sx = (double)x * (nxf - 1) / (nxc - 1);
            const int kx = std::min((int)std::floor(sx), nxf - 2);
            const double wx = sx - kx;
            auto F = [&](int a, int b) { return f[(size_t)b * nxf + a]; };
            double v = (1 - wx) * (1 - wt) * F(kx, kt) + wx * (1 - wt) * F(kx + 1, kt);
            if (ntf > 1) v += (1 - wx) * wt * F(kx, kt + 1) + wx * wt * F(kx + 1, kt + 1);
            c[(size_t)t * nxc + x] = v;
        }
    }
}

}  // namespace

// Linearises the Burgers collocation rows at u (device, [N]) on every level
// and refreshes the smoother and coarse-level data.
void linearise(Posterior& P, const double* u, cudaStream_t s) {
    Level& F = P.levels[0];
    std::vector<double> uf((size_t)F.N);
    GCK(cudaMemcpyAsync(uf.data(), u, sizeof(double) * F.N, cudaMemcpyDeviceToHost, s));
    GCK(cudaStreamSynchronize(s));
    for (size_t l = 0; l < P.levels.size(); ++l) {
        Level& L = P.levels[l];
        std::vector<double> ul;
        if (l == 0) ul = uf;
        else interpolate_level(uf, F.nx, F.nt, L.nx, L.nt, ul);
        std::vector<float> u32(ul.size());
        for (size_t i = 0; i < ul.size(); ++i) u32[i] = (float)ul[i];
        GCK(cudaMemcpyAsync(L.d_mu64, ul.data(), sizeof(double) * ul.size(), cudaMemcpyHostToDevice, s));
        GCK(cudaMemcpyAsync(L.d_mu32, u32.data(), sizeof(float) * u32.size(), cudaMemcpyHostToDevice, s));
        GCK(cudaStreamSynchronize(s));
        L.col.kind = P.colloc_kind;     // 2: collocation, 4: FEM Crank-Nicolson rows
    }
    for (auto& kv : P.ws) {       // captured graphs hold the old coefficients by value
        for (Workspace::Vecs* V : {&kv.second->v32, &kv.second->v64}) {
            if (V->exec) cudaGraphExecDestroy(V->exec);
            if (V->graph) cudaGraphDestroy(V->graph);
            V->exec = nullptr;
            V->graph = nullptr;
            V->graph_tol = -1.0;
        }
        solve_graph_free(kv.second->sgraph);     // the device-driven solve bakes the same coefficients
        kv.second->sgraph = nullptr;
    }
    posterior_refresh_operator(P, s);
    P.use_tsp = tsp_applicable(F, (int)P.nic);
    if (P.use_tsp) tsp_prepare(F, (int)P.nic, s);
    // data right-hand side of the linearised problem, b_lin = A^T R^-1 y + J^T Q_eps (J u - f(u));
    // at a Gauss-Newton fixed point H^-1 b_lin = u, so the mean slot of later
    // sampling calls is the Laplace mean
    if (!P.d_blin) P.d_blin = dev_alloc<double>((size_t)F.N);
    if (P.colloc_kind == 4) k_gn_rhs_fem<<<blocks_of(F.N), 256, 0, s>>>(F.view<double>(), u, P.d_bdata, P.d_blin);
    else k_gn_rhs<<<blocks_of(F.N), 256, 0, s>>>(F.view<double>(), u, P.d_bdata, P.d_blin);
    note_launch();
    P.linearised = true;
}

// -log pi(v) of eq. nonlinear-post-density up to a constant (prior mean 0).
static double neg_log_post(Posterior& P, Workspace& W, const double* v, double* vb, double* tmp, cudaStream_t s) {
    Level& F = P.levels[0];
    const long long N = F.N;
    // 1/2 v^T Q_prior v: the fused stencil without observation or collocation rows
    k_to_slot0<<<blocks_of(N), 256, 0, s>>>(v, vb, N);
    note_launch();
    StencilArgs<double> a{};
    a.L = F.view<double>();
    a.L.ocap = 0;
    a.L.col.kind = 0;
    a.nblk = 1;
    a.x = vb;
    a.out = tmp;
    a.partial = W.partial;
    const int ng = launch_stencil<double>(F.geo, M_APPLY, a, s);
    double val = 0.5 * reduce_host(W, W.partial, ng, s);
    // observation rows (point data and initial condition)
    if (F.nobs > 0) {
        const unsigned nb = blocks_of(F.nobs);
        k_obs_misfit<<<nb, 256, 0, s>>>(F.d_obs, F.nobs, P.d_ypoint, (int)P.m, P.d_icvals, v, W.partial);
        note_launch();
        val += 0.5 * reduce_host(W, W.partial, (int)nb, s);
    }
    // nonlinear collocation rows
    const long long nrow = (long long)(F.nx - 2) * (F.nt - 1);
    const unsigned nb = blocks_of(nrow);
    k_colloc_misfit<<<nb, 256, 0, s>>>(F.view<double>(), P.colloc_nu, v, W.partial);
    note_launch();
    val += 0.5 * P.colloc_qeps * reduce_host(W, W.partial, (int)nb, s);
    return val;
}

static double dot1(Workspace& W, const double* a, const double* b, long long N, cudaStream_t s) {
    const unsigned nb = std::min<unsigned>(blocks_of(N), 2048);
    k_dot1<<<nb, 256, 0, s>>>(a, b, N, W.partial);
    note_launch();
    return reduce_host(W, W.partial, (int)nb, s);
}

GnResult gauss_newton_step(Posterior& P, double* u_io, double* d_io, bool u_dev, bool d_dev, const gmrf_solve_opts& o,
                           cudaStream_t s) {
    if (P.colloc_kind != 2 && P.colloc_kind != 4)
        throw Error(GMRF_E_INVALID, "gauss_newton_step needs Burgers rows (colloc = 2 or 4)");
    Level& F = P.levels[0];
    const long long N = F.N;
    Workspace& W = workspace(P, 1);
    if (!P.d_gn) P.d_gn = dev_alloc<double>((size_t)N * 6);
    double* u = P.d_gn;             // u_k
    double* d = P.d_gn + N;         // direction
    double* g = P.d_gn + 2 * N;     // -grad
    double* v = P.d_gn + 3 * N;     // trial point
    double* tmp = P.d_gn + 5 * N;
    GCK(cudaMemcpyAsync(u, u_io, sizeof(double) * N, u_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    GCK(cudaMemcpyAsync(d, d_io, sizeof(double) * N, d_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    linearise(P, u, s);
    // -grad = b_lin - H u
    k_to_slot0<<<blocks_of(N), 256, 0, s>>>(u, W.b64, N);
    note_launch();
    apply64(P, 1, W.b64, W.r64, s);
    k_from_slot0<<<blocks_of(N), 256, 0, s>>>(W.r64, tmp, N);
    note_launch();
    k_sub<<<blocks_of(N), 256, 0, s>>>(P.d_blin, tmp, g, N);
    note_launch();
    // H d = -grad, warm-started from the previous direction
    k_to_slot0<<<blocks_of(N), 256, 0, s>>>(g, W.b64, N);
    note_launch();
    k_to_slot0<<<blocks_of(N), 256, 0, s>>>(d, W.x64, N);
    note_launch();
    // The solve stops on its residual relative to the starting one.  Near the
    // mode the direction shrinks by orders of magnitude from step to step, so
    // b - H d_prev can be far larger than b and a stop relative to it far too
    // early: start from zero unless the previous direction reduces the
    // residual (both in the D^-1-weighted norm of the stopping test).
    {
        StencilArgs<double> a{};
        a.L = F.view<double>();
        a.nblk = 1;
        a.x = W.x64;
        a.b = W.b64;
        a.out = W.r64;
        a.partial = W.partial;
        a.rweight = F.d_dinv64;
        const int ng = launch_stencil<double>(F.geo, M_RESID, a, s);
        const double r0 = reduce_host(W, W.partial, ng, s);
        launch_norm2w(W.b64, F.d_dinv64, N, 1, W.partial, elem_parts(N), s);
        const double b0 = reduce_host(W, W.partial, elem_parts(N), s);
        if (!(r0 < b0)) GCK(cudaMemsetAsync(W.x64, 0, sizeof(double) * (size_t)N * 4, s));
    }
    GnResult res;
    res.stats = solve_blocked(P, 1, W.b64, W.x64, o, s);
    k_from_slot0<<<blocks_of(N), 256, 0, s>>>(W.x64, d, N);
    note_launch();
    // Newton decrement d^T H d
    apply64(P, 1, W.x64, W.r64, s);
    k_from_slot0<<<blocks_of(N), 256, 0, s>>>(W.r64, tmp, N);
    note_launch();
    res.decrement = dot1(W, d, tmp, N, s);
    // Armijo backtracking on -log pi: phi(u + a d) <= phi(u) + c1 a grad^T d
    const double slope = -dot1(W, g, d, N, s);
    const double phi0 = neg_log_post(P, W, u, W.b64, W.r64, s);
    double alpha = 1.0;
    for (int k = 0; k <= 20; ++k) {
        k_axpy1<<<blocks_of(N), 256, 0, s>>>(u, alpha, d, v, N);
        note_launch();
        const double phi = neg_log_post(P, W, v, W.b64, W.r64, s);
        if (phi <= phi0 + 1e-4 * alpha * slope) break;
        if (k == 20) break;
        alpha *= 0.5;
    }
    res.alpha = alpha;
    k_axpy1<<<blocks_of(N), 256, 0, s>>>(u, alpha, d, v, N);
    note_launch();
    GCK(cudaMemcpyAsync(u_io, v, sizeof(double) * N, u_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    GCK(cudaMemcpyAsync(d_io, d, sizeof(double) * N, d_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    // leave the operator linearised at the new point (Laplace approximation, Sec. 3.3)
    linearise(P, v, s);
    GCK(cudaStreamSynchronize(s));
    return res;
}

}  // namespace gmrf
