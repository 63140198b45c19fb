// Internal structures of the GMRF library (host and device views).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "gmrf.h"

namespace gmrf {

// One observation row on one grid level: up to 8 nodes with interpolation
// weights (P1 barycentric in space x linear in time), its precision 1/sigma^2
// and its global row index (for the Philox draws of perturbation samples).
struct ObsRow {
    int32_t node[8];
    int16_t ox[8], oy[8], ot[8];   // grid coordinates of the nodes
    double wd[8];
    float wf[8];
    double rinv;
    float rinvf;
    int32_t nn;
    int32_t row;
    int32_t pad;
};

// Collocation rows J (Sec. 3.1 collocation; Sec. 3.3 Burgers): at interior
// x and time levels >= 1, coefficients
//   centre 1/dt + da + 2 nu/h^2, x-1: -a/(2h) - nu/h^2, x+1: a/(2h) - nu/h^2,
//   t-1: -1/dt, with a = c (linear) or a = u_k(x) and da = (u_k(x+1) - u_k(x-1))/(2h)
//   (Burgers, linearised at u_k).
//
// FEM rows with Crank-Nicolson in time (kinds 3 and 4; Sec. 3.1 FEM
// observations, A_ij = int phi_i D phi_j, exact integrals of the P1
// interpolant): row (x, k) has taps x-1, x, x+1 on level k (a) and on level
// k-1 (b),
//   a_e =  (h/6dt) [1 4 1]_e + (nu/2h) [-1 2 -1]_e + d_e(level k),
//   b_e = -(h/6dt) [1 4 1]_e + (nu/2h) [-1 2 -1]_e + d_e(level k-1),
// half the convection derivative d: linear c/4 [-1 0 1]; Burgers, from
// int phi_i v v_x = (v_(x+1) - v_(x-1))(v_(x+1) + v_x + v_(x-1))/6 linearised
// at u_k: [-(2u_(x-1) + u_x), u_(x+1) - u_(x-1), 2u_(x+1) + u_x] / 12.
struct Colloc {
    int kind;          // 0 none, 1 linear, 2 Burgers, 3 linear FEM Crank-Nicolson, 4 Burgers FEM Crank-Nicolson
    double qeps;       // 1 / sigma^2, scaled on coarse levels by the row-count ratio
    double inv_dt, inv_2h, nu_h2, c;
    double m6_dt;      // h / (6 dt)   (FEM rows)
    double nu_2h;      // nu / (2 h)   (FEM rows)
    int32_t row0;      // global observation row of the first collocation row
    int32_t sx, st;    // rows observe the PDE where x % sx == 0 and t % st == 0 (1, 1: every row)
};

// row (x, t) of the collocation rows observes the PDE (the others have zero
// weight; they keep their place in the row numbering)
__host__ __device__ __forceinline__ bool colloc_on(const Colloc& c, int x, int t) {
    return (c.sx <= 1 || x % c.sx == 0) && (c.st <= 1 || t % c.st == 0);
}

// half convection derivative d_e of an FEM Crank-Nicolson row centred at x,
// from the linearisation point at x-1, x, x+1 on one level
template <typename T>
__host__ __device__ __forceinline__ void fem_cn_half_conv(const Colloc& c, T ul, T u0, T ur, T d[3]) {
    if (c.kind == 3) {
        const T q = (T)(0.25 * c.c);
        d[0] = -q; d[1] = T(0); d[2] = q;
    } else {
        const T k = T(1) / T(12);
        d[0] = -(T(2) * ul + u0) * k;
        d[1] = (ur - ul) * k;
        d[2] = (T(2) * ur + u0) * k;
    }
}

// the FEM Crank-Nicolson rows touching node (x, t) and the coefficient of
// the node in each: rows (x+d, t) by their tap -d on their own level, rows
// (x+d, t+1) by their tap -d on the level before; mu(x, t) reads the
// linearisation point (kind 4).  Returns the number of rows (<= 6).
template <typename MU>
__host__ __device__ inline int fem_cn_column(const Colloc& c, int nx, int nt, int x, int t, MU mu, int rx[6], int rt[6],
                                             double cf[6]);

// the fixed part of tap e: sign * (h/6dt) [1 4 1]_e + (nu/2h) [-1 2 -1]_e
// (sign +1 on the row's own level, -1 on the level before)
template <typename T>
__host__ __device__ __forceinline__ T fem_cn_fixed(const Colloc& c, int e, T sign) {
    const T m = (T)c.m6_dt * (e == 1 ? T(4) : T(1));
    const T k = (T)c.nu_2h * (e == 1 ? T(2) : T(-1));
    return sign * m + k;
}

template <typename MU>
__host__ __device__ inline int fem_cn_column(const Colloc& c, int nx, int nt, int x, int t, MU mu, int rx[6], int rt[6],
                                             double cf[6]) {
    int n = 0;
    for (int d = -1; d <= 1; ++d) {
        const int r = x + d;
        if (r < 1 || r > nx - 2) continue;
        const bool on_t = t >= 1 && colloc_on(c, r, t), on_t1 = t + 1 <= nt - 1 && colloc_on(c, r, t + 1);
        if (!on_t && !on_t1) continue;
        double hd[3];
        fem_cn_half_conv<double>(c, c.kind == 4 ? mu(r - 1, t) : 0.0, c.kind == 4 ? mu(r, t) : 0.0,
                                 c.kind == 4 ? mu(r + 1, t) : 0.0, hd);
        if (on_t) { rx[n] = r; rt[n] = t; cf[n] = fem_cn_fixed<double>(c, 1 - d, 1.0) + hd[1 - d]; ++n; }
        if (on_t1) { rx[n] = r; rt[n] = t + 1; cf[n] = fem_cn_fixed<double>(c, 1 - d, -1.0) + hd[1 - d]; ++n; }
    }
    return n;
}

// the six taps of FEM Crank-Nicolson row (x, t): a on level t at x-1, x, x+1,
// b on level t-1
template <typename MU>
__host__ __device__ inline void fem_cn_row(const Colloc& c, int x, int t, MU mu, double a[3], double b[3]) {
    double dk[3], dp[3];
    const bool bu = c.kind == 4;
    fem_cn_half_conv<double>(c, bu ? mu(x - 1, t) : 0.0, bu ? mu(x, t) : 0.0, bu ? mu(x + 1, t) : 0.0, dk);
    fem_cn_half_conv<double>(c, bu ? mu(x - 1, t - 1) : 0.0, bu ? mu(x, t - 1) : 0.0, bu ? mu(x + 1, t - 1) : 0.0, dp);
    for (int e = 0; e < 3; ++e) {
        a[e] = fem_cn_fixed<double>(c, e, 1.0) + dk[e];
        b[e] = fem_cn_fixed<double>(c, e, -1.0) + dp[e];
    }
}

// Everything a stencil kernel needs about one level, passed by value.
template <typename T>
struct LevelView {
    int nx, ny, nt;
    long long N;
    int tiles_x, tiles_y, tiles_t;
    T cf[2][NTAP];     // B taps: class 0 = interior (t >= 1 in space-time), class 1 = t = 0
    T inv_eps2;        // Q_kk of a Dirichlet node
    T inv_eps;         // B_kk of a Dirichlet node
    Colloc col;
    const T* mu;       // linearisation point (Burgers), [N] or null
    const ObsRow* obs;
    const int32_t* tile_ptr;
    const int32_t* tile_idx;
    // A^T R^-1 A as a per-node 3^k-point stencil in tile-local tables:
    // omap[tile][node in tile] = entry index or -1; the tile's block of oent
    // holds [entry][OC] coefficients, then int16 node[entry] (-1: unused)
    const int16_t* omap;
    const T* oent;
    int ocap;          // entries per tile (0: no observation rows)
    int ostride;       // bytes per tile of oent (multiple of 16)
    int obs_direct;    // 1: read the tables from global memory instead of staging them (set per launch)
    int periodic;      // 1: the (x, y) torus of a periodic prior (no Dirichlet nodes, neighbours wrap)
    int noise;         // 1: Matern transition noise, B = T_K B_w (1D space-time)
    T tk_c, tk_o;      // T_K between interior rows of levels >= 1: diagonal, x neighbours
};

struct Level {
    int geo = 0;
    int periodic = 0;  // (x, y) torus: nx, ny count the torus nodes, h = (hi - lo) / nx
    int noise = 0;     // Matern transition noise (1D space-time): B = T_K B_w
    double tk_c = 1.0, tk_o = 0.0;
    int nx = 1, ny = 1, nt = 1;
    long long N = 0;
    double hx = 0, hy = 0, dt = 0;
    double cd[2][NTAP] = {};
    double inv_eps2 = 0, inv_eps = 0;
    Colloc col = {};
    int tiles_x = 1, tiles_y = 1, tiles_t = 1;
    // observation rows of this level and their per-tile lists (device)
    int nobs = 0;
    ObsRow* d_obs = nullptr;
    int32_t* d_tile_ptr = nullptr;
    int32_t* d_tile_idx = nullptr;
    std::vector<ObsRow> h_obs;
    int16_t* d_omap = nullptr;
    float* d_oent32 = nullptr;
    double* d_oent64 = nullptr;
    int ocap = 0;
    int ostride32 = 0, ostride64 = 0;
    // linearisation point on this level (Burgers), device
    float* d_mu32 = nullptr;
    double* d_mu64 = nullptr;
    // inverse Jacobi diagonal of Q_u|y, device
    float* d_dinv32 = nullptr;
    double* d_dinv64 = nullptr;
    double* d_diag64 = nullptr;
    // Chebyshev smoother on D^-1 Q: lambda_max estimate
    double lmax = 0;
    // grid transfer to the next coarser level, per axis (device):
    // prolongation: fine i -> coarse j(i), weight w(i) of j(i)+1
    int32_t* d_pj[3] = {nullptr, nullptr, nullptr};
    float* d_pw[3] = {nullptr, nullptr, nullptr};
    double* d_pwd[3] = {nullptr, nullptr, nullptr};
    // restriction: coarse J -> fine range [rs(J), rs(J) + rc(J))
    int32_t* d_rs[3] = {nullptr, nullptr, nullptr};
    int32_t* d_rc[3] = {nullptr, nullptr, nullptr};
    bool coarsen[3] = {false, false, false};
    // largest fine span (x, y) under one restriction tile of kRestrictTX x
    // kRestrictTY coarse nodes (sizes the shared-memory tile)
    int rspan[2] = {0, 0};
    // time-stepping preconditioner factors (collocation levels), device
    float* d_tsp32 = nullptr;
    double* d_tsp64 = nullptr;
    int tsp_ic = 0;                // the initial condition is observed (level 0 of J_t: its rows)
    float* d_tspc32 = nullptr;     // per-row coupling coefficients (FEM rows, mixed PDE / prior rows)
    double* d_tspc64 = nullptr;
    // coarsest level: dense inverse of Q_u|y (device, row-major)
    float* d_dense32 = nullptr;
    double* d_dense64 = nullptr;

    template <typename T> LevelView<T> view() const;
    long long ntiles() const { return (long long)tiles_x * tiles_y * tiles_t; }
};

struct Prior {
    gmrf_prior_desc desc;
    cudaStream_t stream = 0;
    int geo = 0;
    std::vector<Level> levels;   // rebuilt per posterior (observations differ); geometry here
    // exact log det Q and prior trace terms (computed on first use)
    std::mutex det_mu;
    bool det_ready = false;
    double det_logdet = 0.0;
    double det_tr[4] = {0, 0, 0, 0};
};

struct Workspace;
struct SolveGraph;

constexpr double kP1DataShare = 0.5;
constexpr int kRestrictTX = 32, kRestrictTY = 8;
// fine nodes under one coarse node per axis that the plane restriction keeps
// in registers (full coarsening n -> (n - 1)/2 + 1 with n >= 9 gives at most 5)
constexpr int kRestrictMax = 8;

struct Posterior {
    Prior* prior = nullptr;
    std::vector<Level> levels;
    int64_t m = 0;                 // point observations
    int64_t nic = 0;               // initial-condition rows
    int64_t ncol = 0;              // collocation rows on the fine level
    int64_t nrows = 0;             // all observation rows
    std::vector<double> y_point;   // point data values (host)
    std::vector<double> ic_values;
    std::vector<double> colloc_f;
    double* d_bdata = nullptr;     // A^T Q_eps y on the fine level, [N]
    double* d_ypoint = nullptr;
    double* d_bstatic = nullptr;   // IC + linear collocation part of b, [N]
    double* d_icvals = nullptr;    // initial-condition values (device), [nic]
    double* d_blin = nullptr;      // data RHS of the linearised (Gauss-Newton) problem, [N]
    double* d_gn = nullptr;        // Gauss-Newton work vectors, [6 N]
    std::map<int, Workspace*> ws;  // scratch per batch size (blocks of four right-hand sides)
    int colloc_kind = 0;           // requested collocation (2: Burgers, linearised on demand)
    double colloc_qeps = 0.0, colloc_nu = 0.0, colloc_c = 0.0;
    bool linearised = false;
    bool use_tsp = false;          // time-stepping preconditioner instead of the V-cycle
    // Grid transfers in the space plane: P1 interpolation on the triangulation
    // when observation rows dominate the diagonal of some fine-level node,
    // else bilinear.  With P1 transfers on nested grids the coarse space is a
    // subspace of the fine one, so point data rediscretised on a coarse level
    // equals its Galerkin projection; bilinear transfers break that
    // consistency and strongly observed problems then stall, while weakly
    // observed ones converge a little faster with the symmetric bilinear
    // transfer.
    double data_share = 0.0;       // max_n (obs part of diag_n) / diag_n, fine level
    bool transfer_p1 = false;
    double* d_grad_part = nullptr; // partial sums of the gradient contractions
    size_t grad_part_n = 0;
    double ic_rinv = 0.0;          // precision of the initial-condition rows
};

}  // namespace gmrf
