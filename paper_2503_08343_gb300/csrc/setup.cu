// Construction of the multigrid hierarchy: closed-form P1 stencils of the
// stacked prior root B on every level (Sec. 2.2, App. A, App. B), observation
// rows with their per-tile lists, Jacobi diagonals, Chebyshev bounds, grid
// transfers and the dense coarsest-level inverse.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <stdexcept>

#include "host.h"

namespace gmrf {

static const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// closed-form stencils of one level

// The P1 stiffness of the structured triangulation split along
// (i,j)->(i+1,j+1) is the 5-point stencil: centre 2hy/hx + 2hx/hy, x
// neighbours -hy/hx, y neighbours -hx/hy (the hypotenuse couplings vanish
// because the angle opposite a diagonal edge is right).  Lumped mass hx hy.
// The advection matrix int phi_i (c . grad phi_j) from the six triangles
// around a node: (cx hy/6)[x+1: 2, x-1: -2, (+1,+1): 1, (-1,-1): -1, y+1: -1,
// y-1: 1] + (cy hx/6)[y+1: 2, y-1: -2, (+1,+1): 1, (-1,-1): -1, x+1: -1, x-1: 1].
// In 1D: stiffness (1/h)[-1 2 -1], lumped mass h, advection c[-1/2 0 1/2].
struct SpatialOps {
    double M;
    double S[NTAP];
    double A[NTAP];
};

static SpatialOps spatial_ops(int dim, double hx, double hy, double cx, double cy) {
    SpatialOps o;
    std::memset(&o, 0, sizeof(o));
    if (dim == 1) {
        o.M = hx;
        o.S[0] = 2.0 / hx;
        o.S[1] = o.S[2] = -1.0 / hx;
        o.A[1] = -0.5 * cx;
        o.A[2] = 0.5 * cx;
        return o;
    }
    o.M = hx * hy;
    o.S[0] = 2.0 * hy / hx + 2.0 * hx / hy;
    o.S[1] = o.S[2] = -hy / hx;
    o.S[3] = o.S[4] = -hx / hy;
    const double ax = cx * hy / 6.0, ay = cy * hx / 6.0;
    o.A[2] = 2 * ax - ay;    // x+1
    o.A[1] = -2 * ax + ay;   // x-1
    o.A[6] = ax + ay;        // (+1,+1)
    o.A[5] = -ax - ay;       // (-1,-1)
    o.A[4] = -ax + 2 * ay;   // y+1
    o.A[3] = ax - 2 * ay;    // y-1
    return o;
}

static double matern_tau_unit(double kappa, int dim) {
    return dim == 1 ? 1.0 / std::sqrt(4.0 * kappa * kappa * kappa) : 1.0 / std::sqrt(4.0 * kPi * kappa * kappa);
}

void level_coefficients(const gmrf_prior_desc& d, Level& L) {
    std::memset(L.cd, 0, sizeof(L.cd));
    const bool st = d.kind == GMRF_ADVDIFF_ST_1D || d.kind == GMRF_ADVDIFF_ST_2D;
    const int dim = d.kind == GMRF_ADVDIFF_ST_1D ? 1 : 2;
    if (!st) {
        const bool mat = d.kind == GMRF_MATERN2_2D;
        const double nu = mat ? 1.0 : d.nu, cx = mat ? 0.0 : d.cx, cy = mat ? 0.0 : d.cy;
        const SpatialOps o = spatial_ops(2, L.hx, L.hy, cx, cy);
        const double s = d.tau / std::sqrt(o.M);
        for (int t = 0; t < NTAP; ++t) L.cd[0][t] = s * (nu * o.S[t] + o.A[t] + (t == 0 ? d.kappa * d.kappa * o.M : 0.0));
    } else {
        const SpatialOps o = spatial_ops(dim, L.hx, L.hy, d.cx, d.cy);
        const double dt = L.dt;
        const double dk = 1.0 / (d.tau * std::sqrt(dt) * std::sqrt(o.M));
        for (int t = 0; t < NTAP; ++t) L.cd[0][t] = dk * (dt * (d.nu * o.S[t] + o.A[t]) + (t == 0 ? o.M : 0.0));
        L.cd[0][7] = -(1.0 - d.decay) * dk * o.M;        // AR(1) decay of the previous level
        // Matern transition noise (1D): T_K = tau_s Ml^-1/2 K_s Ml^-1/2 with
        // K_s = kappa_s^2 Ml + S, lumped Ml = h: tau_s (kappa_s^2 + 2/h^2) on the
        // diagonal, -tau_s / h^2 to each x neighbour
        L.noise = d.noise_kappa > 0.0 ? 1 : 0;
        if (L.noise) {
            const double ts = matern_tau_unit(d.noise_kappa, dim);
            L.tk_c = ts * (d.noise_kappa * d.noise_kappa + 2.0 / (L.hx * L.hx));
            L.tk_o = -ts / (L.hx * L.hx);
        }
        const double d0 = (matern_tau_unit(d.kappa0, dim) / d.tau) / std::sqrt(o.M);
        for (int t = 0; t < NTAP; ++t) L.cd[1][t] = d0 * (o.S[t] + (t == 0 ? d.kappa0 * d.kappa0 * o.M : 0.0));
        L.cd[1][7] = 0.0;
    }
    L.inv_eps2 = 1.0 / d.eps2;
    L.inv_eps = 1.0 / std::sqrt(d.eps2);
}

// ---------------------------------------------------------------------------
// level geometry

int geometry_of(const gmrf_prior_desc& d) {
    if (d.kind == GMRF_ADVDIFF_ST_1D) return GEO_XT;
    if (d.kind == GMRF_ADVDIFF_ST_2D) return GEO_XYT;
    return GEO_XY;
}

static void set_spacing(const gmrf_prior_desc& d, Level& L) {
    // a torus of n nodes per axis has n intervals
    L.hx = (d.hi[0] - d.lo[0]) / (L.periodic ? L.nx : L.nx - 1);
    L.hy = L.ny > 1 ? (d.hi[1] - d.lo[1]) / (L.periodic ? L.ny : L.ny - 1) : 0.0;
    L.dt = L.nt > 1 ? (d.hi[2] - d.lo[2]) / (L.nt - 1) : 0.0;
    L.N = (long long)L.nx * L.ny * L.nt;
    L.tiles_x = (L.nx + geo_tx(L.geo) - 1) / geo_tx(L.geo);
    L.tiles_y = (L.ny + geo_ty(L.geo) - 1) / geo_ty(L.geo);
    L.tiles_t = (L.nt + geo_tt(L.geo) - 1) / geo_tt(L.geo);
}

// Full coarsening n -> (n - 1)/2 + 1 of every grid axis (time included)
// while a level has more than kCoarseMax nodes; an axis stops at 5 nodes.
static const long long kCoarseMax = 600;

// Periodic (x, y) torus: both axes halve together while both are even and at
// least 8 (the transfers are then the P1 / bilinear interpolation of the
// coarse torus and its transpose); the coarsest level may hold up to
// kCoarseMaxPeriodic nodes.
static const long long kCoarseMaxPeriodic = 1024;

void build_hierarchy(const gmrf_prior_desc& d, std::vector<Level>& levels) {
    levels.clear();
    Level L;
    L.geo = geometry_of(d);
    L.periodic = d.bc == GMRF_BC_PERIODIC ? 1 : 0;
    L.nx = d.nx; L.ny = d.ny; L.nt = d.nt;
    if (L.periodic) { L.nx = d.nx - 1; L.ny = d.ny - 1; }   // the nodes on x = hi, y = hi are mirrors
    set_spacing(d, L);
    level_coefficients(d, L);
    levels.push_back(L);
    if (L.periodic) {
        while (levels.back().N > kCoarseMax) {
            Level& f = levels.back();
            if (f.nx % 2 != 0 || f.ny % 2 != 0 || f.nx < 8 || f.ny < 8) break;
            Level c = f;
            c.nx = f.nx / 2;
            c.ny = f.ny / 2;
            f.coarsen[0] = f.coarsen[1] = true;
            f.coarsen[2] = false;
            c.coarsen[0] = c.coarsen[1] = c.coarsen[2] = false;
            set_spacing(d, c);
            level_coefficients(d, c);
            levels.push_back(c);
        }
        if (levels.back().N > kCoarseMaxPeriodic)
            throw Error(GMRF_E_INVALID, "periodic grid: nx - 1 and ny - 1 must halve (even, >= 8) down to at most " +
                                            std::to_string(kCoarseMaxPeriodic) + " coarsest nodes");
        return;
    }
    const bool ax[3] = {true, L.geo != GEO_XT, L.geo != GEO_XY};
    while (true) {
        Level& f = levels.back();
        if (f.N <= kCoarseMax) break;
        Level c = f;
        bool any = false;
        int* dims_f[3] = {&f.nx, &f.ny, &f.nt};
        int* dims_c[3] = {&c.nx, &c.ny, &c.nt};
        for (int a = 0; a < 3; ++a) {
            f.coarsen[a] = false;
            if (!ax[a] || *dims_f[a] < 9) continue;
            *dims_c[a] = (*dims_f[a] - 1) / 2 + 1;
            f.coarsen[a] = true;
            any = true;
        }
        if (!any) break;
        for (int a = 0; a < 3; ++a) c.coarsen[a] = false;
        set_spacing(d, c);
        level_coefficients(d, c);
        levels.push_back(c);
    }
}

// ---------------------------------------------------------------------------
// observation rows on one level

static void cell1d(double v, double lo, double hi, int n, int& i, double& w) {
    const double h = (hi - lo) / (n - 1);
    double f = std::floor((v - lo) / h);
    i = (int)std::min(std::max(f, 0.0), (double)(n - 2));
    w = (v - (lo + i * h)) / h;
}

// the same on a torus of n nodes (n intervals): the cell's right node is
// (i + 1) mod n
static void cell1d_torus(double v, double lo, double hi, int n, int& i, double& w) {
    const double h = (hi - lo) / n;
    double f = std::floor((v - lo) / h);
    i = (int)std::min(std::max(f, 0.0), (double)(n - 1));
    w = (v - (lo + i * h)) / h;
}

// P1 barycentric weights in space (lower triangle (i,j),(i+1,j),(i+1,j+1)
// when xi >= eta, upper (i,j),(i+1,j+1),(i,j+1) otherwise) times linear
// weights in time.
static void point_row(const gmrf_prior_desc& d, const Level& L, const double* c, ObsRow& o) {
    int nn = 0;
    auto push = [&](int x, int y, int t, double w) {
        if (w == 0.0) return;
        o.node[nn] = (int32_t)(((long long)t * L.ny + y) * L.nx + x);
        o.wd[nn] = w;
        o.wf[nn] = (float)w;
        ++nn;
    };
    if (L.geo == GEO_XT) {
        int i, k;
        double wx, wt;
        cell1d(c[0], d.lo[0], d.hi[0], L.nx, i, wx);
        cell1d(c[1], d.lo[2], d.hi[2], L.nt, k, wt);
        push(i, 0, k, (1 - wx) * (1 - wt));
        push(i + 1, 0, k, wx * (1 - wt));
        push(i, 0, k + 1, (1 - wx) * wt);
        push(i + 1, 0, k + 1, wx * wt);
    } else {
        int i, j, k = 0;
        double xi, eta, wt = 0.0;
        if (L.periodic) {
            cell1d_torus(c[0], d.lo[0], d.hi[0], L.nx, i, xi);
            cell1d_torus(c[1], d.lo[1], d.hi[1], L.ny, j, eta);
        } else {
            cell1d(c[0], d.lo[0], d.hi[0], L.nx, i, xi);
            cell1d(c[1], d.lo[1], d.hi[1], L.ny, j, eta);
        }
        int vx[3], vy[3];
        double w[3];
        if (xi >= eta) {
            vx[0] = i; vy[0] = j; w[0] = 1 - xi;
            vx[1] = i + 1; vy[1] = j; w[1] = xi - eta;
            vx[2] = i + 1; vy[2] = j + 1; w[2] = eta;
        } else {
            vx[0] = i; vy[0] = j; w[0] = 1 - eta;
            vx[1] = i + 1; vy[1] = j + 1; w[1] = xi;
            vx[2] = i; vy[2] = j + 1; w[2] = eta - xi;
        }
        if (L.periodic)      // a node on x = hi or y = hi is its mirror (App. B, N_k = 1)
            for (int a = 0; a < 3; ++a) {
                if (vx[a] == L.nx) vx[a] = 0;
                if (vy[a] == L.ny) vy[a] = 0;
            }
        if (L.geo == GEO_XYT) cell1d(c[2], d.lo[2], d.hi[2], L.nt, k, wt);
        for (int b = 0; b < (L.geo == GEO_XYT ? 2 : 1); ++b) {
            const double ft = L.geo == GEO_XYT ? (b ? wt : 1 - wt) : 1.0;
            for (int a = 0; a < 3; ++a) push(vx[a], vy[a], k + b, w[a] * ft);
        }
    }
    o.nn = nn;
    for (int n = nn; n < 8; ++n) { o.node[n] = o.node[0]; o.wd[n] = 0.0; o.wf[n] = 0.0f; }
}

void build_level_obs(const gmrf_prior_desc& d, const Posterior& P, const std::vector<double>& coords,
                     const std::vector<double>& rinv, Level& L, bool fine) {
    const int dimc = (L.geo == GEO_XYT) ? 3 : 2;
    std::vector<ObsRow>& rows = L.h_obs;
    rows.clear();
    rows.reserve((size_t)(P.m + P.nic));
    for (int64_t k = 0; k < P.m; ++k) {
        ObsRow o;
        std::memset(&o, 0, sizeof(o));
        point_row(d, L, &coords[(size_t)k * dimc], o);
        o.rinv = rinv[(size_t)k];
        o.rinvf = (float)o.rinv;
        o.row = (int32_t)k;
        rows.push_back(o);
    }
    // initial-condition rows: every t = 0 node of the fine grid, as point data
    if (P.nic > 0) {
        const double fhx = (d.hi[0] - d.lo[0]) / (d.nx - 1);
        const double fhy = d.ny > 1 ? (d.hi[1] - d.lo[1]) / (d.ny - 1) : 0.0;
        for (int64_t k = 0; k < P.nic; ++k) {
            ObsRow o;
            std::memset(&o, 0, sizeof(o));
            const int ix = (int)(k % d.nx), iy = (int)(k / d.nx);
            if (fine) {
                o.node[0] = (int32_t)(iy * L.nx + ix);
                o.wd[0] = 1.0;
                o.wf[0] = 1.0f;
                o.nn = 1;
                for (int n = 1; n < 8; ++n) o.node[n] = o.node[0];
            } else {
                double c[3] = {d.lo[0] + ix * fhx, d.lo[1] + iy * fhy, d.lo[2]};
                if (L.geo == GEO_XT) c[1] = d.lo[2];
                point_row(d, L, c, o);
            }
            o.rinv = rinv[(size_t)(P.m + k)];
            o.rinvf = (float)o.rinv;
            o.row = (int32_t)(P.m + k);
            rows.push_back(o);
        }
    }
    for (ObsRow& o : rows)
        for (int n = 0; n < 8; ++n) {
            const long long nd = o.node[n];
            o.ox[n] = (int16_t)(nd % L.nx);
            o.oy[n] = (int16_t)((nd / L.nx) % L.ny);
            o.ot[n] = (int16_t)(nd / ((long long)L.nx * L.ny));
        }
    L.nobs = (int)rows.size();
    // per-tile lists: an observation is listed in every tile holding one of its nodes
    const int TX = geo_tx(L.geo), TY = geo_ty(L.geo), TT = geo_tt(L.geo);
    const long long ntiles = L.ntiles();
    std::vector<int32_t> cnt((size_t)ntiles + 1, 0);
    std::vector<int32_t> tl;
    auto tiles_of = [&](const ObsRow& o, int32_t* out) {
        int m = 0;
        for (int n = 0; n < o.nn; ++n) {
            const long long nd = o.node[n];
            const int x = (int)(nd % L.nx);
            const long long r = nd / L.nx;
            const int y = (int)(r % L.ny), t = (int)(r / L.ny);
            const int32_t tix = (int32_t)(((long long)(t / TT) * L.tiles_y + y / TY) * L.tiles_x + x / TX);
            bool dup = false;
            for (int q = 0; q < m; ++q) dup |= out[q] == tix;
            if (!dup) out[m++] = tix;
        }
        return m;
    };
    int32_t tbuf[8];
    for (const ObsRow& o : rows) {
        const int m = tiles_of(o, tbuf);
        for (int q = 0; q < m; ++q) cnt[(size_t)tbuf[q] + 1]++;
    }
    for (long long t = 0; t < ntiles; ++t) cnt[(size_t)t + 1] += cnt[(size_t)t];
    std::vector<int32_t> idx((size_t)cnt[(size_t)ntiles]);
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
    for (size_t k = 0; k < rows.size(); ++k) {
        const int m = tiles_of(rows[k], tbuf);
        for (int q = 0; q < m; ++q) idx[(size_t)fill[(size_t)tbuf[q]]++] = (int32_t)k;
    }
    dev_upload(&L.d_obs, rows);
    dev_upload(&L.d_tile_ptr, cnt);
    dev_upload(&L.d_tile_idx, idx);
    build_obs_stencil(L);
}

// A^T R^-1 A = sum_k rinv_k w_k w_k^T as a per-node stencil: node i gets
// C[i][off(j - i)] += rinv_k w_ki w_kj for every pair of nodes of row k
// (FP64 sums), laid out per tile for the stencil kernel.
void build_obs_stencil(Level& L) {
    const int TX = geo_tx(L.geo), TY = geo_ty(L.geo), TT = geo_tt(L.geo), TN = TX * TY * TT;
    const int OC = obs_oc(L.geo);
    std::map<long long, std::vector<double>> C;
    for (const ObsRow& o : L.h_obs)
        for (int a = 0; a < o.nn; ++a) {
            std::vector<double>& c = C[o.node[a]];
            if (c.empty()) c.assign((size_t)OC, 0.0);
            for (int b = 0; b < o.nn; ++b) {
                int dx = o.ox[b] - o.ox[a], dy = o.oy[b] - o.oy[a];
                const int dt = o.ot[b] - o.ot[a];
                if (L.periodic) {      // neighbours across the seam of the torus
                    if (dx > 1) dx -= L.nx;
                    if (dx < -1) dx += L.nx;
                    if (dy > 1) dy -= L.ny;
                    if (dy < -1) dy += L.ny;
                }
                int idx;
                if (L.geo == GEO_XY) idx = (dy + 1) * 3 + (dx + 1);
                else if (L.geo == GEO_XT) idx = (dt + 1) * 3 + (dx + 1);
                else idx = ((dt + 1) * 3 + (dy + 1)) * 3 + (dx + 1);
                c[(size_t)idx] += o.rinv * o.wd[a] * o.wd[b];
            }
        }
    const long long ntiles = L.ntiles();
    std::vector<int> count((size_t)ntiles, 0);
    auto tile_of = [&](long long nd, int& local) {
        const int x = (int)(nd % L.nx);
        const long long r = nd / L.nx;
        const int y = (int)(r % L.ny), t = (int)(r / L.ny);
        local = ((t % TT) * TY + (y % TY)) * TX + (x % TX);
        return ((long long)(t / TT) * L.tiles_y + y / TY) * L.tiles_x + x / TX;
    };
    int cap = 0;
    for (auto& kv : C) {
        int local;
        const long long t = tile_of(kv.first, local);
        cap = std::max(cap, ++count[(size_t)t]);
    }
    // per tile: cap entries of OC coefficients, then the tile-local node of
    // each entry as int16 (-1 for unused entries)
    L.ocap = cap;
    L.ostride32 = ((cap * OC * 4 + cap * 2 + 15) / 16) * 16;
    L.ostride64 = ((cap * OC * 8 + cap * 2 + 15) / 16) * 16;
    std::vector<int16_t> map((size_t)ntiles * TN, (int16_t)-1);
    std::vector<float> e32((size_t)ntiles * L.ostride32 / 4, 0.0f);
    std::vector<double> e64((size_t)ntiles * L.ostride64 / 8, 0.0);
    const int16_t none = -1;
    for (long long t = 0; t < ntiles; ++t)
        for (int e = 0; e < cap; ++e) {
            std::memcpy(reinterpret_cast<char*>(e32.data()) + (size_t)t * L.ostride32 + (size_t)cap * OC * 4 + (size_t)e * 2, &none, 2);
            std::memcpy(reinterpret_cast<char*>(e64.data()) + (size_t)t * L.ostride64 + (size_t)cap * OC * 8 + (size_t)e * 2, &none, 2);
        }
    std::fill(count.begin(), count.end(), 0);
    for (auto& kv : C) {
        int local;
        const long long t = tile_of(kv.first, local);
        const int e = count[(size_t)t]++;
        map[(size_t)t * TN + local] = (int16_t)e;
        for (int a = 0; a < OC; ++a) {
            e32[(size_t)t * (L.ostride32 / 4) + (size_t)e * OC + a] = (float)kv.second[(size_t)a];
            e64[(size_t)t * (L.ostride64 / 8) + (size_t)e * OC + a] = kv.second[(size_t)a];
        }
        const int16_t nd = (int16_t)local;
        std::memcpy(reinterpret_cast<char*>(e32.data()) + (size_t)t * L.ostride32 + (size_t)cap * OC * 4 + (size_t)e * 2, &nd, 2);
        std::memcpy(reinterpret_cast<char*>(e64.data()) + (size_t)t * L.ostride64 + (size_t)cap * OC * 8 + (size_t)e * 2, &nd, 2);
    }
    dev_upload(&L.d_omap, map);
    dev_upload(&L.d_oent32, e32);
    dev_upload(&L.d_oent64, e64);
}

// ---------------------------------------------------------------------------
// grid transfers between level f and the next coarser level c

void build_transfer(Level& f, const Level& c) {
    const int nf[3] = {f.nx, f.ny, f.nt}, ncs[3] = {c.nx, c.ny, c.nt};
    if (f.periodic) {
        // torus n -> n / 2: fine i lies at coarse i / 2, between coarse
        // j = i / 2 and (j + 1) mod m with weight w = (i mod 2) / 2 of the
        // second (the kernels wrap j + 1); the restriction of periodic levels
        // gathers its fine nodes directly, so it needs no range tables
        for (int a = 0; a < 2; ++a) {
            const int n = nf[a];
            std::vector<int32_t> pj((size_t)n), zero((size_t)ncs[a], 0);
            std::vector<float> pw((size_t)n);
            std::vector<double> pwd((size_t)n);
            for (int i = 0; i < n; ++i) {
                pj[(size_t)i] = i / 2;
                pwd[(size_t)i] = 0.5 * (i % 2);
                pw[(size_t)i] = (float)pwd[(size_t)i];
            }
            dev_upload(&f.d_pj[a], pj);
            dev_upload(&f.d_pw[a], pw);
            dev_upload(&f.d_pwd[a], pwd);
            dev_upload(&f.d_rs[a], zero);
            dev_upload(&f.d_rc[a], zero);
        }
        return;
    }
    for (int a = 0; a < 3; ++a) {
        if (!f.coarsen[a]) continue;
        const int n = nf[a], m = ncs[a];
        std::vector<int32_t> pj((size_t)n);
        std::vector<float> pw((size_t)n);
        std::vector<double> pwd((size_t)n);
        for (int i = 0; i < n; ++i) {
            const double s = (double)i * (m - 1) / (double)(n - 1);
            int j = (int)std::floor(s);
            j = std::min(std::max(j, 0), m - 2);
            pj[(size_t)i] = j;
            pwd[(size_t)i] = s - j;
            pw[(size_t)i] = (float)(s - j);
        }
        std::vector<int32_t> rs((size_t)m, n), re((size_t)m, -1);
        for (int i = 0; i < n; ++i) {
            for (int J : {pj[(size_t)i], pj[(size_t)i] + 1}) {
                rs[(size_t)J] = std::min(rs[(size_t)J], i);
                re[(size_t)J] = std::max(re[(size_t)J], i);
            }
        }
        std::vector<int32_t> rc((size_t)m);
        for (int J = 0; J < m; ++J) {
            if (re[(size_t)J] < rs[(size_t)J]) { rs[(size_t)J] = 0; rc[(size_t)J] = 0; }
            else rc[(size_t)J] = re[(size_t)J] - rs[(size_t)J] + 1;
            if (a < 2 && rc[(size_t)J] > kRestrictMax)
                throw std::runtime_error("grid transfer: a coarse node collects more fine nodes than the restriction holds");
        }
        if (a < 2) {
            const int T = a == 0 ? kRestrictTX : kRestrictTY;
            int span = 0;
            for (int J0 = 0; J0 < m; J0 += T) {
                const int J1 = std::min(J0 + T, m) - 1;
                span = std::max(span, rs[(size_t)J1] + rc[(size_t)J1] - rs[(size_t)J0]);
            }
            f.rspan[a] = span;
        }
        dev_upload(&f.d_pj[a], pj);
        dev_upload(&f.d_pw[a], pw);
        dev_upload(&f.d_pwd[a], pwd);
        dev_upload(&f.d_rs[a], rs);
        dev_upload(&f.d_rc[a], rc);
    }
}

// ---------------------------------------------------------------------------
// dense coarsest operator (host, FP64) and its inverse

static void coll_coef(const Colloc& c, const double* mu, int nx, int x, int t, double& cC, double& cL, double& cR) {
    double a, da;
    if (c.kind == 1) { a = c.c; da = 0.0; }
    else {
        const double m0 = mu ? mu[(size_t)t * nx + x] : 0.0;
        const double ml = mu ? mu[(size_t)t * nx + x - 1] : 0.0, mr = mu ? mu[(size_t)t * nx + x + 1] : 0.0;
        a = m0;
        da = (mr - ml) * c.inv_2h;
    }
    cC = c.inv_dt + da + 2.0 * c.nu_h2;
    cL = -a * c.inv_2h - c.nu_h2;
    cR = a * c.inv_2h - c.nu_h2;
}

std::vector<double> dense_operator(const Level& L, const double* mu) {
    const long long n = L.N;
    std::vector<double> Q((size_t)(n * n), 0.0);
    auto dir = [&](int x, int y) {
        return !L.periodic && (x == 0 || x == L.nx - 1 || (L.ny > 1 && (y == 0 || y == L.ny - 1)));
    };
    std::vector<std::vector<std::pair<long long, double>>> rows((size_t)n);
    for (long long r = 0; r < n; ++r) {
        const int x = (int)(r % L.nx);
        const long long q = r / L.nx;
        const int y = (int)(q % L.ny), t = (int)(q / L.ny);
        std::vector<std::pair<long long, double>>& row = rows[(size_t)r];
        if (dir(x, y)) {
            row.push_back({r, L.inv_eps});
        } else {
            const int cls = (L.nt > 1 && t == 0) ? 1 : 0;
            for (int o = 0; o < NTAP; ++o) {
                const double c = L.cd[cls][o];
                if (c == 0.0) continue;
                int xx = x + tap_dx(o), yy = y + tap_dy(o);
                const int tt = t + tap_dt(o);
                if (L.periodic) {
                    xx = (xx + L.nx) % L.nx;
                    yy = (yy + L.ny) % L.ny;
                }
                if (xx < 0 || xx >= L.nx || yy < 0 || yy >= L.ny || tt < 0 || tt >= L.nt) continue;
                if (dir(xx, yy)) continue;
                row.push_back({((long long)tt * L.ny + yy) * L.nx + xx, c});
            }
        }
    }
    if (L.noise) {          // B = T_K B_w: interior rows of levels >= 1 mix with their x neighbours
        std::vector<std::vector<std::pair<long long, double>>> out = rows;
        for (long long r = 0; r < n; ++r) {
            const int x = (int)(r % L.nx), t = (int)(r / ((long long)L.nx * L.ny));
            if (t < 1 || x < 1 || x > L.nx - 2) continue;
            std::map<long long, double> acc;
            for (auto& e : rows[(size_t)r]) acc[e.first] += L.tk_c * e.second;
            if (x - 1 >= 1) for (auto& e : rows[(size_t)(r - 1)]) acc[e.first] += L.tk_o * e.second;
            if (x + 1 <= L.nx - 2) for (auto& e : rows[(size_t)(r + 1)]) acc[e.first] += L.tk_o * e.second;
            out[(size_t)r].assign(acc.begin(), acc.end());
        }
        rows.swap(out);
    }
    for (auto& row : rows)
        for (auto& a : row)
            for (auto& b : row) Q[(size_t)(a.first * n + b.first)] += a.second * b.second;
    for (const ObsRow& o : L.h_obs)
        for (int a = 0; a < o.nn; ++a)
            for (int b = 0; b < o.nn; ++b) Q[(size_t)o.node[a] * n + o.node[b]] += o.rinv * o.wd[a] * o.wd[b];
    if (L.col.kind >= 3) {         // FEM Crank-Nicolson rows: six taps each
        auto mu_at = [&](int xx, int tt) { return mu ? mu[(size_t)tt * L.nx + xx] : 0.0; };
        for (int t = 1; t < L.nt; ++t)
            for (int x = 1; x < L.nx - 1; ++x) {
                if (!colloc_on(L.col, x, t)) continue;
                double a[3], b[3];
                fem_cn_row(L.col, x, t, mu_at, a, b);
                long long nd[6];
                double cv[6];
                for (int e = 0; e < 3; ++e) {
                    nd[e] = (long long)t * L.nx + x + e - 1;
                    cv[e] = a[e];
                    nd[3 + e] = (long long)(t - 1) * L.nx + x + e - 1;
                    cv[3 + e] = b[e];
                }
                for (int i = 0; i < 6; ++i)
                    for (int j = 0; j < 6; ++j) Q[(size_t)(nd[i] * n + nd[j])] += L.col.qeps * cv[i] * cv[j];
            }
    } else if (L.col.kind != 0) {
        for (int t = 1; t < L.nt; ++t)
            for (int x = 1; x < L.nx - 1; ++x) {
                if (!colloc_on(L.col, x, t)) continue;
                double cC, cL, cR;
                coll_coef(L.col, mu, L.nx, x, t, cC, cL, cR);
                const long long nd[4] = {(long long)t * L.nx + x, (long long)t * L.nx + x - 1, (long long)t * L.nx + x + 1,
                                         (long long)(t - 1) * L.nx + x};
                const double cv[4] = {cC, cL, cR, -L.col.inv_dt};
                for (int a = 0; a < 4; ++a)
                    for (int b = 0; b < 4; ++b) Q[(size_t)(nd[a] * n + nd[b])] += L.col.qeps * cv[a] * cv[b];
            }
    }
    return Q;
}

// In-place inverse of an SPD matrix by Cholesky; false if not positive definite.
bool spd_inverse(std::vector<double>& A, int n) {
    std::vector<double> L((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) return false;
        const double ljj = std::sqrt(s);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / ljj;
        }
    }
    // inverse of L (lower), then A^-1 = L^-T L^-1
    std::vector<double> Li((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        Li[(size_t)j * n + j] = 1.0 / L[(size_t)j * n + j];
        for (int i = j + 1; i < n; ++i) {
            double s = 0.0;
            for (int k = j; k < i; ++k) s += L[(size_t)i * n + k] * Li[(size_t)k * n + j];
            Li[(size_t)i * n + j] = -s / L[(size_t)i * n + i];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = 0.0;
            for (int k = i; k < n; ++k) s += Li[(size_t)k * n + i] * Li[(size_t)k * n + j];
            A[(size_t)i * n + j] = s;
            A[(size_t)j * n + i] = s;
        }
    return true;
}

}  // namespace gmrf
