// Time-stepping preconditioner for collocation systems (1D space x time).
//
// With near-exact collocation (Sec. 3.1, 3.3) the posterior precision is
// dominated by Jt^T W Jt, where Jt stacks the initial-condition rows (t = 0),
// the Dirichlet rows of the prior at the spatial boundary and the
// collocation rows at interior nodes of levels k >= 1, with W their
// precisions.  Jt is square and block lower-bidiagonal in time (implicit
// Euler): level k reads level k (a tridiagonal stencil in x) and level k-1
// (-1/dt at the same x; FEM Crank-Nicolson rows: a tridiagonal stencil,
// whose coefficients k_tsp_couple stores).  Its inverse is one forward time sweep and Jt^-T one
// backward sweep, each level a tridiagonal solve, so
//     z = M r = Jt^-1 W^-1 Jt^-T r
// costs two sweeps and leaves the prior's interior part and the point data,
// both orders of magnitude smaller, to the outer conjugate gradients.
#include "handles.h"

namespace gmrf {

namespace {

// Each level's tridiagonal system (nx <= kLanes (kRows + 1) rows) is solved
// by the partition method over kLanes = 32 kWarps lanes of one CTA: lane l
// owns the contiguous rows [l m, l m + m), m = ceil(nx / kLanes); the last row
// of each chunk is a separator.  The chunk's interior rows are eliminated by a
// Thomas sweep with three right-hand sides, giving
// x_i = p_i + q_i X_{l-1} + r_i X_l in terms of the neighbouring separators;
// substituting into the separator rows leaves a kLanes-unknown tridiagonal
// system, one unknown per lane, solved by parallel cyclic reduction (warp
// shuffles for strides below 32, shared memory above); the interior rows
// follow by back-substitution.  Spreading a level over four warps keeps each
// lane's recurrences short (at most kRows rows): a level is a dependency
// chain, so its latency, not the throughput, sets the time.
//
// Everything that depends on the matrix alone (the Thomas pivots and
// multipliers, the interface columns q and r, the separator coefficients and
// the cyclic-reduction multipliers) is the same for every right-hand side and
// every application in a solve, so k_tsp_factor computes it once per
// linearisation, for every level and both sweep directions; an application
// (k_tsp) then runs only the right-hand-side recurrences, without divisions,
// on the four right-hand sides of one block at once (a lane carries them as
// one vector).  Each level's inputs and factors are staged in shared memory
// by cp.async one level ahead (double-buffered).
//
// Factors of one (direction, level), in elements of T:
//   row fields [5][kRows][kLanes] (field, chunk row j, lane): A_j/den_j,
//     1/den_j, c'_j (Thomas), Q_j, R_j (interface columns after
//     back-substitution);
//   lane fields [3 + 2 kSteps][kLanes]: separator A and C, 1 / final
//     diagonal, the cyclic-reduction multipliers k1 and k2 of every step.
constexpr int kWarps = 4, kLanes = 32 * kWarps, kSteps = 7;    // 2^kSteps = kLanes
constexpr int kRows = 8;                                        // interior rows per lane
constexpr int kTspMaxNx = kLanes * (kRows + 1);
constexpr int kRowF = 5, kLaneF = 3 + 2 * kSteps;
constexpr int kFactorBlock = kRowF * kRows * kLanes + kLaneF * kLanes;
// FEM Crank-Nicolson rows couple three nodes of the neighbouring level: per
// (direction, level) the coupling coefficients of every row, [3][kRows][kLanes]
// for the chunk rows and [3][kLanes] for the separators (x-1, x, x+1)
constexpr int kCplBlock = 3 * kRows * kLanes + 3 * kLanes;
static_assert((1 << kSteps) == kLanes, "cyclic reduction covers the lanes");

// The rows of J_t: boundary rows (the prior's Dirichlet rows), the initial
// level's data rows (the initial condition observed at every node) or, without
// them, the prior's initial-level rows, and on levels k >= 1 the PDE rows
// where the PDE is observed and the prior's transition rows elsewhere (rows
// between the collocation points, or every row without collocation).
enum TspRow { TR_BND = 0, TR_IC, TR_PRIOR0, TR_COL, TR_PRIOR };
template <typename T>
__device__ __forceinline__ int tsp_row_kind(const LevelView<T>& L, int x, int k, int has_ic) {
    if (x <= 0 || x >= L.nx - 1) return TR_BND;
    if (k == 0) return has_ic ? TR_IC : TR_PRIOR0;
    if (L.col.kind != 0 && colloc_on(L.col, x, k)) return TR_COL;
    return TR_PRIOR;
}

// Level row coefficients of J_t (lower x-1, diagonal, upper x+1) at node x of
// level k, with mu the linearisation point of the level (Burgers).  Prior rows
// are the white-noise root's rows (with Matern transition noise the weight of
// a level's prior rows is T_K^2 instead of one; see k_tsp_tscale).
template <typename T>
__device__ __forceinline__ void j_row(const LevelView<T>& L, const T* mu, int x, int k, int has_ic, T& lo, T& di,
                                      T& up) {
    const int nx = L.nx;
    const int kind = tsp_row_kind<T>(L, x, k, has_ic);
    if (kind == TR_BND || kind == TR_IC) { lo = T(0); di = T(1); up = T(0); return; }
    if (kind == TR_PRIOR0 || kind == TR_PRIOR) {    // the root's taps; Dirichlet columns eliminated
        const int cls = kind == TR_PRIOR0 ? 1 : 0;
        lo = x - 1 >= 1 ? L.cf[cls][1] : T(0);
        di = L.cf[cls][0];
        up = x + 1 <= nx - 2 ? L.cf[cls][2] : T(0);
        return;
    }
    const Colloc& c = L.col;
    if (c.kind >= 3) {         // FEM Crank-Nicolson row: its taps on its own level
        T d[3];
        fem_cn_half_conv<T>(c, mu ? mu[x - 1] : T(0), mu ? mu[x] : T(0), mu ? mu[x + 1] : T(0), d);
        lo = fem_cn_fixed<T>(c, 0, T(1)) + d[0];
        di = fem_cn_fixed<T>(c, 1, T(1)) + d[1];
        up = fem_cn_fixed<T>(c, 2, T(1)) + d[2];
        return;
    }
    T a, da;
    if (c.kind == 1) { a = (T)c.c; da = T(0); }
    else {
        a = mu[x];
        da = (mu[x + 1] - mu[x - 1]) * (T)c.inv_2h;
    }
    di = (T)c.inv_dt + da + T(2) * (T)c.nu_h2;
    lo = -a * (T)c.inv_2h - (T)c.nu_h2;
    up = a * (T)c.inv_2h - (T)c.nu_h2;
}

// Row x of the level system: J's level block D_k (TR = false) or its
// transpose (TR = true: sub-diagonal up(x-1), super-diagonal lo(x+1)).
template <typename T, bool TR>
__device__ __forceinline__ void level_row(const LevelView<T>& L, const T* mu, int x, int k, int has_ic, T& A, T& B, T& C) {
    T lo, di, up;
    j_row<T>(L, mu, x, k, has_ic, lo, di, up);
    B = di;
    if (!TR) { A = lo; C = up; return; }
    T l2, d2, u2;
    A = T(0);
    C = T(0);
    if (x > 0) { j_row<T>(L, mu, x - 1, k, has_ic, l2, d2, u2); A = u2; }
    if (x < L.nx - 1) { j_row<T>(L, mu, x + 1, k, has_ic, l2, d2, u2); C = l2; }
}

// One CTA of kLanes threads per (direction, level): the matrix-only part of
// the partition solve.  blockIdx.x = dir * nt + k, dir 0 = D_k (forward
// sweep), 1 = D_k^T.
template <typename T>
__global__ void __launch_bounds__(kLanes) k_tsp_factor(const LevelView<T> L, int has_ic, T* __restrict__ f) {
    __shared__ T xa[kLanes], xb[kLanes], xc[kLanes];
    const int nx = L.nx, nt = L.nt;
    const int dir = blockIdx.x / nt, k = blockIdx.x % nt;
    const int lane = threadIdx.x;
    const int m = (nx + kLanes - 1) / kLanes, s = lane * m, mi = max(0, min(m, nx - s)), mint = mi - 1;
    const T* mu = (L.col.kind == 2 || L.col.kind == 4) ? L.mu + (size_t)k * nx : nullptr;
    T* blk = f + (size_t)blockIdx.x * kFactorBlock;
    T* rowf = blk;                                   // [field][j][lane]
    T* lanef = blk + kRowF * kRows * kLanes;         // [field][lane]
    auto row = [&](int x, T& A, T& B, T& C) {
        if (dir == 0) level_row<T, false>(L, mu, x, k, has_ic, A, B, C);
        else level_row<T, true>(L, mu, x, k, has_ic, A, B, C);
    };
    T qv[kRows], rv[kRows], cv[kRows];
    T cprev = T(0), qprev = T(0);
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
        T ainv = T(0), inv = T(0), c = T(0), q = T(0), r = T(0);
        if (j < mint) {
            T A, B, C;
            row(s + j, A, B, C);
            inv = T(1) / (B - A * cprev);
            const bool last = j == mint - 1;
            ainv = A * inv;
            c = last ? T(0) : C * inv;
            q = (j == 0 ? -A : -A * qprev) * inv;
            r = last ? -C * inv : T(0);
            cprev = c;
            qprev = q;
        }
        rowf[(0 * kRows + j) * kLanes + lane] = ainv;
        rowf[(1 * kRows + j) * kLanes + lane] = inv;
        rowf[(2 * kRows + j) * kLanes + lane] = c;
        qv[j] = q;
        rv[j] = r;
        cv[j] = c;
    }
    T qn = T(0), rn = T(0), ql = T(1), rl = T(0);
#pragma unroll
    for (int j = kRows - 1; j >= 0; --j) {
        if (j < mint) {
            qv[j] = qv[j] - cv[j] * qn;
            rv[j] = rv[j] - cv[j] * rn;
            qn = qv[j];
            rn = rv[j];
            if (j == mint - 1) { ql = qv[j]; rl = rv[j]; }
        }
        rowf[(3 * kRows + j) * kLanes + lane] = j < mint ? qv[j] : T(0);
        rowf[(4 * kRows + j) * kLanes + lane] = j < mint ? rv[j] : T(0);
    }
    // separator row: A x_{e-2} + B X_l + C x_e, with x_{e-2} = p + ql X_{l-1} + rl X_l
    // (own last interior row) and x_e = p + qf X_l + rf X_{l+1} (next lane's first row)
    T qf = mint > 0 ? qv[0] : T(0), rf = mint > 0 ? rv[0] : T(1);
    if (mi <= 0) { qf = T(0); rf = T(0); }
    xa[lane] = qf;
    xb[lane] = rf;
    __syncthreads();
    const T qnx = lane + 1 < kLanes ? xa[lane + 1] : T(0), rnx = lane + 1 < kLanes ? xb[lane + 1] : T(0);
    __syncthreads();
    T Asep = T(0), Csep = T(0), ra = T(0), rb = T(1), rc = T(0);
    if (mi > 0) {
        T A, B, C;
        row(s + mi - 1, A, B, C);
        if (lane == kLanes - 1 || s + mi >= nx) C = T(0);
        if (mint == 0) { ql = T(1); rl = T(0); }
        if (s == 0 && mint == 0) ql = T(0);
        Asep = A;
        Csep = C;
        ra = lane == 0 ? T(0) : A * ql;      // lane 0 has no left separator
        rb = B + A * rl + C * qnx;
        rc = C * rnx;
    }
    lanef[0 * kLanes + lane] = Asep;
    lanef[1 * kLanes + lane] = Csep;
    int step = 0;
    for (int st = 1; st < kLanes; st <<= 1, ++step) {
        xa[lane] = ra;
        xb[lane] = rb;
        xc[lane] = rc;
        __syncthreads();
        const bool hm = lane - st >= 0, hp = lane + st < kLanes;
        const T am = hm ? xa[lane - st] : T(0), bm = hm ? xb[lane - st] : T(1), cm = hm ? xc[lane - st] : T(0);
        const T ap = hp ? xa[lane + st] : T(0), bp = hp ? xb[lane + st] : T(1), cp2 = hp ? xc[lane + st] : T(0);
        __syncthreads();
        const T k1 = hm ? ra / bm : T(0), k2 = hp ? rc / bp : T(0);
        const T na = hm ? -am * k1 : T(0), nc = hp ? -cp2 * k2 : T(0);
        const T nb = rb - (hm ? cm * k1 : T(0)) - (hp ? ap * k2 : T(0));
        ra = na;
        rb = nb;
        rc = nc;
        lanef[(3 + step) * kLanes + lane] = k1;
        lanef[(3 + kSteps + step) * kLanes + lane] = k2;
    }
    lanef[2 * kLanes + lane] = T(1) / rb;
}

// Coupling coefficients of every row of J_t to the neighbouring level (FEM
// Crank-Nicolson rows, mixed PDE and prior rows), one CTA of kLanes threads
// per (direction, level) like k_tsp_factor: the forward sweep at level k adds
// sum_e -b_e(x, k) z_(k-1)(x + e - 1) to row x's right-hand side (b: row
// (x, k)'s taps on level k-1); the backward sweep at level k adds
// sum_d -b_(1-d)(x + d, k + 1) y_(k+1)(x + d) (the transposed coupling, which
// also reaches the boundary nodes).  Stored as (x-1, x, x+1) coefficients.
template <typename T>
__global__ void __launch_bounds__(kLanes) k_tsp_couple(const LevelView<T> L, int has_ic, T* __restrict__ f) {
    const int nx = L.nx, nt = L.nt;
    const int dir = blockIdx.x / nt, k = blockIdx.x % nt;
    const int lane = threadIdx.x;
    const int m = (nx + kLanes - 1) / kLanes, s = lane * m, mi = max(0, min(m, nx - s)), mint = mi - 1;
    T* blk = f + (size_t)blockIdx.x * kCplBlock;
    const Colloc& c = L.col;
    // taps of row (x, kr) on level kr - 1 (zero unless x is interior and kr >= 1)
    auto btaps = [&](int x, int kr, T b[3]) {
        b[0] = b[1] = b[2] = T(0);
        if (x < 1 || x > nx - 2 || kr < 1 || kr >= nt) return;
        const int kind = tsp_row_kind<T>(L, x, kr, has_ic);
        if (kind == TR_PRIOR) { b[1] = L.cf[0][7]; return; }       // the root's t-1 tap
        if (c.kind == 1 || c.kind == 2) { b[1] = -(T)c.inv_dt; return; }   // implicit-Euler collocation row
        const T* mp = L.mu ? L.mu + (size_t)(kr - 1) * nx : nullptr;
        T d[3];
        fem_cn_half_conv<T>(c, mp ? mp[x - 1] : T(0), mp ? mp[x] : T(0), mp ? mp[x + 1] : T(0), d);
        for (int e = 0; e < 3; ++e) b[e] = fem_cn_fixed<T>(c, e, T(-1)) + d[e];
    };
    auto coeffs = [&](int x, T out[3]) {
        if (dir == 0) {
            T b[3];
            btaps(x, k, b);
            for (int e = 0; e < 3; ++e) out[e] = -b[e];
        } else {
            for (int d = -1; d <= 1; ++d) {
                T b[3];
                btaps(x + d, k + 1, b);
                out[d + 1] = -b[1 - d];
            }
        }
    };
    for (int j = 0; j < kRows; ++j) {
        T o[3] = {T(0), T(0), T(0)};
        if (j < mint) coeffs(s + j, o);
        for (int e = 0; e < 3; ++e) blk[(e * kRows + j) * kLanes + lane] = o[e];
    }
    T o[3] = {T(0), T(0), T(0)};
    if (mi > 0) coeffs(s + mi - 1, o);
    for (int e = 0; e < 3; ++e) blk[3 * kRows * kLanes + e * kLanes + lane] = o[e];
}

// One CTA (kLanes threads) per block of four right-hand sides.  y is scratch
// of the blocked layout; r and z are blocked.  Shared memory: factors
// [2][kFactorBlock], inputs [2][nx + kLanes] four-wide chunks laid out with one
// gap after each lane's chunk (x -> x + x / m: a lane reads its rows at
// base + j, and neighbouring lanes fall in distinct bank groups), the lane
// exchange buffers.
template <typename T, bool FEM>
__global__ void __launch_bounds__(kLanes) k_tsp(const LevelView<T> L, const T* __restrict__ fac, const T* __restrict__ cpl,
                                               T iw_ic, T iw_bnd, T iw_q, int has_ic, int sweep_lo, int sweep_hi,
                                               const T* __restrict__ r, T* __restrict__ y, T* __restrict__ z) {
    extern __shared__ __align__(16) unsigned char tsp_smem[];
    __shared__ V4<T> xch[2][kLanes];
    const int nx = L.nx, nt = L.nt;
    const long long N = L.N;
    const int NXC = nx + kLanes;                         // chunks per input row, gaps included
    T* sfac = reinterpret_cast<T*>(tsp_smem);            // [2][kFactorBlock]
    T* scpl = sfac + 2 * kFactorBlock;                   // FEM: [2][kCplBlock]
    V4<T>* sin = reinterpret_cast<V4<T>*>(scpl + (FEM ? 2 * kCplBlock : 0));   // [2][NXC]
    const int lane = threadIdx.x, wl = lane & 31;
    const int blk = blockIdx.x;
    const int m = (nx + kLanes - 1) / kLanes;
    const float rm = 1.0f / (float)m;
    const int s0 = lane * m, mi = max(0, min(m, nx - s0)), mint = mi - 1;
    const int ibase = s0 + lane;                         // this lane's first row in the staged layout
    const T inv_dt = (T)L.col.inv_dt;
    auto stage = [&](const T* src, int dir, int k, int slot) {
        if (k < 0 || k >= nt) return;
        const char* g = reinterpret_cast<const char*>(src + ((size_t)blk * N + (size_t)k * nx) * RW);
        V4<T>* d = sin + (size_t)slot * NXC;
        for (int x = lane; x < nx; x += kLanes) {
            int own = (int)((float)x * rm);          // x / m without an integer division
            own += (own + 1) * m <= x;
            own -= own * m > x;
            char* dx = reinterpret_cast<char*>(d + x + own);
            cp_async16(dx, g + (size_t)x * sizeof(V4<T>), true);
            if (sizeof(T) == 8) cp_async16(dx + 16, g + (size_t)x * sizeof(V4<T>) + 16, true);
        }
        const char* gf = reinterpret_cast<const char*>(fac + ((size_t)dir * nt + k) * kFactorBlock);
        char* df = reinterpret_cast<char*>(sfac + (size_t)slot * kFactorBlock);
        for (int c = lane; c < (int)(kFactorBlock * sizeof(T) / 16); c += kLanes) cp_async16(df + c * 16, gf + c * 16, true);
        if (FEM) {
            const char* gc = reinterpret_cast<const char*>(cpl + ((size_t)dir * nt + k) * kCplBlock);
            char* dc = reinterpret_cast<char*>(scpl + (size_t)slot * kCplBlock);
            for (int c = lane; c < (int)(kCplBlock * sizeof(T) / 16); c += kLanes) cp_async16(dc + c * 16, gc + c * 16, true);
        }
    };
    // four-wide exchange with the lane d below / above (shuffles within a warp,
    // shared memory across warps; every thread calls it)
    int xsel = 0;
    auto exch = [&](V4<T> v, int d, V4<T>& up, V4<T>& dn) {
        if (d < 32) {
            up = V4<T>{__shfl_up_sync(0xffffffffu, v.a, d), __shfl_up_sync(0xffffffffu, v.b, d),
                       __shfl_up_sync(0xffffffffu, v.c, d), __shfl_up_sync(0xffffffffu, v.d, d)};
            dn = V4<T>{__shfl_down_sync(0xffffffffu, v.a, d), __shfl_down_sync(0xffffffffu, v.b, d),
                       __shfl_down_sync(0xffffffffu, v.c, d), __shfl_down_sync(0xffffffffu, v.d, d)};
            // the neighbour lies in the next or previous warp: through shared memory
            const bool need_up = wl - d < 0 && lane - d >= 0, need_dn = wl + d >= 32 && lane + d < kLanes;
            xch[xsel][lane] = v;
            __syncthreads();
            if (need_up) up = xch[xsel][lane - d];
            if (need_dn) dn = xch[xsel][lane + d];
            if (lane - d < 0) up = v4zero<T>();
            if (lane + d >= kLanes) dn = v4zero<T>();
        } else {
            xch[xsel][lane] = v;
            __syncthreads();
            up = lane - d >= 0 ? xch[xsel][lane - d] : v4zero<T>();
            dn = lane + d < kLanes ? xch[xsel][lane + d] : v4zero<T>();
        }
        xsel ^= 1;          // the next exchange writes the other buffer (no second barrier)
    };
    V4<T> xv[kRows], car[kRows], csep = v4zero<T>();
#pragma unroll
    for (int j = 0; j < kRows; ++j) car[j] = v4zero<T>();
    const int xs = s0 + mi - 1;
    const bool xs_int = xs > 0 && xs < nx - 1;
    // W^-1 of a row: the inverse precision of its observation (initial
    // condition, PDE), of the Dirichlet rows, or one for the prior's rows
    auto wrow = [&](int x, int k) -> T {
        const int kind = tsp_row_kind<T>(L, x, k, has_ic);
        return kind == TR_BND ? iw_bnd : kind == TR_IC ? iw_ic : kind == TR_COL ? iw_q : T(1);
    };
    for (int sweep = sweep_lo; sweep < sweep_hi; ++sweep) {
        // sweep 0, backward: J^T y = r from the last level down, then y / W;
        // sweep 1, forward: J z = W^-1 y from the first level up
        const bool bwd = sweep == 0;
        const T* src = bwd ? r : y;
        T* dst = bwd ? y : z;
        const int dir = bwd ? 1 : 0;
        if (!bwd) {
            __syncthreads();               // every lane's y rows written
#pragma unroll
            for (int j = 0; j < kRows; ++j) car[j] = v4zero<T>();
            csep = v4zero<T>();
        }
        stage(src, dir, bwd ? nt - 1 : 0, 0);
        cp_commit();
        for (int i = 0; i < nt; ++i) {
            const int k = bwd ? nt - 1 - i : i;
            const int slot = i & 1;
            cp_wait<0>();
            __syncthreads();               // level k landed; the other buffers are free
            stage(src, dir, bwd ? k - 1 : k + 1, slot ^ 1);
            cp_commit();
            const V4<T>* in = sin + (size_t)slot * NXC + ibase;
            const T* rowf = sfac + (size_t)slot * kFactorBlock;
            const T* lanef = rowf + kRowF * kRows * kLanes;
            auto F = [&](int field, int j) { return rowf[(field * kRows + j) * kLanes + lane]; };
            const bool couple = bwd ? k + 1 < nt : k > 0;     // the level reached by the time step
            const int jlo = s0 > 0 ? 0 : 1;                  // x = 0 (lane 0, row 0) is a boundary node
            // FEM rows: the coupled level's values at x - 1 and x + 1 across
            // chunk ends (the previous lane's separator, the next lane's first row)
            V4<T> prevsep = v4zero<T>(), nextfirst = v4zero<T>();
            const T* cplf = scpl + (size_t)slot * kCplBlock;
            auto CP = [&](int e, int j) { return cplf[(e * kRows + j) * kLanes + lane]; };
            if (FEM) {
                V4<T> dummy;
                exch(csep, 1, prevsep, dummy);
                exch(mint > 0 ? car[0] : csep, 1, dummy, nextfirst);
            }
            // right-hand sides of the interior rows, then p'_j = d_j / den_j - (A_j / den_j) p'_{j-1}
            V4<T> pprev = v4zero<T>();
#pragma unroll
            for (int j = 0; j < kRows; ++j) {
                if (j < mint) {
                    V4<T> v = in[j];
                    if (FEM) {
                        const V4<T> cl = j > 0 ? car[j > 0 ? j - 1 : 0] : prevsep;
                        const V4<T> cr = j < mint - 1 ? car[j + 1 < kRows ? j + 1 : j] : csep;
                        v = fma4(CP(0, j), cl, fma4(CP(1, j), car[j], fma4(CP(2, j), cr, v)));
                    } else if (couple && j >= jlo) {
                        v = fma4(inv_dt, car[j], v);
                    }
                    pprev = fma4(-F(0, j), pprev, F(1, j) * v);
                    xv[j] = pprev;
                }
            }
            const V4<T> plast = mint > 0 ? pprev : v4zero<T>();
            // backward: P_j = p'_j - c'_j P_{j+1}
            V4<T> pn = v4zero<T>();
#pragma unroll
            for (int j = kRows - 1; j >= 0; --j) {
                if (j < mint) {
                    pn = fma4(-F(2, j), pn, xv[j]);
                    xv[j] = pn;
                }
            }
            // separator row: d - A P_{e-2} - C P_e (P_e: the next lane's first row)
            V4<T> dsep = v4zero<T>();
            if (mi > 0) {
                dsep = in[mi - 1];
                if (FEM) {
                    V4<T> cl = prevsep;
#pragma unroll
                    for (int j = 0; j < kRows; ++j)
                        if (j == mint - 1) cl = car[j];
                    const T* sc = cplf + 3 * kRows * kLanes;
                    dsep = fma4(sc[0 * kLanes + lane], cl, fma4(sc[1 * kLanes + lane], csep, fma4(sc[2 * kLanes + lane], nextfirst, dsep)));
                } else if (couple && xs_int) {
                    dsep = fma4(inv_dt, csep, dsep);
                }
            }
            const V4<T> pf = mint > 0 ? xv[0] : v4zero<T>();
            V4<T> pup, pnx;
            exch(pf, 1, pup, pnx);
            V4<T> rd = v4zero<T>();
            if (mi > 0) rd = fma4(-lanef[1 * kLanes + lane], pnx, fma4(-lanef[0 * kLanes + lane], plast, dsep));
            int step = 0;
#pragma unroll
            for (int st = 1; st < kLanes; st <<= 1, ++step) {
                V4<T> dm, dp;
                exch(rd, st, dm, dp);
                rd = fma4(-lanef[(3 + kSteps + step) * kLanes + lane], dp, fma4(-lanef[(3 + step) * kLanes + lane], dm, rd));
            }
            const V4<T> X = lanef[2 * kLanes + lane] * rd;
            V4<T> Xl, Xr;
            exch(X, 1, Xl, Xr);
            T* ob = dst + ((size_t)blk * N + (size_t)k * nx + s0) * RW;
#pragma unroll
            for (int j = 0; j < kRows; ++j) {
                if (j < mint) {
                    const V4<T> xj = fma4(F(4, j), X, fma4(F(3, j), Xl, xv[j]));
                    car[j] = xj;
                    v4store(ob + (size_t)j * RW, bwd ? wrow(s0 + j, k) * xj : xj);
                }
            }
            if (mi > 0) {
                csep = X;
                v4store(ob + (size_t)(xs - s0) * RW, bwd ? wrow(xs, k) * X : X);
            }
        }
    }
}

// Matern transition noise: the prior rows of a level k >= 1 carry the weight
// T_K^2 (B = T_K B_w), so between the sweeps y_k <- T_P^-2 y_k, with T_P the
// level's T_K between its prior rows (identity on the other rows, which are
// decoupled from them).  One CTA per (level, block): thread 0 forms the
// Thomas multipliers of T_P in shared memory, threads 0..3 solve the four
// right-hand sides twice.
template <typename T>
__global__ void __launch_bounds__(32) k_tsp_tscale(const LevelView<T> L, int has_ic, T* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char ts_smem[];
    T* cp = reinterpret_cast<T*>(ts_smem);           // [nx]: modified super-diagonal
    T* den = cp + L.nx;                              // [nx]: 1 / pivot
    const int nx = L.nx, k = blockIdx.x + 1, blk = blockIdx.y;
    const T tc = (T)L.tk_c, to = (T)L.tk_o;
    auto prior = [&](int x) { return x >= 0 && x < nx && tsp_row_kind<T>(L, x, k, has_ic) == TR_PRIOR; };
    if (threadIdx.x == 0) {
        T cprev = T(0);
        for (int x = 0; x < nx; ++x) {
            const bool px = prior(x);
            const T a = px && prior(x - 1) ? to : T(0);
            const T b = px ? tc : T(1);
            const T c = px && prior(x + 1) ? to : T(0);
            const T inv = T(1) / (b - a * cprev);
            den[x] = inv;
            cprev = c * inv;
            cp[x] = cprev;
        }
    }
    __syncthreads();
    if (threadIdx.x >= 4) return;
    T* v = y + ((size_t)blk * L.N + (size_t)k * nx) * RW + threadIdx.x;
    for (int rep = 0; rep < 2; ++rep) {
        T dprev = T(0);
        for (int x = 0; x < nx; ++x) {
            const T a = prior(x) && prior(x - 1) ? to : T(0);
            dprev = (v[(size_t)x * RW] - a * dprev) * den[x];
            v[(size_t)x * RW] = dprev;
        }
        for (int x = nx - 2; x >= 0; --x) v[(size_t)x * RW] -= cp[x] * v[(size_t)(x + 1) * RW];
    }
}

}  // namespace

// rows of J_t that need the per-row coupling arrays (anything but the
// implicit-Euler collocation rows at every node with the initial condition observed)
static bool tsp_mixed(const Level& L) {
    return L.col.kind >= 3 || L.col.kind == 0 || L.col.sx > 1 || L.col.st > 1 || !L.tsp_ic;
}

// PDE rows (weight Q_eps) next to prior rows (weight one) in J_t: for a
// right-hand side in the span of the PDE rows (what the refinement residual
// mostly is once the PDE is nearly met) the exact M r is of order 1 / Q_eps,
// but the rounding errors of the backward sweep land on the prior rows with
// weight one, about eps * Q_eps |J| / |B| relative to it: beyond one in FP32
// for any useful Q_eps, so such solves run their inner iteration in FP64
bool tsp_mixed_weights(const Level& L) {
    return L.col.kind != 0 && L.col.qeps > 0 && (L.col.sx > 1 || L.col.st > 1 || !L.tsp_ic);
}

bool tsp_applicable(const Level& L, int nic) {
    // PDE rows (collocation or FEM) or a prior with Matern transition noise
    // (whose multigrid is slow: B has a wider stencil); every level block of
    // J_t is tridiagonal either way
    (void)nic;
    return L.geo == GEO_XT && (L.col.kind != 0 || L.noise) && L.nx <= kTspMaxNx;
}

static size_t tsp_smem(const Level& L, size_t elem) {
    const bool fem = tsp_mixed(L);
    return elem * (size_t)2 * (kFactorBlock + (fem ? kCplBlock : 0)) + 4 * elem * (size_t)2 * (L.nx + kLanes);
}

template <typename T> bool tsp_fits(const Level& L) {
    static const int optin = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return 0;
        return v;
    }();
    return tsp_smem(L, sizeof(T)) + 2 * sizeof(V4<T>) * kLanes <= (size_t)optin;
}
template bool tsp_fits<float>(const Level&);
template bool tsp_fits<double>(const Level&);

// Factors of every level and both sweep directions, in both precisions
// (the FP32 inner solve and the plain FP64 path); rerun whenever the
// linearisation point changes.
void tsp_prepare(Level& L, int nic, cudaStream_t s) {
    L.tsp_ic = nic > 0 ? 1 : 0;
    const size_t n = (size_t)2 * L.nt * kFactorBlock;
    if (!L.d_tsp32) L.d_tsp32 = dev_alloc<float>(n);
    if (!L.d_tsp64) L.d_tsp64 = dev_alloc<double>(n);
    k_tsp_factor<float><<<2 * L.nt, kLanes, 0, s>>>(L.view<float>(), L.tsp_ic, L.d_tsp32);
    note_launch();
    k_tsp_factor<double><<<2 * L.nt, kLanes, 0, s>>>(L.view<double>(), L.tsp_ic, L.d_tsp64);
    note_launch();
    if (tsp_mixed(L)) {
        const size_t nc = (size_t)2 * L.nt * kCplBlock;
        if (!L.d_tspc32) L.d_tspc32 = dev_alloc<float>(nc);
        if (!L.d_tspc64) L.d_tspc64 = dev_alloc<double>(nc);
        k_tsp_couple<float><<<2 * L.nt, kLanes, 0, s>>>(L.view<float>(), L.tsp_ic, L.d_tspc32);
        note_launch();
        k_tsp_couple<double><<<2 * L.nt, kLanes, 0, s>>>(L.view<double>(), L.tsp_ic, L.d_tspc64);
        note_launch();
    }
    GCK(cudaGetLastError());
}

template <typename T, bool FEM>
static void launch_tsp_kind(const Level& L, double w_ic, double w_bnd, const T* r, T* y, T* z, int nblk, cudaStream_t s) {
    const size_t smem = tsp_smem(L, sizeof(T));
    const T* fac = sizeof(T) == 4 ? reinterpret_cast<const T*>(L.d_tsp32) : reinterpret_cast<const T*>(L.d_tsp64);
    const T* cpl = sizeof(T) == 4 ? reinterpret_cast<const T*>(L.d_tspc32) : reinterpret_cast<const T*>(L.d_tspc64);
    if (!fac || (FEM && !cpl)) throw Error(GMRF_E_INVALID, "time-stepping preconditioner: factors not prepared");
    static size_t attr = 0;
    if (smem > attr) {
        if (cudaFuncSetAttribute(k_tsp<T, FEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            throw Error(GMRF_E_CUDA, "time-stepping preconditioner: shared memory attribute");
        attr = smem;
    }
    const double iq = L.col.qeps > 0 ? 1.0 / L.col.qeps : 0.0;
    const T a = (T)(1.0 / w_ic), b = (T)(1.0 / w_bnd), q = (T)iq;
    // with Matern transition noise the prior rows' weight T_K^2 is applied
    // between the backward and the forward sweep
    const bool tscale = L.noise && (L.col.kind == 0 || L.col.sx > 1 || L.col.st > 1) && L.nt > 1;
    if (!tscale) {
        k_tsp<T, FEM><<<nblk, kLanes, smem, s>>>(L.view<T>(), fac, cpl, a, b, q, L.tsp_ic, 0, 2, r, y, z);
        note_launch();
        return;
    }
    k_tsp<T, FEM><<<nblk, kLanes, smem, s>>>(L.view<T>(), fac, cpl, a, b, q, L.tsp_ic, 0, 1, r, y, z);
    note_launch();
    const size_t tsm = 2 * sizeof(T) * (size_t)L.nx;
    k_tsp_tscale<T><<<dim3((unsigned)(L.nt - 1), (unsigned)nblk), 32, tsm, s>>>(L.view<T>(), L.tsp_ic, y);
    note_launch();
    k_tsp<T, FEM><<<nblk, kLanes, smem, s>>>(L.view<T>(), fac, cpl, a, b, q, L.tsp_ic, 1, 2, r, y, z);
    note_launch();
}

template <typename T>
void launch_tsp(const Level& L, double w_ic, double w_bnd, const T* r, T* y, T* z, int nblk, cudaStream_t s) {
    if (tsp_mixed(L)) launch_tsp_kind<T, true>(L, w_ic, w_bnd, r, y, z, nblk, s);
    else launch_tsp_kind<T, false>(L, w_ic, w_bnd, r, y, z, nblk, s);
}
template void launch_tsp<float>(const Level&, double, double, const float*, float*, float*, int, cudaStream_t);
template void launch_tsp<double>(const Level&, double, double, const double*, double*, double*, int, cudaStream_t);

}  // namespace gmrf
