// Time-stepping preconditioner for collocation systems (1D space x time).
//
// With near-exact collocation (Sec. 3.1, 3.3) the posterior precision is
// dominated by Jt^T W Jt, where Jt stacks the initial-condition rows (t = 0),
// the Dirichlet rows of the prior at the spatial boundary and the
// collocation rows at interior nodes of levels k >= 1, with W their
// precisions.  Jt is square and block lower-bidiagonal in time (implicit
// Euler): level k reads level k (a tridiagonal stencil in x) and level k-1
// (-1/dt at the same x).  Its inverse is one forward time sweep and Jt^-T one
// backward sweep, each level a tridiagonal solve, so
//     z = M r = Jt^-1 W^-1 Jt^-T r
// costs two sweeps and leaves the prior's interior part and the point data,
// both orders of magnitude smaller, to the outer conjugate gradients.
#include "handles.h"

namespace gmrf {

namespace {

constexpr int kTspRows = 31;                 // interior rows per lane: nx <= 32 (kTspRows + 1)
constexpr int kTspMaxNx = 32 * (kTspRows + 1);

// Each right-hand side is swept by one warp.  A level's tridiagonal system
// (nx <= 32 (M + 1) rows) is solved by the partition method: lane l owns the
// contiguous rows [l m, l m + m), m = ceil(nx / 32); the last row of each chunk
// is a separator.  The chunk's interior rows are eliminated by a Thomas sweep
// with three right-hand sides, giving x_i = p_i + q_i X_{l-1} + r_i X_l in
// terms of the neighbouring separators; substituting into the separator rows
// leaves a 32-unknown tridiagonal system, one unknown per lane, solved by
// parallel cyclic reduction with warp shuffles; the interior rows follow by
// back-substitution.
//
// Everything that depends on the matrix alone (the Thomas pivots and
// multipliers, the interface columns q and r, the separator coefficients and
// the cyclic-reduction multipliers) is the same for every right-hand side and
// every application in a solve, so k_tsp_factor computes it once per
// linearisation, for every level and both sweep directions; an application
// (k_tsp) then runs only the right-hand-side recurrences: no divisions, one
// dependent FMA per row and direction.  A CTA holds the four warps of one
// block of right-hand sides; each level's inputs and factors are staged in
// shared memory by cp.async one level ahead (double-buffered).
//
// Factors of one (direction, level), in elements of T:
//   row fields [5][32][32] (field, chunk row j, lane): A_j/den_j, 1/den_j,
//     c'_j (Thomas), Q_j, R_j (interface columns after back-substitution);
//   lane fields [13][32]: separator A and C, the cyclic-reduction
//     multipliers k1, k2 of its 5 steps, 1 / final diagonal.
constexpr int kRowF = 5, kLaneF = 13;
constexpr int kFactorBlock = kRowF * 32 * 32 + kLaneF * 32;

// Level row coefficients of J (lower x-1, diagonal, upper x+1) at node x of
// level k, with mu the linearisation point of the level (Burgers).
template <typename T>
__device__ __forceinline__ void j_row(const LevelView<T>& L, const T* mu, int x, int k, T& lo, T& di, T& up) {
    const int nx = L.nx;
    if (k == 0 || x <= 0 || x >= nx - 1) { lo = T(0); di = T(1); up = T(0); return; }
    const Colloc& c = L.col;
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
__device__ __forceinline__ void level_row(const LevelView<T>& L, const T* mu, int x, int k, T& A, T& B, T& C) {
    T lo, di, up;
    j_row<T>(L, mu, x, k, lo, di, up);
    B = di;
    if (!TR) { A = lo; C = up; return; }
    T l2, d2, u2;
    A = T(0);
    C = T(0);
    if (x > 0) { j_row<T>(L, mu, x - 1, k, l2, d2, u2); A = u2; }
    if (x < L.nx - 1) { j_row<T>(L, mu, x + 1, k, l2, d2, u2); C = l2; }
}

// One warp per (direction, level): the matrix-only part of the partition
// solve.  blockIdx.x = dir * nt + k, dir 0 = D_k (forward sweep), 1 = D_k^T.
template <typename T>
__global__ void __launch_bounds__(32) k_tsp_factor(const LevelView<T> L, T* __restrict__ f) {
    const unsigned FULL = 0xffffffffu;
    const int nx = L.nx, nt = L.nt;
    const int dir = blockIdx.x / nt, k = blockIdx.x % nt;
    const int lane = threadIdx.x;
    const int m = (nx + 31) / 32, s = lane * m, mi = max(0, min(m, nx - s)), mint = mi - 1;
    const T* mu = L.col.kind == 2 ? L.mu + (size_t)k * nx : nullptr;
    T* blk = f + (size_t)blockIdx.x * kFactorBlock;
    T* rowf = blk;                               // [field][j][lane]
    T* lanef = blk + kRowF * 32 * 32;            // [field][lane]
    auto row = [&](int x, T& A, T& B, T& C) {
        if (dir == 0) level_row<T, false>(L, mu, x, k, A, B, C);
        else level_row<T, true>(L, mu, x, k, A, B, C);
    };
    T qv[32], rv[32], cv[32];
    T cprev = T(0), qprev = T(0);
    for (int j = 0; j < 32; ++j) {
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
        rowf[(0 * 32 + j) * 32 + lane] = ainv;
        rowf[(1 * 32 + j) * 32 + lane] = inv;
        rowf[(2 * 32 + j) * 32 + lane] = c;
        qv[j] = q;
        rv[j] = r;
        cv[j] = c;
    }
    T qn = T(0), rn = T(0);
    for (int j = 31; j >= 0; --j) {
        if (j < mint) {
            qv[j] = qv[j] - cv[j] * qn;
            rv[j] = rv[j] - cv[j] * rn;
            qn = qv[j];
            rn = rv[j];
        }
        rowf[(3 * 32 + j) * 32 + lane] = j < mint ? qv[j] : T(0);
        rowf[(4 * 32 + j) * 32 + lane] = j < mint ? rv[j] : T(0);
    }
    // separator row: A x_{e-2} + B X_l + C x_e, with x_{e-2} = p + ql X_{l-1} + rl X_l
    // (own last interior row) and x_e = p + qf X_l + rf X_{l+1} (next lane's first row)
    T qf = mint > 0 ? qv[0] : T(0), rf = mint > 0 ? rv[0] : T(1);
    if (mi <= 0) { qf = T(0); rf = T(0); }
    const T qnx = __shfl_down_sync(FULL, qf, 1), rnx = __shfl_down_sync(FULL, rf, 1);
    T Asep = T(0), Csep = T(0), ra = T(0), rb = T(1), rc = T(0);
    if (mi > 0) {
        T A, B, C;
        row(s + mi - 1, A, B, C);
        if (lane == 31 || s + mi >= nx) C = T(0);
        T ql = T(1), rl = T(0);
        if (mint > 0) {
            for (int j = 0; j < 32; ++j)
                if (j == mint - 1) { ql = qv[j]; rl = rv[j]; }
        }
        if (s == 0 && mint == 0) ql = T(0);
        Asep = A;
        Csep = C;
        ra = lane == 0 ? T(0) : A * ql;      // lane 0 has no left separator
        rb = B + A * rl + C * qnx;
        rc = C * rnx;
    }
    lanef[0 * 32 + lane] = Asep;
    lanef[1 * 32 + lane] = Csep;
    int step = 0;
    for (int st = 1; st < 32; st <<= 1, ++step) {
        const T am = __shfl_up_sync(FULL, ra, st), bm = __shfl_up_sync(FULL, rb, st), cm = __shfl_up_sync(FULL, rc, st);
        const T ap = __shfl_down_sync(FULL, ra, st), bp = __shfl_down_sync(FULL, rb, st), cp2 = __shfl_down_sync(FULL, rc, st);
        const bool hm = lane - st >= 0, hp = lane + st < 32;
        const T k1 = hm ? ra / bm : T(0), k2 = hp ? rc / bp : T(0);
        const T na = hm ? -am * k1 : T(0), nc = hp ? -cp2 * k2 : T(0);
        const T nb = rb - (hm ? cm * k1 : T(0)) - (hp ? ap * k2 : T(0));
        ra = na;
        rb = nb;
        rc = nc;
        lanef[(2 + step) * 32 + lane] = k1;
        lanef[(7 + step) * 32 + lane] = k2;
    }
    lanef[12 * 32 + lane] = T(1) / rb;
}

// The right-hand-side part of one level solve for the lane's rows (interior
// rows j < mi - 1 in xv[], the separator's right-hand side dsep, its solution
// in X), with the factors of the level staged at rowf / lanef.
template <typename T, int M>
__device__ __forceinline__ void warp_tridiag_rhs(const T* rowf, const T* lanef, int mi, T (&xv)[M], T dsep, T& Xout) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int mint = mi - 1;
    auto F = [&](int field, int j) { return rowf[(field * 32 + j) * 32 + lane]; };
    // forward: p'_j = d_j / den_j - (A_j / den_j) p'_{j-1}
    T pprev = T(0);
#pragma unroll
    for (int j = 0; j < M; ++j) {
        if (j < mint) {
            pprev = xv[j] * F(1, j) - F(0, j) * pprev;
            xv[j] = pprev;
        }
    }
    const T plast = mint > 0 ? pprev : T(0);
    // backward: P_j = p'_j - c'_j P_{j+1}
    T pn = T(0);
#pragma unroll
    for (int j = M - 1; j >= 0; --j) {
        if (j < mint) {
            pn = xv[j] - F(2, j) * pn;
            xv[j] = pn;
        }
    }
    T pf = mint > 0 ? xv[0] : T(0);
    if (mi <= 0) pf = T(0);
    const T pnx = __shfl_down_sync(FULL, pf, 1);
    T rd = mi > 0 ? dsep - lanef[0 * 32 + lane] * plast - lanef[1 * 32 + lane] * pnx : T(0);
    int step = 0;
#pragma unroll
    for (int st = 1; st < 32; st <<= 1, ++step) {
        const T dm = __shfl_up_sync(FULL, rd, st), dp = __shfl_down_sync(FULL, rd, st);
        rd = rd - lanef[(2 + step) * 32 + lane] * dm - lanef[(7 + step) * 32 + lane] * dp;
    }
    const T X = rd * lanef[12 * 32 + lane];
    T Xl = __shfl_up_sync(FULL, X, 1);
    if (lane == 0) Xl = T(0);
#pragma unroll
    for (int j = 0; j < M; ++j)
        if (j < mint) xv[j] = xv[j] + F(3, j) * Xl + F(4, j) * X;
    Xout = X;
}

// One CTA of four warps per block of four right-hand sides; warp w sweeps
// component w.  y is scratch of the blocked layout; r and z are blocked.
template <typename T, int M>
__global__ void __launch_bounds__(128) k_tsp(const LevelView<T> L, const T* __restrict__ fac, T w_ic, T w_bnd,
                                            const T* __restrict__ r, T* __restrict__ y, T* __restrict__ z) {
    extern __shared__ __align__(16) unsigned char tsp_smem[];
    const int nx = L.nx, nt = L.nt;
    const long long N = L.N;
    const int NXP = nx + (nx >> 5) + 1;                  // padded input row
    const int SIN = ((4 * NXP + 3) / 4) * 4;             // elements of one stage of inputs (16-byte multiple)
    T* sfac = reinterpret_cast<T*>(tsp_smem);            // [2][kFactorBlock]
    T* sin = sfac + 2 * kFactorBlock;                    // [2][4][NXP]
    const int blk = blockIdx.x, tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int m = (nx + 31) / 32;
    const int s0 = lane * m, mi = max(0, min(m, nx - s0));
    const T inv_dt = (T)L.col.inv_dt;
    const T wq = (T)L.col.qeps;
    auto stage = [&](const T* src, int dir, int k, int slot) {
        if (k < 0 || k >= nt) return;
        const T* g = src + ((size_t)blk * N + (size_t)k * nx) * RW;
        T* d = sin + (size_t)slot * SIN;
        for (int e = tid; e < 4 * nx; e += 128) {
            const int x = e >> 2, c = e & 3;
            cp_scalar<T>(d + (size_t)c * NXP + x + (x >> 5), g + e, true);
        }
        const char* gf = reinterpret_cast<const char*>(fac + ((size_t)dir * nt + k) * kFactorBlock);
        char* df = reinterpret_cast<char*>(sfac + (size_t)slot * kFactorBlock);
        for (int c = tid; c < (int)(kFactorBlock * sizeof(T) / 16); c += 128) cp_async16(df + c * 16, gf + c * 16, true);
    };
    T xv[M], carry[M], csep = T(0);
#pragma unroll
    for (int j = 0; j < M; ++j) carry[j] = T(0);
    const int xs = s0 + mi - 1;
    const bool xs_int = xs > 0 && xs < nx - 1;
    // backward sweep: J^T y = r from the last level down, then y / W
    stage(r, 1, nt - 1, 0);
    cp_commit();
    for (int k = nt - 1; k >= 0; --k) {
        const int slot = (nt - 1 - k) & 1;
        cp_wait<0>();
        __syncthreads();                  // level k landed; level k+1's buffers are free
        stage(r, 1, k - 1, slot ^ 1);
        cp_commit();
        const T* in = sin + (size_t)slot * SIN + (size_t)w * NXP;
        const T* fk = sfac + (size_t)slot * kFactorBlock;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            if (j < mi - 1) {
                const int x = s0 + j;
                T v = in[x + (x >> 5)];
                if (k + 1 < nt && x > 0 && x < nx - 1) v += inv_dt * carry[j];
                xv[j] = v;
            }
        }
        T dsep = T(0), X = T(0);
        if (mi > 0) {
            dsep = in[xs + (xs >> 5)];
            if (k + 1 < nt && xs_int) dsep += inv_dt * csep;
        }
        warp_tridiag_rhs<T, M>(fk, fk + kRowF * 32 * 32, mi, xv, dsep, X);
        const T wi = k == 0 ? w_ic : wq;                    // interior x; boundary x gets w_bnd
#pragma unroll
        for (int j = 0; j < M; ++j) {
            if (j < mi - 1) {
                const int x = s0 + j;
                carry[j] = xv[j];
                const T wt = (x == 0 || x == nx - 1) ? w_bnd : wi;
                y[((size_t)blk * N + (size_t)k * nx + x) * RW + w] = xv[j] / wt;
            }
        }
        if (mi > 0) {
            csep = X;
            const T wt = (xs == 0 || xs == nx - 1) ? w_bnd : wi;
            y[((size_t)blk * N + (size_t)k * nx + xs) * RW + w] = X / wt;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < M; ++j) carry[j] = T(0);
    csep = T(0);
    // forward sweep: J z = W^-1 y from the first level up
    stage(y, 0, 0, 0);
    cp_commit();
    for (int k = 0; k < nt; ++k) {
        const int slot = k & 1;
        cp_wait<0>();
        __syncthreads();
        stage(y, 0, k + 1, slot ^ 1);
        cp_commit();
        const T* in = sin + (size_t)slot * SIN + (size_t)w * NXP;
        const T* fk = sfac + (size_t)slot * kFactorBlock;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            if (j < mi - 1) {
                const int x = s0 + j;
                T v = in[x + (x >> 5)];
                if (k > 0 && x > 0 && x < nx - 1) v += inv_dt * carry[j];
                xv[j] = v;
            }
        }
        T dsep = T(0), X = T(0);
        if (mi > 0) {
            dsep = in[xs + (xs >> 5)];
            if (k > 0 && xs_int) dsep += inv_dt * csep;
        }
        warp_tridiag_rhs<T, M>(fk, fk + kRowF * 32 * 32, mi, xv, dsep, X);
#pragma unroll
        for (int j = 0; j < M; ++j) {
            if (j < mi - 1) {
                const int x = s0 + j;
                carry[j] = xv[j];
                z[((size_t)blk * N + (size_t)k * nx + x) * RW + w] = xv[j];
            }
        }
        if (mi > 0) {
            csep = X;
            z[((size_t)blk * N + (size_t)k * nx + xs) * RW + w] = X;
        }
    }
}

}  // namespace

bool tsp_applicable(const Level& L, int nic) {
    return L.geo == GEO_XT && L.col.kind != 0 && nic > 0 && L.nx <= kTspMaxNx;
}

// Factors of every level and both sweep directions, in both precisions
// (the FP32 inner solve and the plain FP64 path); rerun whenever the
// linearisation point changes.
void tsp_prepare(Level& L, cudaStream_t s) {
    const size_t n = (size_t)2 * L.nt * kFactorBlock;
    if (!L.d_tsp32) L.d_tsp32 = dev_alloc<float>(n);
    if (!L.d_tsp64) L.d_tsp64 = dev_alloc<double>(n);
    k_tsp_factor<float><<<2 * L.nt, 32, 0, s>>>(L.view<float>(), L.d_tsp32);
    note_launch();
    k_tsp_factor<double><<<2 * L.nt, 32, 0, s>>>(L.view<double>(), L.d_tsp64);
    note_launch();
    GCK(cudaGetLastError());
}

template <typename T>
void launch_tsp(const Level& L, double w_ic, double w_bnd, const T* r, T* y, T* z, int nblk, cudaStream_t s) {
    const int nxp = L.nx + (L.nx >> 5) + 1;
    const size_t smem = sizeof(T) * (size_t)(2 * kFactorBlock + 2 * (((4 * nxp + 3) / 4) * 4));
    const T* fac = sizeof(T) == 4 ? reinterpret_cast<const T*>(L.d_tsp32) : reinterpret_cast<const T*>(L.d_tsp64);
    if (!fac) throw Error(GMRF_E_INVALID, "time-stepping preconditioner: factors not prepared");
    static size_t attr = 0;
    if (smem > attr) {
        if (cudaFuncSetAttribute(k_tsp<T, kTspRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            throw Error(GMRF_E_CUDA, "time-stepping preconditioner: shared memory attribute");
        attr = smem;
    }
    k_tsp<T, kTspRows><<<nblk, 128, smem, s>>>(L.view<T>(), fac, (T)w_ic, (T)w_bnd, r, y, z);
    note_launch();
}
template void launch_tsp<float>(const Level&, double, double, const float*, float*, float*, int, cudaStream_t);
template void launch_tsp<double>(const Level&, double, double, const double*, double*, double*, int, cudaStream_t);

}  // namespace gmrf
