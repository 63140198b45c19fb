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
// back-substitution.  The warp never waits on a block barrier inside a level.
// A CTA holds the four warps of one block of right-hand sides, which share
// the linearisation point; each level's inputs are staged in shared memory by
// cp.async one level ahead (double-buffered), de-interleaved from the blocked
// layout and padded by one slot per 32 so that the lanes' contiguous chunks
// hit distinct banks.

// Level row coefficients of J (lower x-1, diagonal, upper x+1) at node x of
// level k, with mu the staged linearisation point (Burgers) of the level.
template <typename T>
__device__ __forceinline__ void j_row(const LevelView<T>& L, const T* mu, int x, int k, T& lo, T& di, T& up) {
    const int nx = L.nx;
    if (k == 0 || x <= 0 || x >= nx - 1) { lo = T(0); di = T(1); up = T(0); return; }
    const Colloc& c = L.col;
    T a, da;
    if (c.kind == 1) { a = (T)c.c; da = T(0); }
    else {
        a = mu[x + (x >> 5)];
        da = (mu[(x + 1) + ((x + 1) >> 5)] - mu[(x - 1) + ((x - 1) >> 5)]) * (T)c.inv_2h;
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

// Solves one level for the lane's rows s .. s + mi - 1 (mi <= M + 1): the
// interior rows' right-hand sides in xv[0 .. mi-2] on entry, their solution on
// exit; the separator row's right-hand side dsep, its solution in X.  All 32
// lanes must call it.
template <typename T, bool TR, int M>
__device__ __forceinline__ void warp_tridiag(const LevelView<T>& L, const T* mu, int k, int s, int mi, T (&xv)[M], T dsep,
                                             T& Xout) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    T cp[M], pp[M], qp[M], rp[M];
    const int mint = mi - 1;      // interior rows of the chunk (the last row is the separator)
    // Thomas sweep over the interior rows with the three right-hand sides
    // (d, -A_first e_first, -C_last e_last): x_i = p_i + q_i X_{l-1} + r_i X_l.
    // The coefficients of J's rows x-1, x, x+1 slide along (the transposed
    // system reads its neighbours' lower and upper entries).
    // the last interior row's (p, q, r), i.e. x_{e-2} in terms of (X_{l-1}, X_l)
    T pl = T(0), ql = T(1), rl = T(0);
    {
        T lo0, di0, up0, lo1, di1, up1, lo2, di2, up2;
        j_row<T>(L, mu, s - 1, k, lo0, di0, up0);
        j_row<T>(L, mu, s, k, lo1, di1, up1);
        T cprev = T(0), pprev = T(0), qprev = T(0), rlast = T(0);
#pragma unroll
        for (int j = 0; j < M; ++j) {
            if (j < mint) {
                j_row<T>(L, mu, s + j + 1, k, lo2, di2, up2);
                const int x = s + j;
                const T A = TR ? (x > 0 ? up0 : T(0)) : lo1;
                const T B = di1;
                const T C = TR ? (x < L.nx - 1 ? lo2 : T(0)) : up1;
                const T inv = T(1) / (B - A * cprev);
                const bool last = j == mint - 1;
                cp[j] = last ? T(0) : C * inv;
                pp[j] = (xv[j] - A * pprev) * inv;
                qp[j] = (j == 0 ? -A : -A * qprev) * inv;
                rp[j] = last ? -C * inv : T(0);
                if (last) rlast = rp[j];
                cprev = cp[j];
                pprev = pp[j];
                qprev = qp[j];
                lo0 = lo1; di0 = di1; up0 = up1;
                lo1 = lo2; di1 = di2; up1 = up2;
            }
        }
        // the back substitution leaves the last interior row as it is (c' = 0 there)
        if (mint > 0) {
            pl = pprev;
            ql = qprev;
            rl = rlast;
        }
        // back substitution of the three columns
        T pn = T(0), qn = T(0), rn = T(0);
#pragma unroll
        for (int j = M - 1; j >= 0; --j) {
            if (j < mint) {
                pp[j] = pp[j] - cp[j] * pn;
                qp[j] = qp[j] - cp[j] * qn;
                rp[j] = rp[j] - cp[j] * rn;
                pn = pp[j];
                qn = qp[j];
                rn = rp[j];
            }
        }
    }
    // separator row e - 1 of this lane: A x_{e-2} + B X_l + C x_e = d
    T ra = T(0), rb = T(1), rc = T(0), rd = T(0);
    // x_e in terms of (X_l, X_{l+1}) from the next lane's first row
    T pf = mint > 0 ? pp[0] : T(0), qf = mint > 0 ? qp[0] : T(0), rf = mint > 0 ? rp[0] : T(1);
    if (mi <= 0) { pf = T(0); qf = T(0); rf = T(0); }
    const T pn = __shfl_down_sync(FULL, pf, 1), qn = __shfl_down_sync(FULL, qf, 1), rn = __shfl_down_sync(FULL, rf, 1);
    if (mi > 0) {
        T A, B, C;
        level_row<T, TR>(L, mu, s + mi - 1, k, A, B, C);
        if (lane == 31 || s + mi >= L.nx) C = T(0);
        if (s == 0 && mint == 0) ql = T(0);     // no left neighbour at all
        ra = A * ql;
        rb = B + A * rl + C * qn;
        rc = C * rn;
        rd = dsep - A * pl - C * pn;
        if (lane == 0) ra = T(0);
    }
    // parallel cyclic reduction of the 32-lane tridiagonal system
#pragma unroll
    for (int st = 1; st < 32; st <<= 1) {
        const T am = __shfl_up_sync(FULL, ra, st), bm = __shfl_up_sync(FULL, rb, st), cm = __shfl_up_sync(FULL, rc, st),
                dm = __shfl_up_sync(FULL, rd, st);
        const T ap = __shfl_down_sync(FULL, ra, st), bp = __shfl_down_sync(FULL, rb, st), cp2 = __shfl_down_sync(FULL, rc, st),
                dp = __shfl_down_sync(FULL, rd, st);
        const bool hm = lane - st >= 0, hp = lane + st < 32;
        const T k1 = hm ? ra / bm : T(0), k2 = hp ? rc / bp : T(0);
        const T na = hm ? -am * k1 : T(0), nc = hp ? -cp2 * k2 : T(0);
        const T nb = rb - (hm ? cm * k1 : T(0)) - (hp ? ap * k2 : T(0));
        const T nd = rd - (hm ? dm * k1 : T(0)) - (hp ? dp * k2 : T(0));
        ra = na;
        rb = nb;
        rc = nc;
        rd = nd;
    }
    const T X = rd / rb;
    T Xl = __shfl_up_sync(FULL, X, 1);
    if (lane == 0) Xl = T(0);
#pragma unroll
    for (int j = 0; j < M; ++j)
        if (j < mint) xv[j] = pp[j] + qp[j] * Xl + rp[j] * X;
    Xout = X;
}

// One CTA of four warps per block of four right-hand sides; warp w sweeps
// component w.  y is scratch of the blocked layout; r and z are blocked.
template <typename T, int M>
__global__ void __launch_bounds__(128) k_tsp(const LevelView<T> L, T w_ic, T w_bnd, const T* __restrict__ r,
                                            T* __restrict__ y, T* __restrict__ z) {
    extern __shared__ __align__(16) unsigned char tsp_smem[];
    const int nx = L.nx, nt = L.nt;
    const long long N = L.N;
    const int NXP = nx + (nx >> 5) + 1;           // padded row length
    T* sin = reinterpret_cast<T*>(tsp_smem);      // [2][4][NXP] staged input rows
    T* smu = sin + 2 * 4 * NXP;                   // [2][NXP] staged linearisation point
    const int blk = blockIdx.x, tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const bool burgers = L.col.kind == 2;
    const int m = (nx + 31) / 32;
    const int s0 = lane * m, mi = max(0, min(m, nx - s0));
    const T inv_dt = (T)L.col.inv_dt;
    const T wq = (T)L.col.qeps;
    auto stage = [&](const T* src, int k, int slot) {
        if (k < 0 || k >= nt) return;
        const T* g = src + ((size_t)blk * N + (size_t)k * nx) * RW;
        T* d = sin + (size_t)slot * 4 * NXP;
        for (int e = tid; e < 4 * nx; e += 128) {
            const int x = e >> 2, c = e & 3;
            cp_scalar<T>(d + (size_t)c * NXP + x + (x >> 5), g + e, true);
        }
        if (burgers) {
            const T* gm = L.mu + (size_t)k * nx;
            T* dm = smu + (size_t)slot * NXP;
            for (int x = tid; x < nx; x += 128) cp_scalar<T>(dm + x + (x >> 5), gm + x, true);
        }
    };
    // interior rows j < mi - 1 in registers, the separator row (x = s0 + mi - 1) apart
    T xv[M], carry[M], csep = T(0);
#pragma unroll
    for (int j = 0; j < M; ++j) carry[j] = T(0);
    const int xs = s0 + mi - 1;
    const bool xs_int = xs > 0 && xs < nx - 1;
    // backward sweep: J^T y = r from the last level down, then y / W
    stage(r, nt - 1, 0);
    cp_commit();
    for (int k = nt - 1; k >= 0; --k) {
        const int slot = (nt - 1 - k) & 1;
        cp_wait<0>();
        __syncthreads();                  // level k landed; level k+1's buffers are free
        stage(r, k - 1, slot ^ 1);
        cp_commit();
        const T* in = sin + (size_t)slot * 4 * NXP + (size_t)w * NXP;
        const T* mu = smu + (size_t)slot * NXP;
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
        warp_tridiag<T, true, M>(L, mu, k, s0, mi, xv, dsep, X);
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
    // every warp's y rows must be visible to the CTA's staging copies
    __threadfence_block();
#pragma unroll
    for (int j = 0; j < M; ++j) carry[j] = T(0);
    csep = T(0);
    // forward sweep: J z = W^-1 y from the first level up
    stage(y, 0, 0);
    cp_commit();
    for (int k = 0; k < nt; ++k) {
        const int slot = k & 1;
        cp_wait<0>();
        __syncthreads();
        stage(y, k + 1, slot ^ 1);
        cp_commit();
        const T* in = sin + (size_t)slot * 4 * NXP + (size_t)w * NXP;
        const T* mu = smu + (size_t)slot * NXP;
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
        warp_tridiag<T, false, M>(L, mu, k, s0, mi, xv, dsep, X);
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

template <typename T>
void launch_tsp(const Level& L, double w_ic, double w_bnd, const T* r, T* y, T* z, int nblk, cudaStream_t s) {
    const int nxp = L.nx + (L.nx >> 5) + 1;
    const size_t smem = sizeof(T) * (size_t)(2 * 4 * nxp + 2 * nxp);
    static size_t attr = 0;
    if (smem > attr) {
        if (cudaFuncSetAttribute(k_tsp<T, kTspRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            throw Error(GMRF_E_CUDA, "time-stepping preconditioner: shared memory attribute");
        attr = smem;
    }
    k_tsp<T, kTspRows><<<nblk, 128, smem, s>>>(L.view<T>(), (T)w_ic, (T)w_bnd, r, y, z);
    note_launch();
}
template void launch_tsp<float>(const Level&, double, double, const float*, float*, float*, int, cudaStream_t);
template void launch_tsp<double>(const Level&, double, double, const double*, double*, double*, int, cudaStream_t);

}  // namespace gmrf
