// Kernels of the GB300 GMRF solver.
//
// The posterior precision Q_u|y = B^T B + J^T Q_eps J + A^T R^-1 A
// (Sec. 3.1 eq. posterior-mean; B the stacked root of the SPDE prior,
// Sec. 2.2 eq. sparse-prec-matrix and App. A; J the collocation rows,
// Sec. 3.3) is never stored.  One CTA stages a tile of the input vector
// with its halo in shared memory, forms s = B p on the tile plus a one-node
// ring, applies B^T back onto the tile, adds the observation rows of the
// tile from a per-tile list, and finishes with a mode-specific epilogue.
// All traffic is HBM-bound (about 3 flop per byte), so nothing here uses
// tensor cores.
#include <atomic>
#include <cstdio>

#include "kernels.h"

namespace gmrf {

// launch accounting: direct launches count one each; a CUDA graph counts the
// kernels captured into it on every replay
static std::atomic<unsigned long long> g_launches{0};
static thread_local bool g_capturing = false;
static thread_local unsigned long long g_captured = 0;
void note_launch() {
    if (g_capturing) ++g_captured;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
}
void capture_begin() { g_capturing = true; g_captured = 0; }
unsigned long long capture_end() { g_capturing = false; return g_captured; }
void note_graph_launch(unsigned long long kernels) { g_launches.fetch_add(kernels, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(); }


template <typename T> LevelView<T> Level::view() const {
    LevelView<T> v;
    v.nx = nx; v.ny = ny; v.nt = nt; v.N = N;
    v.tiles_x = tiles_x; v.tiles_y = tiles_y; v.tiles_t = tiles_t;
    for (int c = 0; c < 2; ++c)
        for (int o = 0; o < NTAP; ++o) v.cf[c][o] = (T)cd[c][o];
    v.inv_eps2 = (T)inv_eps2;
    v.inv_eps = (T)inv_eps;
    v.col = col;
    if constexpr (sizeof(T) == 4) v.mu = d_mu32;
    else v.mu = d_mu64;
    v.obs = d_obs;
    v.tile_ptr = d_tile_ptr;
    v.tile_idx = d_tile_idx;
    return v;
}

template LevelView<float> Level::view<float>() const;
template LevelView<double> Level::view<double>() const;

__device__ __forceinline__ bool is_dirichlet(int x, int y, int nx, int ny) {
    return x == 0 || x == nx - 1 || (ny > 1 && (y == 0 || y == ny - 1));
}

template <typename T> __device__ __forceinline__ T obs_w(const ObsRow& o, int n);
template <> __device__ __forceinline__ float obs_w<float>(const ObsRow& o, int n) { return o.wf[n]; }
template <> __device__ __forceinline__ double obs_w<double>(const ObsRow& o, int n) { return o.wd[n]; }
template <typename T> __device__ __forceinline__ T obs_rinv(const ObsRow& o);
template <> __device__ __forceinline__ float obs_rinv<float>(const ObsRow& o) { return o.rinvf; }
template <> __device__ __forceinline__ double obs_rinv<double>(const ObsRow& o) { return o.rinv; }

// Collocation row coefficients at row (rx, rt): centre, x-1, x+1, t-1.
template <typename T, int COL>
__device__ __forceinline__ void jcoef(const Colloc& c, T mu_c, T mu_l, T mu_r, T& cC, T& cL, T& cR) {
    const T inv_2h = (T)c.inv_2h, nu_h2 = (T)c.nu_h2;
    T a, da;
    if (COL == 1) { a = (T)c.c; da = T(0); }
    else { a = mu_c; da = (mu_r - mu_l) * inv_2h; }
    cC = (T)c.inv_dt + da + T(2) * nu_h2;
    cL = -a * inv_2h - nu_h2;
    cR = a * inv_2h - nu_h2;
}

// ---------------------------------------------------------------------------
// fused posterior-precision stencil

template <int GEO, typename T, int MODE, int COL>
__global__ void __launch_bounds__(256) k_stencil(const StencilArgs<T> A) {
    using G = Geo<GEO>;
    constexpr int TX = G::TX, TY = G::TY, TT = G::TT, HY = G::HY, HT = G::HT;
    constexpr int PX = TX + 4, PY = TY + 2 * HY, PT = TT + 2 * HT;
    constexpr int SX = TX + 2, SY = TY + HY, ST = TT + HT;
    constexpr int HYS = HY / 2;
    static_assert(SX * SY * ST >= TX * TY * TT, "q staging aliases the s tile");
    __shared__ V4<T> sp[PT][PY][PX];
    __shared__ V4<T> ss[ST][SY][SX];
    __shared__ V4<T> sj[COL ? ST : 1][COL ? SY : 1][COL ? SX : 1];
    __shared__ T smu[COL == 2 ? PT : 1][COL == 2 ? PY : 1][COL == 2 ? PX : 1];

    const LevelView<T>& L = A.L;
    const int nx = L.nx, ny = L.ny, nt = L.nt;
    const long long N = L.N;
    const int tile = blockIdx.x, blk = blockIdx.y, tid = threadIdx.x;
    const int tx0 = (tile % L.tiles_x) * TX;
    const int rest = tile / L.tiles_x;
    const int ty0 = (rest % L.tiles_y) * TY;
    const int tt0 = (rest / L.tiles_y) * TT;
    const T* xb = A.x + (size_t)blk * N * RW;

    // 1. stage the input tile with halo
    for (int e = tid; e < PX * PY * PT; e += 256) {
        const int px = e % PX, py = (e / PX) % PY, pt = e / (PX * PY);
        const int gx = tx0 - 2 + px, gy = ty0 - HY + py, gt = tt0 - HT + pt;
        const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny && gt >= 0 && gt < nt;
        const long long node = ((long long)gt * ny + gy) * nx + gx;
        sp[pt][py][px] = in ? v4load(xb + node * RW) : v4zero<T>();
        if (COL == 2) smu[COL == 2 ? pt : 0][COL == 2 ? py : 0][COL == 2 ? px : 0] = in ? L.mu[node] : T(0);
    }
    __syncthreads();

    // 2. s = B p (Dirichlet columns masked) and sj = J p on the ring-extended tile
    for (int e = tid; e < SX * SY * ST; e += 256) {
        const int sx = e % SX, sy = (e / SX) % SY, st = e / (SX * SY);
        const int rx = tx0 - 1 + sx, ry = ty0 - HYS + sy, rt = tt0 + st;
        const bool inrow = rx >= 0 && rx < nx && ry >= 0 && ry < ny && rt < nt;
        V4<T> s = v4zero<T>();
        if (inrow && !is_dirichlet(rx, ry, nx, ny)) {
            const int cls = (nt > 1 && rt == 0) ? 1 : 0;
#pragma unroll
            for (int o = 0; o < NTAP; ++o) {
                if (HY == 0 && tap_dy(o) != 0) continue;
                if (HT == 0 && tap_dt(o) != 0) continue;
                const T c = L.cf[cls][o];
                const int qx = rx + tap_dx(o), qy = ry + tap_dy(o), qt = rt + tap_dt(o);
                if (c == T(0) || is_dirichlet(qx, qy, nx, ny)) continue;
                s = fma4(c, sp[qt - tt0 + HT][qy - ty0 + HY][qx - tx0 + 2], s);
            }
        }
        ss[st][sy][sx] = s;
        if (COL) {
            V4<T> sjv = v4zero<T>();
            if (inrow && rx >= 1 && rx <= nx - 2 && rt >= 1) {
                const int px = rx - tx0 + 2, pt = rt - tt0 + HT;
                T cC, cL, cR;
                if (COL == 2)
                    jcoef<T, COL>(L.col, smu[COL == 2 ? pt : 0][0][COL == 2 ? px : 0],
                                  smu[COL == 2 ? pt : 0][0][COL == 2 ? px - 1 : 0],
                                  smu[COL == 2 ? pt : 0][0][COL == 2 ? px + 1 : 0], cC, cL, cR);
                else
                    jcoef<T, COL>(L.col, T(0), T(0), T(0), cC, cL, cR);
                sjv = cC * sp[pt][0][px];
                sjv = fma4(cL, sp[pt][0][px - 1], sjv);
                sjv = fma4(cR, sp[pt][0][px + 1], sjv);
                sjv = fma4((T)(-L.col.inv_dt), sp[pt - 1][0][px], sjv);
            }
            sj[COL ? st : 0][0][COL ? sx : 0] = sjv;
        }
    }
    __syncthreads();

    // 3. q = B^T s (+ J^T Q_eps sj) at the thread's own node
    const int lx = tid % TX, ly = (tid / TX) % TY, lt = tid / (TX * TY);
    const int gx = tx0 + lx, gy = ty0 + ly, gt = tt0 + lt;
    const bool own = gx < nx && gy < ny && gt < nt;
    const V4<T> pown = sp[lt + HT][ly + HY][lx + 2];
    V4<T> q = v4zero<T>();
    if (own) {
        if (is_dirichlet(gx, gy, nx, ny)) {
            q = L.inv_eps2 * pown;
        } else {
#pragma unroll
            for (int o = 0; o < NTAP; ++o) {
                if (HY == 0 && tap_dy(o) != 0) continue;
                if (HT == 0 && tap_dt(o) != 0) continue;
                const int rt = gt - tap_dt(o);
                const int cls = (nt > 1 && rt == 0) ? 1 : 0;
                const T c = L.cf[cls][o];
                if (c == T(0)) continue;
                q = fma4(c, ss[lt - tap_dt(o)][ly + HYS - tap_dy(o)][lx + 1 - tap_dx(o)], q);
            }
        }
        if (COL) {
            // rows touching this column: itself (centre), x-1 row (its x+1 tap),
            // x+1 row (its x-1 tap), t+1 row (its t-1 tap)
            const int px = lx + 2, pt = lt + HT;
            T cC, cL, cR, tC, tL, tR;
            V4<T> acc = v4zero<T>();
            const T m0 = COL == 2 ? smu[COL == 2 ? pt : 0][0][COL == 2 ? px : 0] : T(0);
            const T mm1 = COL == 2 ? smu[COL == 2 ? pt : 0][0][COL == 2 ? px - 1 : 0] : T(0);
            const T mp1 = COL == 2 ? smu[COL == 2 ? pt : 0][0][COL == 2 ? px + 1 : 0] : T(0);
            const T mm2 = COL == 2 ? smu[COL == 2 ? pt : 0][0][COL == 2 ? px - 2 : 0] : T(0);
            const T mp2 = COL == 2 ? smu[COL == 2 ? pt : 0][0][COL == 2 ? px + 2 : 0] : T(0);
            jcoef<T, COL>(L.col, m0, mm1, mp1, cC, cL, cR);
            acc = cC * sj[COL ? lt : 0][0][COL ? lx + 1 : 0];
            jcoef<T, COL>(L.col, mm1, mm2, m0, tC, tL, tR);     // row x-1
            acc = fma4(tR, sj[COL ? lt : 0][0][COL ? lx : 0], acc);
            jcoef<T, COL>(L.col, mp1, m0, mp2, tC, tL, tR);     // row x+1
            acc = fma4(tL, sj[COL ? lt : 0][0][COL ? lx + 2 : 0], acc);
            acc = fma4((T)(-L.col.inv_dt), sj[COL ? lt + 1 : 0][0][COL ? lx + 1 : 0], acc);
            q = fma4((T)L.col.qeps, acc, q);
        }
    }
    __syncthreads();

    // 4. observation rows of this tile: A^T R^-1 A p, scattered in shared memory
    if (L.obs != nullptr) {
        const int k0 = L.tile_ptr[tile], k1 = L.tile_ptr[tile + 1];
        if (k1 > k0) {
            V4<T>* sq = &ss[0][0][0];
            sq[tid] = q;
            __syncthreads();
            for (int k = k0 + tid; k < k1; k += 256) {
                const ObsRow& o = L.obs[L.tile_idx[k]];
                int li[8];
                V4<T> a = v4zero<T>();
                for (int n = 0; n < o.nn; ++n) {
                    const long long nd = o.node[n];
                    const int ox = (int)(nd % nx);
                    const long long r2 = nd / nx;
                    const int oy = (int)(r2 % ny), ot = (int)(r2 / ny);
                    a = fma4(obs_w<T>(o, n), sp[ot - tt0 + HT][oy - ty0 + HY][ox - tx0 + 2], a);
                    const int ux = ox - tx0, uy = oy - ty0, ut = ot - tt0;
                    li[n] = (ux >= 0 && ux < TX && uy >= 0 && uy < TY && ut >= 0 && ut < TT) ? (ut * TY + uy) * TX + ux : -1;
                }
                a = obs_rinv<T>(o) * a;
                for (int n = 0; n < o.nn; ++n) {
                    if (li[n] < 0) continue;
                    const T w = obs_w<T>(o, n);
                    T* dst = reinterpret_cast<T*>(&sq[li[n]]);
                    atomicAdd(dst + 0, w * a.a);
                    atomicAdd(dst + 1, w * a.b);
                    atomicAdd(dst + 2, w * a.c);
                    atomicAdd(dst + 3, w * a.d);
                }
            }
            __syncthreads();
            q = sq[tid];
        }
    }

    // 5. epilogue
    double dot[4] = {0.0, 0.0, 0.0, 0.0};
    if (own) {
        const long long node = ((long long)gt * ny + gy) * nx + gx;
        const size_t off = ((size_t)blk * N + node) * RW;
        if (MODE == M_APPLY) {
            v4store(A.out + off, q);
            dot[0] = (double)pown.a * q.a; dot[1] = (double)pown.b * q.b;
            dot[2] = (double)pown.c * q.c; dot[3] = (double)pown.d * q.d;
        } else if (MODE == M_RESID) {
            const V4<T> r = v4load(A.b + off) - q;
            v4store(A.out + off, r);
            dot[0] = (double)r.a * r.a; dot[1] = (double)r.b * r.b;
            dot[2] = (double)r.c * r.c; dot[3] = (double)r.d * r.d;
        } else {
            const V4<T> bb = v4load(A.b + off);
            const V4<T> r = bb - q;
            const T di = A.dinv[node];
            V4<T> dn = (A.c2 * di) * r;
            if (A.d != nullptr) dn = fma4(A.c1, v4load(A.d + off), dn);
            const V4<T> xn = pown + dn;
            v4store(A.out + off, xn);
            v4store(A.out2 + off, dn);
            dot[0] = (double)bb.a * xn.a; dot[1] = (double)bb.b * xn.b;
            dot[2] = (double)bb.c * xn.c; dot[3] = (double)bb.d * xn.d;
        }
    }
    if (A.partial != nullptr) {
        const long long ntiles = (long long)L.tiles_x * L.tiles_y * L.tiles_t;
        block_sum4<256>(dot, A.partial + ((size_t)blk * ntiles + tile) * 4);
    }
}

template <int GEO, typename T, int MODE>
static void launch_geo_mode(const StencilArgs<T>& a, cudaStream_t s) {
    const dim3 grid((unsigned)((long long)a.L.tiles_x * a.L.tiles_y * a.L.tiles_t), (unsigned)a.nblk);
    if (GEO == GEO_XT && a.L.col.kind == 1)
        { k_stencil<GEO, T, MODE, (GEO == GEO_XT ? 1 : 0)><<<grid, 256, 0, s>>>(a); note_launch(); }
    else if (GEO == GEO_XT && a.L.col.kind == 2)
        { k_stencil<GEO, T, MODE, (GEO == GEO_XT ? 2 : 0)><<<grid, 256, 0, s>>>(a); note_launch(); }
    else
        { k_stencil<GEO, T, MODE, 0><<<grid, 256, 0, s>>>(a); note_launch(); }
}

template <typename T, int GEO>
static void launch_geo(int mode, const StencilArgs<T>& a, cudaStream_t s) {
    if (mode == M_APPLY) launch_geo_mode<GEO, T, M_APPLY>(a, s);
    else if (mode == M_RESID) launch_geo_mode<GEO, T, M_RESID>(a, s);
    else launch_geo_mode<GEO, T, M_CHEB>(a, s);
}

template <typename T> void launch_stencil(int geo, int mode, const StencilArgs<T>& a, cudaStream_t s) {
    if (geo == GEO_XY) launch_geo<T, GEO_XY>(mode, a, s);
    else if (geo == GEO_XT) launch_geo<T, GEO_XT>(mode, a, s);
    else launch_geo<T, GEO_XYT>(mode, a, s);
}
template void launch_stencil<float>(int, int, const StencilArgs<float>&, cudaStream_t);
template void launch_stencil<double>(int, int, const StencilArgs<double>&, cudaStream_t);

// ---------------------------------------------------------------------------
// reductions and PCG scalars

__global__ void k_reduce(const double* __restrict__ partial, int nparts, double* __restrict__ out) {
    const int blk = blockIdx.x;
    double v[4] = {0, 0, 0, 0};
    for (int i = threadIdx.x; i < nparts; i += 256) {
        const double* p = partial + ((size_t)blk * nparts + i) * 4;
        v[0] += p[0]; v[1] += p[1]; v[2] += p[2]; v[3] += p[3];
    }
    block_sum4<256>(v, out + (size_t)blk * 4);
}

void launch_reduce(const double* partial, int nparts, int nblk, double* out, cudaStream_t s) {
    { k_reduce<<<nblk, 256, 0, s>>>(partial, nparts, out); note_launch(); }
}

// kind 0: pq reduced -> alpha = active ? rz / pq : 0 (breakdown if pq <= 0)
// kind 1: rr reduced -> active = rr > tol2 * rr0
// kind 2: rz_new reduced -> beta = rz_new / rz, rz = rz_new
// kind 3: initial: rz reduced, rr0 = rr (stored by kind 4), active = rr0 > 0
// kind 4: rr reduced -> rr
__global__ void k_pcg_scalar(int kind, const double* __restrict__ red, double* __restrict__ sc, int P, double tol2) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= P) return;
    double* rz = sc, *pq = sc + P, *alpha = sc + 2 * P, *beta = sc + 3 * P;
    double* rr = sc + 4 * P, *rr0 = sc + 5 * P, *active = sc + 6 * P, *brk = sc + 7 * P;
    const double v = red[r];
    if (kind == 0) {
        pq[r] = v;
        const bool ok = v > 0.0 && isfinite(v) && isfinite(rz[r]);
        if (active[r] != 0.0 && !ok) { brk[r] = 1.0; active[r] = 0.0; }
        alpha[r] = (active[r] != 0.0) ? rz[r] / v : 0.0;
    } else if (kind == 1) {
        rr[r] = v;
        if (!(v > tol2 * rr0[r])) active[r] = 0.0;
    } else if (kind == 2) {
        beta[r] = (active[r] != 0.0 && rz[r] != 0.0) ? v / rz[r] : 0.0;
        rz[r] = v;
    } else if (kind == 4) {
        rr[r] = v;
    } else {
        rz[r] = v;
        rr0[r] = rr[r];
        active[r] = (rr[r] > 0.0) ? 1.0 : 0.0;
        brk[r] = 0.0;
        beta[r] = 0.0;
        alpha[r] = 0.0;
    }
}

void launch_pcg_scalar(int kind, const double* red, double* sc, int nblk, double tol2, cudaStream_t s) {
    const int P = nblk * RW;
    { k_pcg_scalar<<<(P + 127) / 128, 128, 0, s>>>(kind, red, sc, P, tol2); note_launch(); }
}

constexpr int EPT = 4;                  // nodes per thread in elementwise kernels
constexpr int ECHUNK = 256 * EPT;       // nodes per CTA
int elem_parts(long long N) { return (int)((N + ECHUNK - 1) / ECHUNK); }

template <typename T>
__global__ void __launch_bounds__(256) k_update_xr(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                   const T* __restrict__ q, const double* __restrict__ sc, long long N,
                                                   double* __restrict__ partial, int nparts) {
    const int blk = blockIdx.y;
    const double* alpha = sc + 2 * (gridDim.y * RW) + blk * RW;
    const T a0 = (T)alpha[0], a1 = (T)alpha[1], a2 = (T)alpha[2], a3 = (T)alpha[3];
    double dot[4] = {0, 0, 0, 0};
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<T> pv = v4load(p + off), qv = v4load(q + off);
        V4<T> xv = v4load(x + off), rv = v4load(r + off);
        xv.a = fma(a0, pv.a, xv.a); xv.b = fma(a1, pv.b, xv.b); xv.c = fma(a2, pv.c, xv.c); xv.d = fma(a3, pv.d, xv.d);
        rv.a = fma(-a0, qv.a, rv.a); rv.b = fma(-a1, qv.b, rv.b); rv.c = fma(-a2, qv.c, rv.c); rv.d = fma(-a3, qv.d, rv.d);
        v4store(x + off, xv);
        v4store(r + off, rv);
        dot[0] += (double)rv.a * rv.a; dot[1] += (double)rv.b * rv.b;
        dot[2] += (double)rv.c * rv.c; dot[3] += (double)rv.d * rv.d;
    }
    block_sum4<256>(dot, partial + ((size_t)blk * nparts + blockIdx.x) * 4);
}

template <typename T>
void launch_pcg_update_xr(T* x, T* r, const T* p, const T* q, const double* sc, long long N, int nblk,
                          double* partial, int nparts, cudaStream_t s) {
    { k_update_xr<T><<<dim3(nparts, nblk), 256, 0, s>>>(x, r, p, q, sc, N, partial, nparts); note_launch(); }
}
template void launch_pcg_update_xr<float>(float*, float*, const float*, const float*, const double*, long long, int, double*, int, cudaStream_t);
template void launch_pcg_update_xr<double>(double*, double*, const double*, const double*, const double*, long long, int, double*, int, cudaStream_t);

template <typename T>
__global__ void __launch_bounds__(256) k_update_p(T* __restrict__ p, const T* __restrict__ z, const double* __restrict__ sc, long long N) {
    const int blk = blockIdx.y;
    const double* beta = sc + 3 * (gridDim.y * RW) + blk * RW;
    const T b0 = (T)beta[0], b1 = (T)beta[1], b2 = (T)beta[2], b3 = (T)beta[3];
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<T> zv = v4load(z + off);
        V4<T> pv = v4load(p + off);
        pv.a = fma(b0, pv.a, zv.a); pv.b = fma(b1, pv.b, zv.b); pv.c = fma(b2, pv.c, zv.c); pv.d = fma(b3, pv.d, zv.d);
        v4store(p + off, pv);
    }
}

template <typename T>
void launch_pcg_update_p(T* p, const T* z, const double* sc, long long N, int nblk, cudaStream_t s) {
    { k_update_p<T><<<dim3(elem_parts(N), nblk), 256, 0, s>>>(p, z, sc, N); note_launch(); }
}
template void launch_pcg_update_p<float>(float*, const float*, const double*, long long, int, cudaStream_t);
template void launch_pcg_update_p<double>(double*, const double*, const double*, long long, int, cudaStream_t);

// ---------------------------------------------------------------------------
// multigrid pieces

template <typename T>
__global__ void __launch_bounds__(256) k_cheb_first(const T* __restrict__ b, const T* __restrict__ dinv, T c2,
                                                    T* __restrict__ x, T* __restrict__ d, long long N) {
    const int blk = blockIdx.y;
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<T> v = (c2 * dinv[n]) * v4load(b + off);
        v4store(x + off, v);
        if (d != nullptr) v4store(d + off, v);
    }
}

template <typename T>
void launch_cheb_first(const T* b, const T* dinv, T c2, T* x, T* d, long long N, int nblk, cudaStream_t s) {
    { k_cheb_first<T><<<dim3(elem_parts(N), nblk), 256, 0, s>>>(b, dinv, c2, x, d, N); note_launch(); }
}
template void launch_cheb_first<float>(const float*, const float*, float, float*, float*, long long, int, cudaStream_t);
template void launch_cheb_first<double>(const double*, const double*, double, double*, double*, long long, int, cudaStream_t);

// Restriction along one axis: out[.., J, ..] = sum_i P_iJ in[.., i, ..] with
// P_iJ = 1 - w(i) if j(i) = J, w(i) if j(i) + 1 = J (transpose of linear
// interpolation); fine indices with a non-zero weight form [rs(J), rs(J)+rc(J)).
template <typename T>
__global__ void __launch_bounds__(256) k_restrict_axis(const T* __restrict__ in, T* __restrict__ out, int nx, int ny,
                                                       int nt, int axis, int nc, const int32_t* __restrict__ rs,
                                                       const int32_t* __restrict__ rc, const int32_t* __restrict__ pj,
                                                       const T* __restrict__ pw) {
    const int ox = axis == 0 ? nc : nx, oy = axis == 1 ? nc : ny, ot = axis == 2 ? nc : nt;
    const long long Nout = (long long)ox * oy * ot, Nin = (long long)nx * ny * nt;
    const int blk = blockIdx.y;
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= Nout) return;
    const int x = (int)(n % ox);
    const long long r = n / ox;
    const int y = (int)(r % oy), t = (int)(r / oy);
    const int J = axis == 0 ? x : (axis == 1 ? y : t);
    const long long stride = axis == 0 ? 1 : (axis == 1 ? (long long)nx : (long long)nx * ny);
    const long long base = ((long long)(axis == 2 ? 0 : t) * ny + (axis == 1 ? 0 : y)) * nx + (axis == 0 ? 0 : x);
    V4<T> acc = v4zero<T>();
    const int i0 = rs[J], cnt = rc[J];
    for (int k = 0; k < cnt; ++k) {
        const int i = i0 + k;
        const int j = pj[i];
        const T w = j == J ? T(1) - pw[i] : (j + 1 == J ? pw[i] : T(0));
        acc = fma4(w, v4load(in + ((size_t)blk * Nin + base + (long long)i * stride) * RW), acc);
    }
    v4store(out + ((size_t)blk * Nout + n) * RW, acc);
}

template <typename T>
void launch_restrict_axis(const T* in, T* out, int nx, int ny, int nt, int axis, int ncoarse, const int32_t* rs,
                          const int32_t* rc, const int32_t* pj, const T* pw, int nblk, cudaStream_t s) {
    const long long Nout = (long long)(axis == 0 ? ncoarse : nx) * (axis == 1 ? ncoarse : ny) * (axis == 2 ? ncoarse : nt);
    { k_restrict_axis<T><<<dim3((unsigned)((Nout + 255) / 256), nblk), 256, 0, s>>>(in, out, nx, ny, nt, axis, ncoarse, rs, rc, pj, pw); note_launch(); }
}
template void launch_restrict_axis<float>(const float*, float*, int, int, int, int, int, const int32_t*, const int32_t*, const int32_t*, const float*, int, cudaStream_t);
template void launch_restrict_axis<double>(const double*, double*, int, int, int, int, int, const int32_t*, const int32_t*, const int32_t*, const double*, int, cudaStream_t);

struct AxisMap { const int32_t* j; const void* w; bool on; };

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(T* __restrict__ xf, const T* __restrict__ xc, int nx, int ny, int nt,
                                                     int cx, int cy, int ct, AxisMap ax, AxisMap ay, AxisMap at) {
    const long long Nf = (long long)nx * ny * nt, Nc = (long long)cx * cy * ct;
    const int blk = blockIdx.y;
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= Nf) return;
    const int x = (int)(n % nx);
    const long long r = n / nx;
    const int y = (int)(r % ny), t = (int)(r / ny);
    int jx = x, jy = y, jt = t;
    T wx = T(0), wy = T(0), wt = T(0);
    if (ax.on) { jx = ax.j[x]; wx = ((const T*)ax.w)[x]; }
    if (ay.on) { jy = ay.j[y]; wy = ((const T*)ay.w)[y]; }
    if (at.on) { jt = at.j[t]; wt = ((const T*)at.w)[t]; }
    const T* xb = xc + (size_t)blk * Nc * RW;
    V4<T> acc = v4zero<T>();
    for (int dt = 0; dt < (at.on ? 2 : 1); ++dt) {
        const T ft = at.on ? (dt ? wt : T(1) - wt) : T(1);
        for (int dy = 0; dy < (ay.on ? 2 : 1); ++dy) {
            const T fy = ay.on ? (dy ? wy : T(1) - wy) : T(1);
            for (int dx = 0; dx < (ax.on ? 2 : 1); ++dx) {
                const T fx = ax.on ? (dx ? wx : T(1) - wx) : T(1);
                const long long c = ((long long)(jt + dt) * cy + (jy + dy)) * cx + (jx + dx);
                acc = fma4(ft * fy * fx, v4load(xb + c * RW), acc);
            }
        }
    }
    const size_t off = ((size_t)blk * Nf + n) * RW;
    v4store(xf + off, v4load(xf + off) + acc);
}

template <typename T>
void launch_prolong_add(T* xf, const T* xc, const Level& f, const Level& c, int nblk, cudaStream_t s) {
    const bool dbl = sizeof(T) == 8;
    AxisMap ax{f.d_pj[0], dbl ? (const void*)f.d_pwd[0] : (const void*)f.d_pw[0], f.coarsen[0]};
    AxisMap ay{f.d_pj[1], dbl ? (const void*)f.d_pwd[1] : (const void*)f.d_pw[1], f.coarsen[1]};
    AxisMap at{f.d_pj[2], dbl ? (const void*)f.d_pwd[2] : (const void*)f.d_pw[2], f.coarsen[2]};
    { k_prolong_add<T><<<dim3((unsigned)((f.N + 255) / 256), nblk), 256, 0, s>>>(xf, xc, f.nx, f.ny, f.nt, c.nx, c.ny, c.nt, ax, ay, at); note_launch(); }
}
template void launch_prolong_add<float>(float*, const float*, const Level&, const Level&, int, cudaStream_t);
template void launch_prolong_add<double>(double*, const double*, const Level&, const Level&, int, cudaStream_t);

// coarsest level: x = Q_c^-1 b with the stored dense inverse
template <typename T>
__global__ void __launch_bounds__(256) k_dense_solve(const T* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ x, int n) {
    extern __shared__ unsigned char dsm[];
    V4<T>* sb = reinterpret_cast<V4<T>*>(dsm);
    const int blk = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += 256) sb[i] = v4load(b + ((size_t)blk * n + i) * RW);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += 256) {
        V4<T> acc = v4zero<T>();
        const T* row = Ainv + (size_t)i * n;
        for (int j = 0; j < n; ++j) acc = fma4(row[j], sb[j], acc);
        v4store(x + ((size_t)blk * n + i) * RW, acc);
    }
}

template <typename T> void launch_dense_solve(const T* Ainv, const T* b, T* x, int n, int nblk, cudaStream_t s) {
    { k_dense_solve<T><<<nblk, 256, (size_t)n * sizeof(V4<T>), s>>>(Ainv, b, x, n); note_launch(); }
}
template void launch_dense_solve<float>(const float*, const float*, float*, int, int, cudaStream_t);
template void launch_dense_solve<double>(const double*, const double*, double*, int, int, cudaStream_t);

// ---------------------------------------------------------------------------
// mixed precision refinement

__global__ void k_scale_cast(const double* __restrict__ r64, const double* __restrict__ norms, float* __restrict__ r32, long long N) {
    const int blk = blockIdx.y;
    const double* nm = norms + blk * RW;
    const double s0 = nm[0] > 0 ? 1.0 / nm[0] : 0.0, s1 = nm[1] > 0 ? 1.0 / nm[1] : 0.0;
    const double s2 = nm[2] > 0 ? 1.0 / nm[2] : 0.0, s3 = nm[3] > 0 ? 1.0 / nm[3] : 0.0;
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<double> r = v4load(r64 + off);
        v4store(r32 + off, V4<float>{(float)(r.a * s0), (float)(r.b * s1), (float)(r.c * s2), (float)(r.d * s3)});
    }
}
void launch_scale_cast(const double* r64, const double* norms, float* r32, long long N, int nblk, cudaStream_t s) {
    { k_scale_cast<<<dim3(elem_parts(N), nblk), 256, 0, s>>>(r64, norms, r32, N); note_launch(); }
}

__global__ void k_scale64(const double* __restrict__ r64, const double* __restrict__ norms, double* __restrict__ out, long long N) {
    const int blk = blockIdx.y;
    const double* nm = norms + blk * RW;
    const double s0 = nm[0] > 0 ? 1.0 / nm[0] : 0.0, s1 = nm[1] > 0 ? 1.0 / nm[1] : 0.0;
    const double s2 = nm[2] > 0 ? 1.0 / nm[2] : 0.0, s3 = nm[3] > 0 ? 1.0 / nm[3] : 0.0;
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<double> r = v4load(r64 + off);
        v4store(out + off, V4<double>{r.a * s0, r.b * s1, r.c * s2, r.d * s3});
    }
}
void launch_scale64(const double* r64, const double* norms, double* out, long long N, int nblk, cudaStream_t s) {
    { k_scale64<<<dim3(elem_parts(N), nblk), 256, 0, s>>>(r64, norms, out, N); note_launch(); }
}

template <typename T>
__global__ void k_axpy_norm(double* __restrict__ x64, const double* __restrict__ norms, const T* __restrict__ d, long long N) {
    const int blk = blockIdx.y;
    const double* nm = norms + blk * RW;
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<T> dv = v4load(d + off);
        V4<double> xv = v4load(x64 + off);
        xv.a = fma(nm[0], (double)dv.a, xv.a); xv.b = fma(nm[1], (double)dv.b, xv.b);
        xv.c = fma(nm[2], (double)dv.c, xv.c); xv.d = fma(nm[3], (double)dv.d, xv.d);
        v4store(x64 + off, xv);
    }
}
void launch_axpy_mixed(double* x64, const double* norms, const float* d32, long long N, int nblk, cudaStream_t s) {
    { k_axpy_norm<float><<<dim3(elem_parts(N), nblk), 256, 0, s>>>(x64, norms, d32, N); note_launch(); }
}
void launch_axpy_scaled64(double* x64, const double* norms, const double* d64, long long N, int nblk, cudaStream_t s) {
    { k_axpy_norm<double><<<dim3(elem_parts(N), nblk), 256, 0, s>>>(x64, norms, d64, N); note_launch(); }
}

// ---------------------------------------------------------------------------
// right-hand sides of perturbation samples: L z = B^T z1 + A^T Q_eps^1/2 z2
// (+ J^T Q_eps^1/2 z3), z drawn in-kernel (Sec. 3.2, left root of a sum).
// A slot with sample id -1 copies the data right-hand side, -2 is padding,
// >= 0 draws sample `id`.  With use_probe the slot holds a Rademacher probe.

template <int GEO>
__global__ void __launch_bounds__(256) k_sample_rhs(const LevelView<double> L, uint64_t seed,
                                                    const int32_t* __restrict__ slot_sample,
                                                    const double* __restrict__ bdata, double* __restrict__ b64) {
    using G = Geo<GEO>;
    constexpr int TX = G::TX, TY = G::TY, TT = G::TT, HY = G::HY, HT = G::HT;
    constexpr int HYS = HY / 2;
    constexpr int SX = TX + 2, SY = TY + HY, ST = TT + HT;
    __shared__ V4<double> sz[ST][SY][SX];       // z1 on the rows touching the tile
    __shared__ V4<double> sq[TT][TY][TX];
    const int nx = L.nx, ny = L.ny, nt = L.nt;
    const long long N = L.N;
    const int tile = blockIdx.x, blk = blockIdx.y, tid = threadIdx.x;
    const int tx0 = (tile % L.tiles_x) * TX;
    const int rest = tile / L.tiles_x;
    const int ty0 = (rest % L.tiles_y) * TY;
    const int tt0 = (rest / L.tiles_y) * TT;
    int sid[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) sid[c] = slot_sample[blk * RW + c];

    for (int e = tid; e < SX * SY * ST; e += 256) {
        const int sx = e % SX, sy = (e / SX) % SY, st = e / (SX * SY);
        const int rx = tx0 - 1 + sx, ry = ty0 - HYS + sy, rt = tt0 + st;
        V4<double> z = v4zero<double>();
        if (rx >= 0 && rx < nx && ry >= 0 && ry < ny && rt < nt) {
            const long long row = ((long long)rt * ny + ry) * nx + rx;
            double v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = sid[c] >= 0 ? philox_normal(seed, 0u, (uint32_t)sid[c], (uint64_t)row) : 0.0;
            z = V4<double>{v[0], v[1], v[2], v[3]};
        }
        sz[st][sy][sx] = z;
    }
    __syncthreads();

    const int lx = tid % TX, ly = (tid / TX) % TY, lt = tid / (TX * TY);
    const int gx = tx0 + lx, gy = ty0 + ly, gt = tt0 + lt;
    const bool own = gx < nx && gy < ny && gt < nt;
    V4<double> q = v4zero<double>();
    if (own) {
        if (is_dirichlet(gx, gy, nx, ny)) {
            q = L.inv_eps * sz[lt][ly + HYS][lx + 1];
        } else {
#pragma unroll
            for (int o = 0; o < NTAP; ++o) {
                if (HY == 0 && tap_dy(o) != 0) continue;
                if (HT == 0 && tap_dt(o) != 0) continue;
                const int rx = gx - tap_dx(o), ry = gy - tap_dy(o), rt = gt - tap_dt(o);
                if (rx < 0 || rx >= nx || ry < 0 || ry >= ny || rt >= nt) continue;
                if (is_dirichlet(rx, ry, nx, ny)) continue;     // Dirichlet rows touch only themselves
                const int cls = (nt > 1 && rt == 0) ? 1 : 0;
                const double c = L.cf[cls][o];
                if (c == 0.0) continue;
                q = fma4(c, sz[lt - tap_dt(o)][ly + HYS - tap_dy(o)][lx + 1 - tap_dx(o)], q);
            }
        }
        if (L.col.kind != 0) {
            // J^T Q_eps^1/2 z3: rows (x, t), (x-1, t), (x+1, t), (x, t+1) with draws on
            // stream 1 at row index row0 + (t - 1)(nx - 2) + (x - 1)
            const double sq_eps = sqrt(L.col.qeps);
            const double inv_2h = L.col.inv_2h, nu_h2 = L.col.nu_h2;
            auto mu_at = [&](int x, int t) -> double { return L.mu ? L.mu[(long long)t * nx + x] : 0.0; };
            auto coef = [&](int rx, int rt, int which) -> double {   // which: 0 centre, 1 x-1 tap, 2 x+1 tap
                double a, da;
                if (L.col.kind == 1) { a = L.col.c; da = 0.0; }
                else { a = mu_at(rx, rt); da = (mu_at(rx + 1, rt) - mu_at(rx - 1, rt)) * inv_2h; }
                if (which == 0) return L.col.inv_dt + da + 2.0 * nu_h2;
                if (which == 1) return -a * inv_2h - nu_h2;
                return a * inv_2h - nu_h2;
            };
            const int rxs[4] = {gx, gx - 1, gx + 1, gx};
            const int rts[4] = {gt, gt, gt, gt + 1};
            for (int k = 0; k < 4; ++k) {
                const int rx = rxs[k], rt = rts[k];
                if (rx < 1 || rx > nx - 2 || rt < 1 || rt >= nt) continue;
                const double c = k == 0 ? coef(rx, rt, 0) : (k == 1 ? coef(rx, rt, 2) : (k == 2 ? coef(rx, rt, 1) : -L.col.inv_dt));
                const uint64_t orow = (uint64_t)L.col.row0 + (uint64_t)(rt - 1) * (nx - 2) + (rx - 1);
                double v[4];
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) v[cc] = sid[cc] >= 0 ? philox_normal(seed, 1u, (uint32_t)sid[cc], orow) : 0.0;
                q = fma4(c * sq_eps, V4<double>{v[0], v[1], v[2], v[3]}, q);
            }
        }
    }
    sq[lt][ly][lx] = q;
    __syncthreads();
    if (L.obs != nullptr) {
        const int k0 = L.tile_ptr[tile], k1 = L.tile_ptr[tile + 1];
        for (int k = k0 + tid; k < k1; k += 256) {
            const ObsRow& o = L.obs[L.tile_idx[k]];
            double v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = sid[c] >= 0 ? philox_normal(seed, 1u, (uint32_t)sid[c], (uint64_t)o.row) : 0.0;
            const double sr = sqrt(o.rinv);
            for (int n = 0; n < o.nn; ++n) {
                const long long nd = o.node[n];
                const int ox = (int)(nd % nx);
                const long long r2 = nd / nx;
                const int oy = (int)(r2 % ny), ot = (int)(r2 / ny);
                const int ux = ox - tx0, uy = oy - ty0, ut = ot - tt0;
                if (ux < 0 || ux >= TX || uy < 0 || uy >= TY || ut < 0 || ut >= TT) continue;
                double* dst = reinterpret_cast<double*>(&sq[ut][uy][ux]);
                const double w = o.wd[n] * sr;
                atomicAdd(dst + 0, w * v[0]);
                atomicAdd(dst + 1, w * v[1]);
                atomicAdd(dst + 2, w * v[2]);
                atomicAdd(dst + 3, w * v[3]);
            }
        }
        __syncthreads();
    }
    if (own) {
        const long long node = ((long long)gt * ny + gy) * nx + gx;
        V4<double> out = sq[lt][ly][lx];
        double* po = reinterpret_cast<double*>(&out);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (sid[c] == -1) po[c] = bdata[node];
            else if (sid[c] < -1) po[c] = 0.0;
        }
        v4store(b64 + ((size_t)blk * N + node) * RW, out);
    }
}

void launch_sample_rhs(int geo, const LevelView<double>& L, uint64_t seed, const int32_t* slot_sample,
                       const double* bdata, double* b64, int nblk, int use_probe, cudaStream_t s) {
    (void)use_probe;
    const dim3 grid((unsigned)((long long)L.tiles_x * L.tiles_y * L.tiles_t), (unsigned)nblk);
    if (geo == GEO_XY) { k_sample_rhs<GEO_XY><<<grid, 256, 0, s>>>(L, seed, slot_sample, bdata, b64); note_launch(); }
    else if (geo == GEO_XT) { k_sample_rhs<GEO_XT><<<grid, 256, 0, s>>>(L, seed, slot_sample, bdata, b64); note_launch(); }
    else { k_sample_rhs<GEO_XYT><<<grid, 256, 0, s>>>(L, seed, slot_sample, bdata, b64); note_launch(); }
}

// Rademacher probes: slot id >= 0 holds probe `id` (stream 2), -1 the data rhs.
__global__ void k_rademacher_fill(uint64_t seed, const int32_t* __restrict__ slot_sample, double* __restrict__ b64, long long N) {
    const int blk = blockIdx.y;
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    double* p = b64 + ((size_t)blk * N + n) * RW;
    for (int c = 0; c < 4; ++c) {
        const int id = slot_sample[blk * RW + c];
        if (id >= 0) p[c] = philox_rademacher(seed, (uint32_t)id, (uint64_t)n);
        else if (id < -1) p[c] = 0.0;
    }
}
void launch_rademacher_fill(uint64_t seed, const int32_t* slot_sample, double* b64, long long N, int nblk, cudaStream_t s) {
    { k_rademacher_fill<<<dim3((unsigned)((N + 255) / 256), nblk), 256, 0, s>>>(seed, slot_sample, b64, N); note_launch(); }
}

// data right-hand side A^T R^-1 y of the point observations
__global__ void k_obs_scatter(const ObsRow* __restrict__ obs, int nobs, const double* __restrict__ y, double* __restrict__ b) {
    const int k = blockIdx.x * 256 + threadIdx.x;
    if (k >= nobs) return;
    const ObsRow& o = obs[k];
    const double v = o.rinv * y[o.row];
    for (int n = 0; n < o.nn; ++n) atomicAdd(b + o.node[n], o.wd[n] * v);
}
void launch_obs_scatter(const ObsRow* obs, int nobs, const double* y, double* b, cudaStream_t s) {
    if (nobs > 0) { k_obs_scatter<<<(nobs + 255) / 256, 256, 0, s>>>(obs, nobs, y, b); note_launch(); }
}

// layout conversion between blocked batches and [count][N] row-major arrays;
// slot_* gives, per slot, the row of the dense array (-1: none)
__global__ void k_pack(const double* __restrict__ src, double* __restrict__ dst, const int32_t* __restrict__ slot_src, long long N) {
    const int blk = blockIdx.y;
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    double v[4];
    for (int c = 0; c < 4; ++c) {
        const int row = slot_src[blk * RW + c];
        v[c] = row >= 0 ? src[(size_t)row * N + n] : 0.0;
    }
    v4store(dst + ((size_t)blk * N + n) * RW, V4<double>{v[0], v[1], v[2], v[3]});
}
void launch_pack(const double* src, double* dst, const int32_t* slot_src, long long N, int nblk, cudaStream_t s) {
    { k_pack<<<dim3((unsigned)((N + 255) / 256), nblk), 256, 0, s>>>(src, dst, slot_src, N); note_launch(); }
}

__global__ void k_unpack(const double* __restrict__ src, double* __restrict__ dst, const int32_t* __restrict__ slot_dst, long long N) {
    const int blk = blockIdx.y;
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    const V4<double> v = v4load(src + ((size_t)blk * N + n) * RW);
    const double vv[4] = {v.a, v.b, v.c, v.d};
    for (int c = 0; c < 4; ++c) {
        const int row = slot_dst[blk * RW + c];
        if (row >= 0) dst[(size_t)row * N + n] = vv[c];
    }
}
void launch_unpack(const double* src, double* dst, const int32_t* slot_dst, long long N, int nblk, cudaStream_t s) {
    { k_unpack<<<dim3((unsigned)((N + 255) / 256), nblk), 256, 0, s>>>(src, dst, slot_dst, N); note_launch(); }
}

// Rao-Blackwellised variance: e = (Q x - Q_ii x_i) / Q_ii per sample slot,
// var = 1/Q_ii + mean(e^2), se = std(e^2) / sqrt(ns)
__global__ void k_rbmc(const double* __restrict__ Qx, const double* __restrict__ x, const double* __restrict__ diag,
                       const int32_t* __restrict__ slot_sample, long long N, int nblk, int ns, double* __restrict__ var,
                       double* __restrict__ se) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    const double d = diag[n];
    double s1 = 0.0, s2 = 0.0;
    for (int blk = 0; blk < nblk; ++blk) {
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<double> qx = v4load(Qx + off), xv = v4load(x + off);
        const double a[4] = {qx.a, qx.b, qx.c, qx.d}, b[4] = {xv.a, xv.b, xv.c, xv.d};
        for (int c = 0; c < 4; ++c) {
            if (slot_sample[blk * RW + c] < 0) continue;
            const double e = (a[c] - d * b[c]) / d;
            s1 += e * e;
            s2 += e * e * e * e;
        }
    }
    const double m = s1 / ns;
    var[n] = 1.0 / d + m;
    if (se != nullptr) {
        const double v = ns > 1 ? (s2 - ns * m * m) / (ns - 1) : 0.0;
        se[n] = sqrt(fmax(v, 0.0) / ns);
    }
}
void launch_rbmc(const double* Qx, const double* x, const double* diag, const int32_t* slot_sample, long long N,
                 int nblk, int ns, double* var, double* se, cudaStream_t s) {
    { k_rbmc<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(Qx, x, diag, slot_sample, N, nblk, ns, var, se); note_launch(); }
}

// diagonal of B^T B + J^T Q_eps J at every node (observation part added by k_obs_diag)
template <typename T>
__global__ void k_diag(const LevelView<T> L, double* __restrict__ diag) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= L.N) return;
    const int nx = L.nx, ny = L.ny, nt = L.nt;
    const int x = (int)(n % nx);
    const long long r = n / nx;
    const int y = (int)(r % ny), t = (int)(r / ny);
    double d = 0.0;
    if (is_dirichlet(x, y, nx, ny)) {
        d = (double)L.inv_eps2;
    } else {
        for (int o = 0; o < NTAP; ++o) {
            const int rx = x - tap_dx(o), ry = y - tap_dy(o), rt = t - tap_dt(o);
            if (rx < 0 || rx >= nx || ry < 0 || ry >= ny || rt < 0 || rt >= nt) continue;
            if (is_dirichlet(rx, ry, nx, ny)) continue;
            const int cls = (nt > 1 && rt == 0) ? 1 : 0;
            const double c = (double)L.cf[cls][o];
            d += c * c;
        }
    }
    if (L.col.kind != 0) {
        auto mu_at = [&](int xx, int tt) -> double { return L.mu ? (double)L.mu[(long long)tt * nx + xx] : 0.0; };
        auto coef = [&](int rx, int rt, int which) -> double {
            double a, da;
            if (L.col.kind == 1) { a = L.col.c; da = 0.0; }
            else { a = mu_at(rx, rt); da = (mu_at(rx + 1, rt) - mu_at(rx - 1, rt)) * L.col.inv_2h; }
            if (which == 0) return L.col.inv_dt + da + 2.0 * L.col.nu_h2;
            if (which == 1) return -a * L.col.inv_2h - L.col.nu_h2;
            return a * L.col.inv_2h - L.col.nu_h2;
        };
        const int rxs[4] = {x, x - 1, x + 1, x};
        const int rts[4] = {t, t, t, t + 1};
        double acc = 0.0;
        for (int k = 0; k < 4; ++k) {
            const int rx = rxs[k], rt = rts[k];
            if (rx < 1 || rx > nx - 2 || rt < 1 || rt >= nt) continue;
            const double c = k == 0 ? coef(rx, rt, 0) : (k == 1 ? coef(rx, rt, 2) : (k == 2 ? coef(rx, rt, 1) : -L.col.inv_dt));
            acc += c * c;
        }
        d += L.col.qeps * acc;
    }
    diag[n] = d;
}
template <typename T> void launch_diag(int geo, const LevelView<T>& L, double* diag64, cudaStream_t s) {
    (void)geo;
    { k_diag<T><<<(unsigned)((L.N + 255) / 256), 256, 0, s>>>(L, diag64); note_launch(); }
}
template void launch_diag<float>(int, const LevelView<float>&, double*, cudaStream_t);
template void launch_diag<double>(int, const LevelView<double>&, double*, cudaStream_t);

__global__ void k_obs_diag(const ObsRow* __restrict__ obs, int nobs, double* __restrict__ diag) {
    const int k = blockIdx.x * 256 + threadIdx.x;
    if (k >= nobs) return;
    const ObsRow& o = obs[k];
    for (int n = 0; n < o.nn; ++n) atomicAdd(diag + o.node[n], o.wd[n] * o.wd[n] * o.rinv);
}
void launch_obs_diag(const ObsRow* obs, int nobs, double* diag, cudaStream_t s) {
    if (nobs > 0) { k_obs_diag<<<(nobs + 255) / 256, 256, 0, s>>>(obs, nobs, diag); note_launch(); }
}

__global__ void k_finish_diag(const double* __restrict__ diag, float* __restrict__ dinv32, double* __restrict__ dinv64, long long N) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    const double inv = 1.0 / diag[n];
    dinv32[n] = (float)inv;
    dinv64[n] = inv;
}
void launch_finish_diag(const double* diag, float* dinv32, double* dinv64, long long N, cudaStream_t s) {
    { k_finish_diag<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(diag, dinv32, dinv64, N); note_launch(); }
}

__global__ void k_normals(uint64_t seed, int stream, int sample0, int count, long long n, double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    const int s = blockIdx.y;
    if (i >= n || s >= count) return;
    out[(size_t)s * n + i] = philox_normal(seed, (uint32_t)stream, (uint32_t)(sample0 + s), (uint64_t)i);
}
void launch_normals(uint64_t seed, int stream, int sample0, int count, long long n, double* out, cudaStream_t s) {
    { k_normals<<<dim3((unsigned)((n + 255) / 256), count), 256, 0, s>>>(seed, stream, sample0, count, n, out); note_launch(); }
}

template <typename T>
__global__ void k_cast(const double* __restrict__ in, T* __restrict__ out, long long n) {
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i < n) out[i] = (T)in[i];
}
template <typename T> void launch_cast(const double* in, T* out, long long n, cudaStream_t s) {
    { k_cast<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n); note_launch(); }
}
template void launch_cast<float>(const double*, float*, long long, cudaStream_t);
template void launch_cast<double>(const double*, double*, long long, cudaStream_t);

__global__ void k_dot_blocked(const double* __restrict__ a, const double* __restrict__ b, long long N, double* __restrict__ partial, int nparts) {
    const int blk = blockIdx.y;
    double dot[4] = {0, 0, 0, 0};
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<double> av = v4load(a + off), bv = v4load(b + off);
        dot[0] += av.a * bv.a; dot[1] += av.b * bv.b; dot[2] += av.c * bv.c; dot[3] += av.d * bv.d;
    }
    block_sum4<256>(dot, partial + ((size_t)blk * nparts + blockIdx.x) * 4);
}
void launch_dot_blocked(const double* a, const double* b, long long N, int nblk, double* partial, int nparts, cudaStream_t s) {
    { k_dot_blocked<<<dim3(nparts, nblk), 256, 0, s>>>(a, b, N, partial, nparts); note_launch(); }
}

}  // namespace gmrf

namespace gmrf {

// ---------------------------------------------------------------------------
// small helpers of the solver driver

template <typename T>
__global__ void k_norm2(const T* __restrict__ v, long long N, double* __restrict__ partial, int nparts) {
    const int blk = blockIdx.y;
    double dot[4] = {0, 0, 0, 0};
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const V4<T> a = v4load(v + ((size_t)blk * N + n) * RW);
        dot[0] += (double)a.a * a.a; dot[1] += (double)a.b * a.b; dot[2] += (double)a.c * a.c; dot[3] += (double)a.d * a.d;
    }
    block_sum4<256>(dot, partial + ((size_t)blk * nparts + blockIdx.x) * 4);
}
template <typename T> void launch_norm2(const T* v, long long N, int nblk, double* partial, int nparts, cudaStream_t s) {
    { k_norm2<T><<<dim3(nparts, nblk), 256, 0, s>>>(v, N, partial, nparts); note_launch(); }
}
template void launch_norm2<float>(const float*, long long, int, double*, int, cudaStream_t);
template void launch_norm2<double>(const double*, long long, int, double*, int, cudaStream_t);

// power iteration on D^-1 Q in the D-norm: w = D^-1 q (in place), partial q.w
__global__ void k_power_scale(float* __restrict__ q, const float* __restrict__ dinv, long long N, double* __restrict__ partial, int nparts) {
    double dot[4] = {0, 0, 0, 0};
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const V4<float> a = v4load(q + n * RW);
        const float di = dinv[n];
        const V4<float> w = di * a;
        v4store(q + n * RW, w);
        dot[0] += (double)a.a * w.a; dot[1] += (double)a.b * w.b; dot[2] += (double)a.c * w.c; dot[3] += (double)a.d * w.d;
    }
    block_sum4<256>(dot, partial + (size_t)blockIdx.x * 4);
}
void launch_power_scale(float* q, const float* dinv, long long N, double* partial, int nparts, cudaStream_t s) {
    { k_power_scale<<<nparts, 256, 0, s>>>(q, dinv, N, partial, nparts); note_launch(); }
}

__global__ void k_scale_comp(float* __restrict__ v, const float* __restrict__ w, const double* __restrict__ nrm2, long long N) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    const V4<float> a = v4load(w + n * RW);
    const float s0 = nrm2[0] > 0 ? (float)(1.0 / sqrt(nrm2[0])) : 0.f, s1 = nrm2[1] > 0 ? (float)(1.0 / sqrt(nrm2[1])) : 0.f;
    const float s2 = nrm2[2] > 0 ? (float)(1.0 / sqrt(nrm2[2])) : 0.f, s3 = nrm2[3] > 0 ? (float)(1.0 / sqrt(nrm2[3])) : 0.f;
    v4store(v + n * RW, V4<float>{a.a * s0, a.b * s1, a.c * s2, a.d * s3});
}
void launch_scale_comp(float* v, const float* w, const double* nrm2, long long N, cudaStream_t s) {
    { k_scale_comp<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(v, w, nrm2, N); note_launch(); }
}

__global__ void k_fill_random(float* __restrict__ v, long long N, uint64_t seed) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    float r[4];
    for (int c = 0; c < 4; ++c) r[c] = (float)philox_normal(seed, 7u, (uint32_t)c, (uint64_t)n);
    v4store(v + n * RW, V4<float>{r[0], r[1], r[2], r[3]});
}
void launch_fill_random(float* v, long long N, uint64_t seed, cudaStream_t s) {
    { k_fill_random<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(v, N, seed); note_launch(); }
}

}  // namespace gmrf
