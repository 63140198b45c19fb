// Vector, transfer, reduction, sampling and variance kernels of the GB300
// GMRF solver (the posterior-precision stencils are in stencil.cu and
// stencil_march.cu).  All of them are HBM-bound elementwise or gather
// passes over blocked right-hand-side batches [nblk][N][4].
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <stdexcept>
#include <string>

#include <cuda.h>

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

static void cuda_ok(cudaError_t e) {
    if (e != cudaSuccess) throw std::runtime_error(std::string("kernel setup: ") + cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// Standard normals: the Box-Muller transform of two 53-bit uniforms of one
// Philox draw (normal 2j: cosine branch, 2j + 1: sine branch of counter
// (j, sample, stream, 0)).  The FP64 pipe of GB300 is narrow, so the
// logarithm and the sine / cosine are table-driven with short polynomials:
//   ln u, Tang's table-driven method (ACM TOMS 16(4), 1990): u = 2^e m with m
//     in [1, 2); F = 1 + j/128 keeps the leading 7 fraction bits of m and
//     f = m - F is exact; ln u = e ln 2 + ln F + ln(1 + q) with q = f / F in
//     [0, 2^-7), by the series of ln(1 + q) through q^7 (remainder below
//     2^-59).  Within 2^-7 of 1 the series runs on the exact t = u - 1, so
//     that ln u keeps its relative accuracy as u -> 1.
//   sin and cos of 2 pi u: j = nearest integer to 256 u, g = u - j/256 exact
//     (|g| <= 1/512), phi = 2 pi g; the addition theorem combines the table
//     values sin, cos(2 pi j / 256) with the Taylor series of sin phi through
//     phi^7 and of cos phi through phi^8 (remainders below 1e-19).
struct BoxMullerTables {
    double inv_f[128];   // 1 / (1 + j/128)
    double ln_f[128];    // ln(1 + j/128)
    double sn[256];      // sin(pi j / 128)
    double cs[256];      // cos(pi j / 128)
};
__device__ BoxMullerTables g_bm;
constexpr double kLn2 = 0.693147180559945309417232121458;
constexpr double kTwoPi = 6.283185307179586476925286766559;

__global__ void k_bm_tables() {
    const int j = threadIdx.x;
    if (j < 128) {
        g_bm.inv_f[j] = 1.0 / (1.0 + j / 128.0);
        g_bm.ln_f[j] = log1p(j / 128.0);
    }
    g_bm.sn[j] = sinpi(j / 128.0);
    g_bm.cs[j] = cospi(j / 128.0);
}

// Fills the tables once per process (the library drives one GPU per process).
static void bm_tables_ready() {
    static std::once_flag once;
    std::call_once(once, [] {
        k_bm_tables<<<1, 256>>>();
        note_launch();
        cuda_ok(cudaGetLastError());
        cuda_ok(cudaDeviceSynchronize());
    });
}

__device__ __forceinline__ double bm_log(double u) {          // u in (0, 1]
    const int hi = __double2hiint(u), lo = __double2loint(u);
    const int e = ((hi >> 20) & 0x7ff) - 1023;
    const int j = (hi >> 13) & 0x7f;
    const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);
    const double F = __hiloint2double((hi & 0x000fe000) | 0x3ff00000, 0);
    const bool near1 = u >= 1.0 - 1.0 / 128.0;
    const double q = near1 ? u - 1.0 : (m - F) * __ldg(&g_bm.inv_f[j]);
    const double base = near1 ? 0.0 : fma((double)e, kLn2, __ldg(&g_bm.ln_f[j]));
    double s = 1.0 / 7.0;
    s = fma(s, q, -1.0 / 6.0);
    s = fma(s, q, 1.0 / 5.0);
    s = fma(s, q, -0.25);
    s = fma(s, q, 1.0 / 3.0);
    s = fma(s, q, -0.5);
    s = fma(s, q, 1.0);
    return fma(q, s, base);
}

__device__ __forceinline__ void bm_sincos2pi(double u, double& sn, double& cs) {
    const int j = __double2int_rn(u * 256.0);
    const double g = fma((double)j, -1.0 / 256.0, u);
    const double phi = g * kTwoPi;
    const double p2 = phi * phi;
    double ss = -1.0 / 5040.0;
    ss = fma(ss, p2, 1.0 / 120.0);
    ss = fma(ss, p2, -1.0 / 6.0);
    const double sp = fma(phi * p2, ss, phi);
    double cc = 1.0 / 40320.0;
    cc = fma(cc, p2, -1.0 / 720.0);
    cc = fma(cc, p2, 1.0 / 24.0);
    cc = fma(cc, p2, -0.5);
    const double cp = fma(cc, p2, 1.0);
    const int k = j & 255;
    const double S = __ldg(&g_bm.sn[k]), C = __ldg(&g_bm.cs[k]);
    sn = fma(S, cp, C * sp);
    cs = fma(C, cp, -(S * sp));
}

__device__ __forceinline__ void philox_normal_pair(uint64_t seed, uint32_t stream, uint32_t sample, uint64_t j,
                                                   double& z0, double& z1) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)j, sample, stream, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const double u1 = u53(w.x, w.y), u2 = u53(w.z, w.w);
    const double r = sqrt(-2.0 * bm_log(u1));
    double sn, cs;
    bm_sincos2pi(u2, sn, cs);
    z0 = r * cs;
    z1 = r * sn;
}

__device__ __forceinline__ double philox_normal(uint64_t seed, uint32_t stream, uint32_t sample, uint64_t idx) {
    double z0, z1;
    philox_normal_pair(seed, stream, sample, idx >> 1, z0, z1);
    return (idx & 1) ? z1 : z0;
}


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
    v.omap = d_omap;
    if constexpr (sizeof(T) == 4) { v.oent = d_oent32; v.ostride = ostride32; }
    else { v.oent = d_oent64; v.ostride = ostride64; }
    v.ocap = d_omap ? ocap : 0;
    v.obs_direct = 0;
    v.periodic = periodic;
    v.noise = noise;
    v.tk_c = (T)tk_c;
    v.tk_o = (T)tk_o;
    return v;
}

template LevelView<float> Level::view<float>() const;
template LevelView<double> Level::view<double>() const;


// ---------------------------------------------------------------------------
// reductions and PCG scalars

__global__ void k_reduce(const double* __restrict__ partial, int nparts, double* __restrict__ out) {
    const int blk = blockIdx.x;
    double v[4] = {0, 0, 0, 0};
    for (int i = threadIdx.x; i < nparts; i += 256) {
        const double* p = partial + ((size_t)blk * nparts + i) * 4;
        v[0] += p[0]; v[1] += p[1]; v[2] += p[2]; v[3] += p[3];
    }
    block_sum4<256, double>(v, out + (size_t)blk * 4);
}

void reduce_prepare() {
    cudaFuncAttributes fa;
    cuda_ok(cudaFuncGetAttributes(&fa, k_reduce));
}

void launch_reduce(const double* partial, int nparts, int nblk, double* out, cudaStream_t s) {
    { k_reduce<<<nblk, 256, 0, s>>>(partial, nparts, out); note_launch(); }
}

// kind 0: pq reduced -> alpha = active ? rz / pq : 0 (breakdown if pq <= 0)
// kind 1: rr reduced -> rr (reported only)
// kind 2: rz_new reduced -> beta = rz_new / rz, rz = rz_new; a right-hand side
//         stops once rz_new <= tol2 * rz_0 (preconditioned residual norm,
//         invariant under diagonal scaling of the system)
// kind 3: initial: rz reduced, rz_0 = rz, active = rz_0 > 0
// kind 4: rr reduced -> rr
__device__ __forceinline__ void pcg_scalar_update(int kind, int r, double v, double* __restrict__ sc, int P, double tol2) {
    double* rz = sc, *pq = sc + P, *alpha = sc + 2 * P, *beta = sc + 3 * P;
    double* rr = sc + 4 * P, *rr0 = sc + 5 * P, *active = sc + 6 * P, *brk = sc + 7 * P;
    if (kind == 0) {
        pq[r] = v;
        const bool ok = v > 0.0 && isfinite(v) && isfinite(rz[r]);
        if (active[r] != 0.0 && !ok) { brk[r] = 1.0; active[r] = 0.0; }
        alpha[r] = (active[r] != 0.0) ? rz[r] / v : 0.0;
    } else if (kind == 2) {
        beta[r] = (active[r] != 0.0 && rz[r] != 0.0) ? v / rz[r] : 0.0;
        rz[r] = v;
        if (!(v > tol2 * rr0[r])) { active[r] = 0.0; beta[r] = 0.0; }
    } else if (kind == 4) {
        rr[r] = v;
    } else {
        rz[r] = v;
        rr0[r] = v;
        active[r] = (v > 0.0) ? 1.0 : 0.0;
        brk[r] = 0.0;
        beta[r] = 0.0;
        alpha[r] = 0.0;
    }
}

__global__ void k_pcg_scalar(int kind, const double* __restrict__ red, double* __restrict__ sc, int P, double tol2) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= P) return;
    pcg_scalar_update(kind, r, red[r], sc, P, tol2);
}

// k_reduce and k_pcg_scalar in one launch: CTA blk sums the partials of its
// block, and its threads 0..3 update the scalars of the block's four
// right-hand sides (the update of a right-hand side reads only its own).
__global__ void k_reduce_scalar(int kind, const double* __restrict__ partial, int nparts, double* __restrict__ red,
                                double* __restrict__ sc, int P, double tol2) {
    const int blk = blockIdx.x;
    double v[4] = {0, 0, 0, 0};
    for (int i = threadIdx.x; i < nparts; i += 256) {
        const double* p = partial + ((size_t)blk * nparts + i) * 4;
        v[0] += p[0]; v[1] += p[1]; v[2] += p[2]; v[3] += p[3];
    }
    block_sum4<256, double>(v, red + (size_t)blk * 4);   // threads 0..3 wrote red[blk * 4 + tid]
    if (threadIdx.x < 4) {
        const int r = blk * 4 + threadIdx.x;
        pcg_scalar_update(kind, r, red[r], sc, P, tol2);
    }
}

void launch_reduce_scalar(int kind, const double* partial, int nparts, int nblk, double* red, double* sc, double tol2,
                          cudaStream_t s) {
    { k_reduce_scalar<<<nblk, 256, 0, s>>>(kind, partial, nparts, red, sc, nblk * 4, tol2); note_launch(); }
}

void launch_pcg_scalar(int kind, const double* red, double* sc, int nblk, double tol2, cudaStream_t s) {
    const int P = nblk * RW;
    { k_pcg_scalar<<<(P + 127) / 128, 128, 0, s>>>(kind, red, sc, P, tol2); note_launch(); }
}

int elem_parts(long long N) { return (int)((N + ECHUNK - 1) / ECHUNK); }

// r -= alpha q (the stopping test uses r^T z, so no |r|^2 here)
template <typename T>
__global__ void __launch_bounds__(256) k_update_r(T* __restrict__ r, const T* __restrict__ q, const double* __restrict__ sc,
                                                  long long N) {
    const int blk = blockIdx.y;
    const double* alpha = sc + 2 * (gridDim.y * RW) + blk * RW;
    const T a0 = (T)alpha[0], a1 = (T)alpha[1], a2 = (T)alpha[2], a3 = (T)alpha[3];
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<T> qv = v4load(q + off);
        V4<T> rv = v4load(r + off);
        rv.a = fma(-a0, qv.a, rv.a); rv.b = fma(-a1, qv.b, rv.b); rv.c = fma(-a2, qv.c, rv.c); rv.d = fma(-a3, qv.d, rv.d);
        v4store(r + off, rv);
    }
}

template <typename T>
void launch_pcg_update_r(T* r, const T* q, const double* sc, long long N, int nblk, cudaStream_t s) {
    { k_update_r<T><<<dim3(elem_parts(N), nblk), 256, 0, s>>>(r, q, sc, N); note_launch(); }
}
template void launch_pcg_update_r<float>(float*, const float*, const double*, long long, int, cudaStream_t);
template void launch_pcg_update_r<double>(double*, const double*, const double*, long long, int, cudaStream_t);

// x += alpha p with the iteration's p, then p = z + beta p: one pass over p
template <typename T>
__global__ void __launch_bounds__(256) k_update_xp(T* __restrict__ x, T* __restrict__ p, const T* __restrict__ z,
                                                   const double* __restrict__ sc, long long N) {
    const int blk = blockIdx.y;
    const double* alpha = sc + 2 * (gridDim.y * RW) + blk * RW;
    const double* beta = sc + 3 * (gridDim.y * RW) + blk * RW;
    const T a0 = (T)alpha[0], a1 = (T)alpha[1], a2 = (T)alpha[2], a3 = (T)alpha[3];
    const T b0 = (T)beta[0], b1 = (T)beta[1], b2 = (T)beta[2], b3 = (T)beta[3];
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<T> zv = v4load(z + off);
        V4<T> pv = v4load(p + off), xv = v4load(x + off);
        xv.a = fma(a0, pv.a, xv.a); xv.b = fma(a1, pv.b, xv.b); xv.c = fma(a2, pv.c, xv.c); xv.d = fma(a3, pv.d, xv.d);
        pv.a = fma(b0, pv.a, zv.a); pv.b = fma(b1, pv.b, zv.b); pv.c = fma(b2, pv.c, zv.c); pv.d = fma(b3, pv.d, zv.d);
        v4store(x + off, xv);
        v4store(p + off, pv);
    }
}

// x += alpha p: the iterate's last update after the fused iterations
template <typename T>
__global__ void __launch_bounds__(256) k_update_x(T* __restrict__ x, const T* __restrict__ p, const double* __restrict__ sc,
                                                  long long N) {
    const int blk = blockIdx.y;
    const double* alpha = sc + 2 * (gridDim.y * RW) + blk * RW;
    const T a0 = (T)alpha[0], a1 = (T)alpha[1], a2 = (T)alpha[2], a3 = (T)alpha[3];
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<T> pv = v4load(p + off);
        V4<T> xv = v4load(x + off);
        xv.a = fma(a0, pv.a, xv.a); xv.b = fma(a1, pv.b, xv.b); xv.c = fma(a2, pv.c, xv.c); xv.d = fma(a3, pv.d, xv.d);
        v4store(x + off, xv);
    }
}

template <typename T>
void launch_pcg_update_x(T* x, const T* p, const double* sc, long long N, int nblk, cudaStream_t s) {
    { k_update_x<T><<<dim3(elem_parts(N), nblk), 256, 0, s>>>(x, p, sc, N); note_launch(); }
}
template void launch_pcg_update_x<float>(float*, const float*, const double*, long long, int, cudaStream_t);
template void launch_pcg_update_x<double>(double*, const double*, const double*, long long, int, cudaStream_t);

template <typename T>
void launch_pcg_update_xp(T* x, T* p, const T* z, const double* sc, long long N, int nblk, cudaStream_t s) {
    { k_update_xp<T><<<dim3(elem_parts(N), nblk), 256, 0, s>>>(x, p, z, sc, N); note_launch(); }
}
template void launch_pcg_update_xp<float>(float*, float*, const float*, const double*, long long, int, cudaStream_t);
template void launch_pcg_update_xp<double>(double*, double*, const double*, const double*, long long, int, cudaStream_t);

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
    const unsigned n = blockIdx.x * 256u + threadIdx.x;      // levels hold fewer than 2^31 nodes
    if (n >= (unsigned long long)Nout) return;
    const int x = (int)(n % (unsigned)ox);
    const unsigned r = n / (unsigned)ox;
    const int y = (int)(r % (unsigned)oy), t = (int)(r / (unsigned)oy);
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
    if ((long long)nx * ny * nt >= (1LL << 31)) throw std::runtime_error("restriction: a level holds 2^31 or more nodes");
    { k_restrict_axis<T><<<dim3((unsigned)((Nout + 255) / 256), nblk), 256, 0, s>>>(in, out, nx, ny, nt, axis, ncoarse, rs, rc, pj, pw); note_launch(); }
}
template void launch_restrict_axis<float>(const float*, float*, int, int, int, int, int, const int32_t*, const int32_t*, const int32_t*, const float*, int, cudaStream_t);
template void launch_restrict_axis<double>(const double*, double*, int, int, int, int, int, const int32_t*, const int32_t*, const int32_t*, const double*, int, cudaStream_t);

// Weight of the coarse corner (dx, dy) of a cell for a fine node at cell
// offsets (wx, wy) in [0, 1]^2 under P1 interpolation on the triangulation
// with diagonals (i, j)-(i+1, j+1): the coarse finite-element function
// evaluated at the fine node.  On nested grids the coarse space is then a
// subspace of the fine one, so point data rediscretised on a coarse level
// equals its Galerkin projection.
template <typename T>
__device__ __forceinline__ T p1_weight(int dx, int dy, T wx, T wy) {
    if (dx == 0 && dy == 0) return T(1) - (wx > wy ? wx : wy);
    if (dx == 1 && dy == 0) return wx > wy ? wx - wy : T(0);
    if (dx == 0 && dy == 1) return wy > wx ? wy - wx : T(0);
    if (dx == 1 && dy == 1) return wx < wy ? wx : wy;
    return T(0);
}

// Restriction in the (x, y) plane when both space axes coarsen (transpose of
// the P1 interpolation when p1, else of the bilinear one):
// out[.., Jy, Jx] = sum P(x, y; Jx, Jy) in[.., y, x] over the fine ranges of
// Jx and Jy.  A CTA owns kRestrictTX x kRestrictTY coarse nodes of one time
// level and block: it stages the fine region under them (span W x H, all
// rows in flight at once) and the transfer tables of its columns and rows in
// shared memory.  Each thread then sums its node: it keeps the (offset,
// weight) data of its up to kRestrictMax fine columns in registers and walks
// its fine rows, without branches (a zero weight adds zero).

template <typename T>
__global__ void __launch_bounds__(256) k_restrict_xy(const T* __restrict__ in, T* __restrict__ out, int nx, int ny, int nt,
                                                     int cx, int cy, const int32_t* __restrict__ rsx,
                                                     const int32_t* __restrict__ rcx, const int32_t* __restrict__ pjx,
                                                     const T* __restrict__ pwx, const int32_t* __restrict__ rsy,
                                                     const int32_t* __restrict__ rcy, const int32_t* __restrict__ pjy,
                                                     const T* __restrict__ pwy, bool p1, int W, int H, int tiles_cy) {
    extern __shared__ __align__(16) unsigned char rsm[];
    V4<T>* tile = reinterpret_cast<V4<T>*>(rsm);
    T* twx = reinterpret_cast<T*>(rsm + (size_t)W * H * sizeof(V4<T>));   // weights first: aligned for T
    T* twy = twx + W;
    int* tjx = reinterpret_cast<int*>(twy + H);
    int* tjy = tjx + W;
    const int blk = blockIdx.z;
    const int t = blockIdx.y / tiles_cy;
    const int Jx0 = blockIdx.x * kRestrictTX, Jy0 = (blockIdx.y - t * tiles_cy) * kRestrictTY;
    const int Jx1 = min(Jx0 + kRestrictTX, cx), Jy1 = min(Jy0 + kRestrictTY, cy);
    const int fx0 = rsx[Jx0], fx1 = rsx[Jx1 - 1] + rcx[Jx1 - 1];
    const int fy0 = rsy[Jy0], fy1 = rsy[Jy1 - 1] + rcy[Jy1 - 1];
    const long long Nin = (long long)nx * ny * nt;
    const T* src = in + ((size_t)blk * Nin + (size_t)t * nx * ny) * RW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int y = fy0 + warp; y < fy1; y += 8)
        for (int x = fx0 + lane; x < fx1; x += 32)
            cp_v4<T>(&tile[(y - fy0) * W + (x - fx0)], src + ((size_t)y * nx + x) * RW, true);
    cp_commit();
    for (int i = threadIdx.x; i < fx1 - fx0; i += 256) { tjx[i] = pjx[fx0 + i]; twx[i] = pwx[fx0 + i]; }
    for (int i = threadIdx.x; i < fy1 - fy0; i += 256) { tjy[i] = pjy[fy0 + i]; twy[i] = pwy[fy0 + i]; }
    cp_wait<0>();
    __syncthreads();
    const int Jx = Jx0 + (threadIdx.x % kRestrictTX), Jy = Jy0 + (threadIdx.x / kRestrictTX);
    if (Jx >= Jx1 || Jy >= Jy1) return;
    const int x0 = rsx[Jx] - fx0, kx = rcx[Jx], y0 = rsy[Jy] - fy0, ky = rcy[Jy];
    // per fine column: offset dx = Jx - pj and weight w (bilinear: the x factor)
    int dxs[kRestrictMax];
    T wxs[kRestrictMax];
#pragma unroll
    for (int a = 0; a < kRestrictMax; ++a) {
        const bool on = a < kx;
        const int xx = on ? x0 + a : x0;
        const int dx = Jx - tjx[xx];
        const T wx = twx[xx];
        dxs[a] = dx;
        wxs[a] = p1 ? wx : (dx == 0 ? T(1) - wx : (dx == 1 ? wx : T(0)));
    }
    V4<T> acc = v4zero<T>();
    for (int b = 0; b < ky; ++b) {
        const int yy = y0 + b;
        const int dy = Jy - tjy[yy];
        const T wy = twy[yy];
        const V4<T>* row = tile + (size_t)yy * W + x0;
        if (p1) {
#pragma unroll
            for (int a = 0; a < kRestrictMax; ++a) {
                if (a >= kx) break;
                acc = fma4(p1_weight<T>(dxs[a], dy, wxs[a], wy), row[a], acc);
            }
        } else {
            const T ay = dy == 0 ? T(1) - wy : (dy == 1 ? wy : T(0));
            V4<T> r = v4zero<T>();
#pragma unroll
            for (int a = 0; a < kRestrictMax; ++a) {
                if (a >= kx) break;
                r = fma4(wxs[a], row[a], r);
            }
            acc = fma4(ay, r, acc);
        }
    }
    const long long Nout = (long long)cx * cy * nt;
    v4store(out + ((size_t)blk * Nout + ((size_t)t * cy + Jy) * cx + Jx) * RW, acc);
}

template <typename T>
void launch_restrict_xy(const T* in, T* out, int nx, int ny, int nt, int cx, int cy, const int32_t* const rs[2],
                        const int32_t* const rc[2], const int32_t* const pj[2], const T* const pw[2], bool p1,
                        const int span[2], int nblk, cudaStream_t s) {
    static_assert(kRestrictTX * kRestrictTY == 256, "one thread per coarse node of the tile");
    const int tiles_cx = (cx + kRestrictTX - 1) / kRestrictTX, tiles_cy = (cy + kRestrictTY - 1) / kRestrictTY;
    const size_t smem = (size_t)span[0] * span[1] * sizeof(V4<T>) + (size_t)(span[0] + span[1]) * (sizeof(int) + sizeof(T));
    static std::once_flag once;
    std::call_once(once, [] {
        cuda_ok(cudaFuncSetAttribute(k_restrict_xy<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    });
    if (smem > 200 * 1024) throw std::runtime_error("restriction tile exceeds shared memory");
    const dim3 grid((unsigned)tiles_cx, (unsigned)(tiles_cy * nt), (unsigned)nblk);
    { k_restrict_xy<T><<<grid, 256, smem, s>>>(in, out, nx, ny, nt, cx, cy, rs[0], rc[0], pj[0], pw[0], rs[1], rc[1], pj[1], pw[1], p1, span[0], span[1], tiles_cy); note_launch(); }
}
template void launch_restrict_xy<float>(const float*, float*, int, int, int, int, int, const int32_t* const[2], const int32_t* const[2], const int32_t* const[2], const float* const[2], bool, const int[2], int, cudaStream_t);
template void launch_restrict_xy<double>(const double*, double*, int, int, int, int, int, const int32_t* const[2], const int32_t* const[2], const int32_t* const[2], const double* const[2], bool, const int[2], int, cudaStream_t);

struct AxisMap { const int32_t* j; const void* w; bool on; };

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(T* __restrict__ xf, const T* __restrict__ xc, int nx, int ny, int nt,
                                                     int cx, int cy, int ct, AxisMap ax, AxisMap ay, AxisMap at, bool p1,
                                                     bool per) {
    const long long Nf = (long long)nx * ny * nt, Nc = (long long)cx * cy * ct;
    const int blk = blockIdx.y;
    const unsigned n = blockIdx.x * 256u + threadIdx.x;      // levels hold fewer than 2^31 nodes
    if (n >= (unsigned long long)Nf) return;
    const int x = (int)(n % (unsigned)nx);
    const unsigned r = n / (unsigned)nx;
    const int y = (int)(r % (unsigned)ny), t = (int)(r / (unsigned)ny);
    int jx = x, jy = y, jt = t;
    T wx = T(0), wy = T(0), wt = T(0);
    if (ax.on) { jx = ax.j[x]; wx = ((const T*)ax.w)[x]; }
    if (ay.on) { jy = ay.j[y]; wy = ((const T*)ay.w)[y]; }
    if (at.on) { jt = at.j[t]; wt = ((const T*)at.w)[t]; }
    const T* xb = xc + (size_t)blk * Nc * RW;
    V4<T> acc = v4zero<T>();
    // space: P1 on the triangulation (p1) or bilinear; both reduce to linear
    // along a single coarsened axis, where the other offset is 0.  Time: linear.
    for (int dt = 0; dt < (at.on ? 2 : 1); ++dt) {
        const T ft = at.on ? (dt ? wt : T(1) - wt) : T(1);
        for (int dy = 0; dy < (ay.on ? 2 : 1); ++dy) {
            for (int dx = 0; dx < (ax.on ? 2 : 1); ++dx) {
                const T fs = p1 ? p1_weight<T>(dx, dy, wx, wy) : (dx ? wx : T(1) - wx) * (dy ? wy : T(1) - wy);
                const T f = ft * fs;
                if (f == T(0)) continue;
                int ux = jx + dx, uy = jy + dy;
                if (per) {      // coarse torus: node cx is node 0
                    if (ux == cx) ux = 0;
                    if (uy == cy) uy = 0;
                }
                const long long c = ((long long)(jt + dt) * cy + uy) * cx + ux;
                acc = fma4(f, v4load(xb + c * RW), acc);
            }
        }
    }
    const size_t off = ((size_t)blk * Nf + n) * RW;
    v4store(xf + off, v4load(xf + off) + acc);
}

template <typename T>
void launch_prolong_add(T* xf, const T* xc, const Level& f, const Level& c, bool p1, int nblk, cudaStream_t s) {
    const bool dbl = sizeof(T) == 8;
    AxisMap ax{f.d_pj[0], dbl ? (const void*)f.d_pwd[0] : (const void*)f.d_pw[0], f.coarsen[0]};
    AxisMap ay{f.d_pj[1], dbl ? (const void*)f.d_pwd[1] : (const void*)f.d_pw[1], f.coarsen[1]};
    AxisMap at{f.d_pj[2], dbl ? (const void*)f.d_pwd[2] : (const void*)f.d_pw[2], f.coarsen[2]};
    if (f.N >= (1LL << 31)) throw std::runtime_error("prolongation: a level holds 2^31 or more nodes");
    { k_prolong_add<T><<<dim3((unsigned)((f.N + 255) / 256), nblk), 256, 0, s>>>(xf, xc, f.nx, f.ny, f.nt, c.nx, c.ny, c.nt, ax, ay, at, p1, f.periodic != 0); note_launch(); }
}

// Restriction between periodic levels (torus n -> n / 2 in x and y), the
// transpose of the interpolation of k_prolong_add: coarse node (X, Y) sums
// P(i, j; X, Y) in[j][i] over the fine nodes 2X - 1 .. 2X + 1 and
// 2Y - 1 .. 2Y + 1 (mod n), where fine i lies between coarse i / 2 and
// (i / 2 + 1) mod m with weight (i mod 2) / 2 of the second.
template <typename T>
__global__ void __launch_bounds__(256) k_restrict_torus(const T* __restrict__ in, T* __restrict__ out, int nx, int ny,
                                                        int cx, int cy, bool p1) {
    const long long Nf = (long long)nx * ny, Nc = (long long)cx * cy;
    const int blk = blockIdx.y;
    const unsigned n = blockIdx.x * 256u + threadIdx.x;
    if (n >= (unsigned long long)Nc) return;
    const int X = (int)(n % (unsigned)cx), Y = (int)(n / (unsigned)cx);
    const T* ib = in + (size_t)blk * Nf * RW;
    V4<T> acc = v4zero<T>();
    for (int b = -1; b <= 1; ++b) {
        const int iy = wrap_idx(2 * Y + b, ny);
        const int jy = iy / 2;
        const T wy = (iy & 1) ? T(0.5) : T(0);
        for (int a = -1; a <= 1; ++a) {
            const int ix = wrap_idx(2 * X + a, nx);
            const int jx = ix / 2;
            const T wx = (ix & 1) ? T(0.5) : T(0);
            T w = T(0);
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int ux = jx + dx == cx ? 0 : jx + dx, uy = jy + dy == cy ? 0 : jy + dy;
                    if (ux != X || uy != Y) continue;
                    w += p1 ? p1_weight<T>(dx, dy, wx, wy) : (dx ? wx : T(1) - wx) * (dy ? wy : T(1) - wy);
                }
            if (w != T(0)) acc = fma4(w, v4load(ib + ((size_t)iy * nx + ix) * RW), acc);
        }
    }
    v4store(out + ((size_t)blk * Nc + n) * RW, acc);
}

template <typename T>
void launch_restrict_torus(const T* in, T* out, const Level& f, const Level& c, bool p1, int nblk, cudaStream_t s) {
    if (!f.periodic || c.nx * 2 != f.nx || c.ny * 2 != f.ny || f.nt != 1)
        throw std::runtime_error("torus restriction: levels are not a periodic 2:1 pair");
    { k_restrict_torus<T><<<dim3((unsigned)((c.N + 255) / 256), nblk), 256, 0, s>>>(in, out, f.nx, f.ny, c.nx, c.ny, p1); note_launch(); }
}
template void launch_restrict_torus<float>(const float*, float*, const Level&, const Level&, bool, int, cudaStream_t);
template void launch_restrict_torus<double>(const double*, double*, const Level&, const Level&, bool, int, cudaStream_t);
template void launch_prolong_add<float>(float*, const float*, const Level&, const Level&, bool, int, cudaStream_t);
template void launch_prolong_add<double>(double*, const double*, const Level&, const Level&, bool, int, cudaStream_t);

// coarsest level: x = Q_c^-1 b with the stored dense inverse.  The inverse is
// stored exactly symmetric, so lane i walks column i (A[j][i] = A[i][j]) and
// a warp's loads of one j are contiguous.  A CTA owns 32 rows of one block;
// its eight warps split the columns and add their partial sums in a fixed
// order through shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_dense_solve(const T* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ x, int n) {
    extern __shared__ unsigned char dsm[];
    V4<T>* sb = reinterpret_cast<V4<T>*>(dsm);          // b of the block [n]
    V4<T>* part = sb + n;                                // warp partial sums [8][32]
    const int blk = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    for (int k = threadIdx.x; k < n; k += 256) sb[k] = v4load(b + ((size_t)blk * n + k) * RW);
    __syncthreads();
    const int per = (n + 7) / 8;
    const int j0 = min(n, warp * per), j1 = min(n, j0 + per);
    V4<T> acc = v4zero<T>();
    if (i < n) {
        int j = j0;
        for (; j + 8 <= j1; j += 8) {        // eight independent loads in flight
            T a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = Ainv[(size_t)(j + u) * n + i];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc = fma4(a[u], sb[j + u], acc);
        }
        for (; j < j1; ++j) acc = fma4(Ainv[(size_t)j * n + i], sb[j], acc);
    }
    part[warp * 32 + lane] = acc;
    __syncthreads();
    if (warp == 0 && i < n) {
        V4<T> sum = part[lane];
#pragma unroll
        for (int w = 1; w < 8; ++w) sum = sum + part[w * 32 + lane];
        v4store(x + ((size_t)blk * n + i) * RW, sum);
    }
}

template <typename T> void launch_dense_solve(const T* Ainv, const T* b, T* x, int n, int nblk, cudaStream_t s) {
    const size_t smem = ((size_t)n + 256) * sizeof(V4<T>);
    static std::once_flag once;
    std::call_once(once, [] {
        cuda_ok(cudaFuncSetAttribute(k_dense_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    });
    if (smem > 200 * 1024) throw std::runtime_error("coarsest level too large for the dense solve");
    { k_dense_solve<T><<<dim3((unsigned)((n + 31) / 32), (unsigned)nblk), 256, smem, s>>>(Ainv, b, x, n); note_launch(); }
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

// x64 += norm * d per right-hand side; partial sums of |norm d|^2 (partial)
// and |x_new|^2 (partial + nblk * nparts * 4) for the forward-error test.
template <typename T>
__global__ void __launch_bounds__(256) k_axpy_norm(double* __restrict__ x64, const double* __restrict__ norms,
                                                   const T* __restrict__ d, long long N, double* __restrict__ partial) {
    // x += norm * d in FP64 (one rounding).  For the forward-error stopping
    // test: |d|^2 of the inner solution d (the increment is norm * d; the
    // host applies the norm) and |x|^2, both in FP64: d and x may lie far
    // outside the FP32 range of squares (linearised Burgers systems do).
    const int blk = blockIdx.y;
    const double* nm = norms + blk * RW;
    double dd[4] = {0, 0, 0, 0}, xx[4] = {0, 0, 0, 0};
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<T> dv = v4load(d + off);
        const double d0 = dv.a, d1 = dv.b, d2 = dv.c, d3 = dv.d;
        V4<double> xv = v4load(x64 + off);
        xv.a = fma(nm[0], d0, xv.a); xv.b = fma(nm[1], d1, xv.b); xv.c = fma(nm[2], d2, xv.c); xv.d = fma(nm[3], d3, xv.d);
        v4store(x64 + off, xv);
        dd[0] = fma(d0, d0, dd[0]); dd[1] = fma(d1, d1, dd[1]); dd[2] = fma(d2, d2, dd[2]); dd[3] = fma(d3, d3, dd[3]);
        xx[0] += xv.a * xv.a; xx[1] += xv.b * xv.b; xx[2] += xv.c * xv.c; xx[3] += xv.d * xv.d;
    }
    const size_t np = gridDim.x;
    block_sum4<256, double>(dd, partial + ((size_t)blk * np + blockIdx.x) * 4);
    block_sum4<256, double>(xx, partial + (size_t)gridDim.y * np * 4 + ((size_t)blk * np + blockIdx.x) * 4);
}
void launch_axpy_mixed(double* x64, const double* norms, const float* d32, long long N, int nblk, double* partial, cudaStream_t s) {
    { k_axpy_norm<float><<<dim3(elem_parts(N), nblk), 256, 0, s>>>(x64, norms, d32, N, partial); note_launch(); }
}
void launch_axpy_scaled64(double* x64, const double* norms, const double* d64, long long N, int nblk, double* partial, cudaStream_t s) {
    { k_axpy_norm<double><<<dim3(elem_parts(N), nblk), 256, 0, s>>>(x64, norms, d64, N, partial); note_launch(); }
}

// ---------------------------------------------------------------------------
// right-hand sides of perturbation samples: L z = B^T z1 + A^T Q_eps^1/2 z2
// (+ J^T Q_eps^1/2 z3), z drawn in-kernel (Sec. 3.2, left root of a sum).
// A slot with sample id -1 copies the data right-hand side, -2 is padding,
// >= 0 draws sample `id`.  With use_probe the slot holds a Rademacher probe.

// z1[blk][n][c]: the prior-row normals (stream 0) of the sample in slot
// (blk, c), and z2[blk][row][c] those of the observation rows (stream 1);
// zero for slots without a sample.  One thread per Box-Muller pair of rows
// (2j, 2j + 1), so each pair's transcendentals run once; threads past the
// N / 2 pairs of stream 0 take the pairs of stream 1.
__global__ void __launch_bounds__(256) k_sample_normals(uint64_t seed, const int32_t* __restrict__ slot_sample,
                                                        long long N, double* __restrict__ z1, long long rows,
                                                        double* __restrict__ z2) {
    const int blk = blockIdx.y;
    const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
    const long long p0 = (N + 1) / 2;
    const bool s1 = t >= p0;
    const long long j = s1 ? t - p0 : t;
    const long long M = s1 ? rows : N;
    const long long n0 = 2 * j;
    if (n0 >= M) return;
    double a[4], b[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int sid = slot_sample[blk * RW + c];
        a[c] = b[c] = 0.0;
        if (sid >= 0) philox_normal_pair(seed, s1 ? 1u : 0u, (uint32_t)sid, (uint64_t)j, a[c], b[c]);
    }
    double* p = (s1 ? z2 : z1) + ((size_t)blk * M + n0) * RW;
    v4store(p, V4<double>{a[0], a[1], a[2], a[3]});
    if (n0 + 1 < M) v4store(p + RW, V4<double>{b[0], b[1], b[2], b[3]});
}

constexpr int kObsChunk = 64;      // observation rows staged at a time by k_sample_rhs

template <int GEO>
__global__ void __launch_bounds__(256) k_sample_rhs(const LevelView<double> L, uint64_t seed,
                                                    const int32_t* __restrict__ slot_sample,
                                                    const double* __restrict__ bdata, const double* __restrict__ z1,
                                                    const double* __restrict__ z2, long long rows,
                                                    double* __restrict__ b64) {
    using G = Geo<GEO>;
    constexpr int TX = G::TX, TY = G::TY, TT = G::TT, HY = G::HY, HT = G::HT;
    constexpr int HYS = HY / 2;
    constexpr int SX = TX + 2, SY = TY + HY, ST = TT + HT;
    __shared__ V4<double> sz[ST][SY][SX];       // z1 on the rows touching the tile
    __shared__ int32_t s_onode[kObsChunk][8];   // a chunk of the tile's observation rows
    __shared__ double s_ow[kObsChunk][8];
    __shared__ int32_t s_orow[kObsChunk];
    // Matern transition noise: B^T z1 = B_w^T (T_K z1), z1 staged on rows two
    // past the tile first
    constexpr int SXN = GEO == GEO_XT ? SX + 2 : 1;
    __shared__ V4<double> zw[GEO == GEO_XT ? ST : 1][SXN];
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

    if (GEO == GEO_XT && L.noise) {
        for (int e = tid; e < SXN * ST; e += 256) {
            const int sx = e % SXN, st = e / SXN;
            const int rx = tx0 - 2 + sx, rt = tt0 + st;
            V4<double> z = v4zero<double>();
            if (z1 != nullptr && rx >= 0 && rx < nx && rt < nt) z = v4load(z1 + ((size_t)blk * N + (long long)rt * nx + rx) * RW);
            zw[GEO == GEO_XT ? st : 0][GEO == GEO_XT ? sx : 0] = z;
        }
        __syncthreads();
        const double tc = L.tk_c, to = L.tk_o;
        for (int e = tid; e < SX * ST; e += 256) {
            const int sx = e % SX, st = e / SX;
            const int rx = tx0 - 1 + sx, rt = tt0 + st;
            const V4<double>* row = &zw[GEO == GEO_XT ? st : 0][0];
            V4<double> v = row[sx + 1];
            if (rt >= 1 && rt < nt && rx >= 1 && rx <= nx - 2) {       // interior rows of levels >= 1
                V4<double> w = tc * v;
                if (rx - 1 >= 1) w = fma4(to, row[sx], w);
                if (rx + 1 <= nx - 2) w = fma4(to, row[sx + 2], w);
                v = w;
            }
            sz[st][0][sx] = v;
        }
    } else
    for (int e = tid; e < SX * SY * ST; e += 256) {
        const int sx = e % SX, sy = (e / SX) % SY, st = e / (SX * SY);
        int rx = tx0 - 1 + sx, ry = ty0 - HYS + sy;
        const int rt = tt0 + st;
        if (L.periodic) {           // rows across the seam of the torus
            if (rx <= nx) rx = wrap_idx(rx, nx);
            if (ry <= ny) ry = wrap_idx(ry, ny);
        }
        V4<double> z = v4zero<double>();
        if (z1 != nullptr && rx >= 0 && rx < nx && ry >= 0 && ry < ny && rt < nt) {
            const long long row = ((long long)rt * ny + ry) * nx + rx;
            z = v4load(z1 + ((size_t)blk * N + row) * RW);
        }
        sz[st][sy][sx] = z;
    }
    __syncthreads();

    const int lx = tid % TX, ly = (tid / TX) % TY, lt = tid / (TX * TY);
    const int gx = tx0 + lx, gy = ty0 + ly, gt = tt0 + lt;
    const bool own = gx < nx && gy < ny && gt < nt;
    V4<double> q = v4zero<double>();
    if (own) {
        const bool per = L.periodic != 0;
        if (!per && is_dirichlet(gx, gy, nx, ny)) {
            q = L.inv_eps * sz[lt][ly + HYS][lx + 1];
        } else {
#pragma unroll
            for (int o = 0; o < NTAP; ++o) {
                if (HY == 0 && tap_dy(o) != 0) continue;
                if (HT == 0 && tap_dt(o) != 0) continue;
                const int rx = gx - tap_dx(o), ry = gy - tap_dy(o), rt = gt - tap_dt(o);
                if (!per && (rx < 0 || rx >= nx || ry < 0 || ry >= ny)) continue;
                if (rt >= nt) continue;
                if (!per && is_dirichlet(rx, ry, nx, ny)) continue;     // Dirichlet rows touch only themselves
                const int cls = (nt > 1 && rt == 0) ? 1 : 0;
                const double c = L.cf[cls][o];
                if (c == 0.0) continue;
                q = fma4(c, sz[lt - tap_dt(o)][ly + HYS - tap_dy(o)][lx + 1 - tap_dx(o)], q);
            }
        }
        if (L.col.kind >= 3) {
            // FEM Crank-Nicolson rows: J^T Q_eps^1/2 z3 over the (up to six) rows
            // touching the node, draws as for the collocation rows below
            const double sq_eps = sqrt(L.col.qeps);
            auto mu_at = [&](int x, int t) -> double { return L.mu ? L.mu[(long long)t * nx + x] : 0.0; };
            int rxs[6], rts[6];
            double cfs[6];
            const int nr = fem_cn_column(L.col, nx, nt, gx, gt, mu_at, rxs, rts, cfs);
            for (int k = 0; k < nr; ++k) {
                const uint64_t orow = (uint64_t)L.col.row0 + (uint64_t)(rts[k] - 1) * (nx - 2) + (rxs[k] - 1);
                double v[4];
                const double* zr = z2 + ((size_t)blk * rows + orow) * RW;
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) v[cc] = (sid[cc] >= 0 && z2 != nullptr) ? zr[cc] : 0.0;
                q = fma4(cfs[k] * sq_eps, V4<double>{v[0], v[1], v[2], v[3]}, q);
            }
        } else if (L.col.kind != 0) {
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
                if (rx < 1 || rx > nx - 2 || rt < 1 || rt >= nt || !colloc_on(L.col, rx, rt)) continue;
                const double c = k == 0 ? coef(rx, rt, 0) : (k == 1 ? coef(rx, rt, 2) : (k == 2 ? coef(rx, rt, 1) : -L.col.inv_dt));
                const uint64_t orow = (uint64_t)L.col.row0 + (uint64_t)(rt - 1) * (nx - 2) + (rx - 1);
                double v[4];
#pragma unroll
                const double* zr = z2 + ((size_t)blk * rows + orow) * RW;
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) v[cc] = (sid[cc] >= 0 && z2 != nullptr) ? zr[cc] : 0.0;
                q = fma4(c * sq_eps, V4<double>{v[0], v[1], v[2], v[3]}, q);
            }
        }
    }
    if (L.obs != nullptr) {
        // A^T R^-1/2 z2 at the own node: the tile's observation rows are
        // staged in chunks (nodes, weights w sqrt(rinv), rows), then each
        // node adds its terms in list order (ascending row index) and node
        // order within a row, so the sum is the same on every run
        const int32_t me = own ? (int32_t)(((long long)gt * ny + gy) * nx + gx) : -1;
        const int k0 = L.tile_ptr[tile], k1 = L.tile_ptr[tile + 1];
        for (int c0 = k0; c0 < k1; c0 += kObsChunk) {        // the same trip count in every thread
            const int cn = min(kObsChunk, k1 - c0);
            __syncthreads();                                  // the previous chunk has been read
            for (int e = tid; e < cn * 8; e += 256) {
                const int j = e >> 3, n = e & 7;
                const ObsRow& o = L.obs[L.tile_idx[c0 + j]];
                s_onode[j][n] = n < o.nn ? o.node[n] : -1;
                s_ow[j][n] = n < o.nn ? o.wd[n] * sqrt(o.rinv) : 0.0;
                if (n == 0) s_orow[j] = o.row;
            }
            __syncthreads();
            if (own) {
                for (int j = 0; j < cn; ++j) {
#pragma unroll
                    for (int n = 0; n < 8; ++n) {
                        if (s_onode[j][n] != me) continue;
                        double v[4];
                        const double* zr = z2 + ((size_t)blk * rows + s_orow[j]) * RW;
#pragma unroll
                        for (int c = 0; c < 4; ++c) v[c] = (sid[c] >= 0 && z2 != nullptr) ? zr[c] : 0.0;
                        q = fma4(s_ow[j][n], V4<double>{v[0], v[1], v[2], v[3]}, q);
                    }
                }
            }
        }
    }
    if (own) {
        const long long node = ((long long)gt * ny + gy) * nx + gx;
        V4<double> out = q;
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
                       const double* bdata, double* b64, double* z1, double* z2, long long rows, int nblk,
                       cudaStream_t s) {
    if ((z1 == nullptr) != (z2 == nullptr)) throw std::runtime_error("sample right-hand sides: z1 and z2 go together");
    if (z1 != nullptr) {
        bm_tables_ready();
        const long long pairs = (L.N + 1) / 2 + (rows + 1) / 2;
        k_sample_normals<<<dim3((unsigned)((pairs + 255) / 256), (unsigned)nblk), 256, 0, s>>>(seed, slot_sample, L.N, z1,
                                                                                                rows, z2);
        note_launch();
    }
    const dim3 grid((unsigned)((long long)L.tiles_x * L.tiles_y * L.tiles_t), (unsigned)nblk);
    if (geo == GEO_XY) { k_sample_rhs<GEO_XY><<<grid, 256, 0, s>>>(L, seed, slot_sample, bdata, z1, z2, rows, b64); note_launch(); }
    else if (geo == GEO_XT) { k_sample_rhs<GEO_XT><<<grid, 256, 0, s>>>(L, seed, slot_sample, bdata, z1, z2, rows, b64); note_launch(); }
    else { k_sample_rhs<GEO_XYT><<<grid, 256, 0, s>>>(L, seed, slot_sample, bdata, z1, z2, rows, b64); note_launch(); }
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

// Observation sums at the nodes, gathered per tile: each node of the tile
// adds the terms of the tile's observation rows that touch it, in list order
// (ascending row index) and node order within a row, so the result is the
// same on every run (no atomics).  kind 0: the data right-hand side
// A^T R^-1 y over the point rows (row index < nrows_y); kind 1: the
// observation part sum_k rinv_k w_kn^2 of the diagonal over every row.
template <int GEO>
__global__ void __launch_bounds__(256) k_obs_gather(const LevelView<double> L, int kind, int nrows_y,
                                                    const double* __restrict__ y, double* __restrict__ out) {
    using G = Geo<GEO>;
    constexpr int TX = G::TX, TY = G::TY;
    const int nx = L.nx, ny = L.ny, nt = L.nt;
    const int tile = blockIdx.x, tid = threadIdx.x;
    const int tx0 = (tile % L.tiles_x) * TX;
    const int rest = tile / L.tiles_x;
    const int ty0 = (rest % L.tiles_y) * TY;
    const int tt0 = (rest / L.tiles_y) * G::TT;
    const int gx = tx0 + tid % TX, gy = ty0 + (tid / TX) % TY, gt = tt0 + tid / (TX * TY);
    if (gx >= nx || gy >= ny || gt >= nt) return;
    const int32_t me = (int32_t)(((long long)gt * ny + gy) * nx + gx);
    const int k0 = L.tile_ptr[tile], k1 = L.tile_ptr[tile + 1];
    double acc = out[me];
    bool hit = false;
    for (int k = k0; k < k1; ++k) {
        const ObsRow& o = L.obs[L.tile_idx[k]];
        if (kind == 0 && o.row >= nrows_y) continue;
        for (int n = 0; n < o.nn; ++n) {
            if (o.node[n] != me) continue;
            acc += kind == 0 ? o.wd[n] * (o.rinv * y[o.row]) : o.wd[n] * o.wd[n] * o.rinv;
            hit = true;
        }
    }
    if (hit) out[me] = acc;
}

static void launch_obs_gather(const Level& Lv, int kind, int nrows_y, const double* y, double* out, cudaStream_t s) {
    if (Lv.nobs <= 0) return;
    const LevelView<double> L = Lv.view<double>();
    const unsigned grid = (unsigned)((long long)L.tiles_x * L.tiles_y * L.tiles_t);
    if (Lv.geo == GEO_XY) k_obs_gather<GEO_XY><<<grid, 256, 0, s>>>(L, kind, nrows_y, y, out);
    else if (Lv.geo == GEO_XT) k_obs_gather<GEO_XT><<<grid, 256, 0, s>>>(L, kind, nrows_y, y, out);
    else k_obs_gather<GEO_XYT><<<grid, 256, 0, s>>>(L, kind, nrows_y, y, out);
    note_launch();
}

void launch_obs_data_rhs(const Level& L, int nrows_y, const double* y, double* b, cudaStream_t s) {
    if (nrows_y > 0) launch_obs_gather(L, 0, nrows_y, y, b, s);
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
template <typename QT>
__global__ void k_rbmc(const QT* __restrict__ Qx, const double* __restrict__ x, const double* __restrict__ diag,
                       const int32_t* __restrict__ slot_sample, long long N, int nblk, int ns, double* __restrict__ var,
                       double* __restrict__ se) {
    // e = ((Q x)_n - d x_n) / d = (Q x)_n / d - x_n per sample slot, in the
    // precision of Q x (an FP32 product carries no more digits than FP32
    // arithmetic keeps); the sums over the slots are widened at the end
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    const double d = diag[n];
    const QT invd = (QT)(1.0 / d);
    QT s1 = QT(0), s2 = QT(0);
    for (int blk = 0; blk < nblk; ++blk) {
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<QT> qx = v4load(Qx + off);
        const V4<double> xv = v4load(x + off);
        const QT a[4] = {qx.a, qx.b, qx.c, qx.d};
        const QT b[4] = {(QT)xv.a, (QT)xv.b, (QT)xv.c, (QT)xv.d};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (slot_sample[blk * RW + c] < 0) continue;
            const QT e = a[c] * invd - b[c];
            const QT e2 = e * e;
            s1 += e2;
            s2 += e2 * e2;
        }
    }
    const double m = (double)s1 / ns;
    var[n] = 1.0 / d + m;
    if (se != nullptr) {
        const double v = ns > 1 ? ((double)s2 - ns * m * m) / (ns - 1) : 0.0;
        se[n] = sqrt(fmax(v, 0.0) / ns);
    }
}
template <typename QT>
void launch_rbmc(const QT* Qx, const double* x, const double* diag, const int32_t* slot_sample, long long N,
                 int nblk, int ns, double* var, double* se, cudaStream_t s) {
    { k_rbmc<QT><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(Qx, x, diag, slot_sample, N, nblk, ns, var, se); note_launch(); }
}
template void launch_rbmc<float>(const float*, const double*, const double*, const int32_t*, long long, int, int, double*,
                                 double*, cudaStream_t);
template void launch_rbmc<double>(const double*, const double*, const double*, const int32_t*, long long, int, int,
                                  double*, double*, cudaStream_t);

// diagonal of B^T B + J^T Q_eps J at every node (observation part added by k_obs_gather)
template <typename T>
__global__ void k_diag(const LevelView<T> L, double* __restrict__ diag) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= L.N) return;
    const int nx = L.nx, ny = L.ny, nt = L.nt;
    const int x = (int)(n % nx);
    const long long r = n / nx;
    const int y = (int)(r % ny), t = (int)(r / ny);
    double d = 0.0;
    const bool per = L.periodic != 0;       // torus: every row is an interior row
    if (!per && is_dirichlet(x, y, nx, ny)) {
        d = (double)L.inv_eps2;
    } else if (L.noise) {
        // B = T_K B_w (1D space-time): column n of B_w has rows (x-1..x+1, t)
        // and (x, t+1); T_K mixes interior rows of levels >= 1 with their x
        // neighbours, so the column of B lives on rows x-2..x+2 of level t and
        // x-1..x+1 of level t+1
        auto bw = [&](int rx, int rt) -> double {      // B_w[(rx, rt), (x, t)]
            if (rx < 1 || rx > nx - 2 || rt < 0 || rt >= nt) return 0.0;
            const int cls = (nt > 1 && rt == 0) ? 1 : 0;
            for (int o = 0; o < NTAP; ++o)
                if (rx + tap_dx(o) == x && tap_dy(o) == 0 && rt + tap_dt(o) == t && x >= 1 && x <= nx - 2)
                    return (double)L.cf[cls][o];
            return 0.0;
        };
        for (int rt = t; rt <= t + 1 && rt < nt; ++rt)
            for (int rx = x - 2; rx <= x + 2; ++rx) {
                if (rx < 0 || rx >= nx) continue;
                double v = bw(rx, rt);
                if (rt >= 1 && rx >= 1 && rx <= nx - 2) {
                    v = L.tk_c * v;
                    if (rx - 1 >= 1) v += L.tk_o * bw(rx - 1, rt);
                    if (rx + 1 <= nx - 2) v += L.tk_o * bw(rx + 1, rt);
                }
                d += v * v;
            }
    } else {
        for (int o = 0; o < NTAP; ++o) {
            const int rx = x - tap_dx(o), ry = y - tap_dy(o), rt = t - tap_dt(o);
            if (rt < 0 || rt >= nt) continue;
            if (!per && (rx < 0 || rx >= nx || ry < 0 || ry >= ny)) continue;
            if (!per && is_dirichlet(rx, ry, nx, ny)) continue;
            const int cls = (nt > 1 && rt == 0) ? 1 : 0;
            const double c = (double)L.cf[cls][o];
            d += c * c;
        }
    }
    if (L.col.kind >= 3) {
        auto mu_at = [&](int xx, int tt) -> double { return L.mu ? (double)L.mu[(long long)tt * nx + xx] : 0.0; };
        int rxs[6], rts[6];
        double cfs[6];
        const int nr = fem_cn_column(L.col, nx, nt, x, t, mu_at, rxs, rts, cfs);
        double acc = 0.0;
        for (int k = 0; k < nr; ++k) acc += cfs[k] * cfs[k];
        d += L.col.qeps * acc;
    } else if (L.col.kind != 0) {
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
            if (rx < 1 || rx > nx - 2 || rt < 1 || rt >= nt || !colloc_on(L.col, rx, rt)) continue;
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

void launch_obs_diag(const Level& L, double* diag, cudaStream_t s) { launch_obs_gather(L, 1, 0, nullptr, diag, s); }

// max_n (total_n - prior_n) / total_n: the largest share of a node's diagonal
// contributed by the observation rows.  Non-negative doubles order like their
// bit patterns, so the block maxima combine with an integer atomicMax.
__global__ void k_max_share(const double* __restrict__ prior, const double* __restrict__ total, long long N,
                            unsigned long long* __restrict__ out) {
    __shared__ double red[256];
    double m = 0.0;
    for (long long n = (long long)blockIdx.x * 256 + threadIdx.x; n < N; n += (long long)gridDim.x * 256) {
        const double t = total[n];
        if (t > 0.0) m = fmax(m, fmax(0.0, (t - prior[n]) / t));
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(red[0]));
}
void launch_max_share(const double* prior, const double* total, long long N, unsigned long long* out, cudaStream_t s) {
    const long long want = (N + 255) / 256;
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(want, 4 * 152));
    { k_max_share<<<grid, 256, 0, s>>>(prior, total, N, out); note_launch(); }
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
    bm_tables_ready();
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
    block_sum4<256, double>(dot, partial + ((size_t)blk * nparts + blockIdx.x) * 4);
}
void launch_dot_blocked(const double* a, const double* b, long long N, int nblk, double* partial, int nparts, cudaStream_t s) {
    { k_dot_blocked<<<dim3(nparts, nblk), 256, 0, s>>>(a, b, N, partial, nparts); note_launch(); }
}

}  // namespace gmrf

namespace gmrf {

// ---------------------------------------------------------------------------
// small helpers of the solver driver

template <typename T>
__global__ void k_widen(const T* __restrict__ in, double* __restrict__ out, long long n) {
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}
template <typename T> void launch_widen(const T* in, double* out, long long n, cudaStream_t s) {
    { k_widen<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n); note_launch(); }
}
template void launch_widen<float>(const float*, double*, long long, cudaStream_t);
template void launch_widen<double>(const double*, double*, long long, cudaStream_t);

template <typename T>
__global__ void k_norm2(const T* __restrict__ v, long long N, double* __restrict__ partial, int nparts) {
    const int blk = blockIdx.y;
    T dot[4] = {T(0), T(0), T(0), T(0)};
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const V4<T> a = v4load(v + ((size_t)blk * N + n) * RW);
        dot[0] += a.a * a.a; dot[1] += a.b * a.b; dot[2] += a.c * a.c; dot[3] += a.d * a.d;
    }
    block_sum4<256, T>(dot, partial + ((size_t)blk * nparts + blockIdx.x) * 4);
}
// sum_n w[n] v_n^2 per right-hand side (the D^-1-weighted residual norm)
__global__ void k_norm2w(const double* __restrict__ v, const double* __restrict__ w, long long N, double* __restrict__ partial,
                         int nparts) {
    const int blk = blockIdx.y;
    double dot[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const V4<double> a = v4load(v + ((size_t)blk * N + n) * RW);
        const double wn = w[n];
        dot[0] += wn * a.a * a.a; dot[1] += wn * a.b * a.b; dot[2] += wn * a.c * a.c; dot[3] += wn * a.d * a.d;
    }
    block_sum4<256, double>(dot, partial + ((size_t)blk * nparts + blockIdx.x) * 4);
}
void launch_norm2w(const double* v, const double* w, long long N, int nblk, double* partial, int nparts, cudaStream_t s) {
    { k_norm2w<<<dim3(nparts, nblk), 256, 0, s>>>(v, w, N, partial, nparts); note_launch(); }
}

template <typename T> void launch_norm2(const T* v, long long N, int nblk, double* partial, int nparts, cudaStream_t s) {
    { k_norm2<T><<<dim3(nparts, nblk), 256, 0, s>>>(v, N, partial, nparts); note_launch(); }
}
template void launch_norm2<float>(const float*, long long, int, double*, int, cudaStream_t);
template void launch_norm2<double>(const double*, long long, int, double*, int, cudaStream_t);

template <typename T>
__global__ void k_dot(const T* __restrict__ a, const T* __restrict__ b, long long N, double* __restrict__ partial, int nparts) {
    const int blk = blockIdx.y;
    T dot[4] = {T(0), T(0), T(0), T(0)};
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4<T> av = v4load(a + off), bv = v4load(b + off);
        dot[0] += av.a * bv.a; dot[1] += av.b * bv.b; dot[2] += av.c * bv.c; dot[3] += av.d * bv.d;
    }
    block_sum4<256, T>(dot, partial + ((size_t)blk * nparts + blockIdx.x) * 4);
}
template <typename T> void launch_dot(const T* a, const T* b, long long N, int nblk, double* partial, int nparts, cudaStream_t s) {
    { k_dot<T><<<dim3(nparts, nblk), 256, 0, s>>>(a, b, N, partial, nparts); note_launch(); }
}
template void launch_dot<float>(const float*, const float*, long long, int, double*, int, cudaStream_t);
template void launch_dot<double>(const double*, const double*, long long, int, double*, int, cudaStream_t);

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
    block_sum4<256, double>(dot, partial + (size_t)blockIdx.x * 4);
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

// Standard normals, each node scaled by sqrt(dinv[n]) when dinv is given.
__global__ void k_fill_random(float* __restrict__ v, long long N, uint64_t seed, const float* __restrict__ dinv) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    const float sc = dinv ? sqrtf(dinv[n]) : 1.f;
    float r[4];
    for (int c = 0; c < 4; ++c) r[c] = sc * (float)philox_normal(seed, 7u, (uint32_t)c, (uint64_t)n);
    v4store(v + n * RW, V4<float>{r[0], r[1], r[2], r[3]});
}
void launch_fill_random(float* v, long long N, uint64_t seed, cudaStream_t s, const float* dinv) {
    bm_tables_ready();
    { k_fill_random<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(v, N, seed, dinv); note_launch(); }
}

}  // namespace gmrf
