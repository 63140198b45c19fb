// Fused posterior-precision stencil for 2D space and 1D space x time.
//
// The posterior precision Q_u|y = B^T B + J^T Q_eps J + A^T R^-1 A
// (Sec. 3.1 eq. posterior-mean; B the stacked root of the SPDE prior,
// Sec. 2.2 eq. sparse-prec-matrix and App. A; J the collocation rows,
// Sec. 3.3) is never stored.  A persistent CTA walks a contiguous chunk of
// work units (tile, block of four right-hand sides).  For each unit it
// receives the input tile with its halo and the own tiles of b and d as TMA
// boxes on an mbarrier (the next unit's boxes in flight), forms s = B p on
// the tile plus a one-node ring, applies B^T back onto the tile, adds the
// observation rows of the tile from per-tile tables, and finishes with a
// mode-specific epilogue (apply, residual, Chebyshev step).  The work is
// HBM-bound (about 3 flop per byte), so nothing here uses tensor cores.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <stdexcept>
#include <string>

#include <cuda.h>

#include "autotune.h"
#include "kernels.h"

namespace gmrf {

static void cuda_ok(cudaError_t e) {
    if (e != cudaSuccess) throw std::runtime_error(std::string("kernel setup: ") + cudaGetErrorString(e));
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
// Shared memory of one CTA: NS stages of the unit's input tile with halo
// (TMA destinations first, on 128-byte boundaries), the s tile and the
// per-node scalars.

// NOISE (1D space-time with Matern transition noise): B = T_K B_w with T_K a
// three-point operator per level, so the input halo is 4 in x, B_w p is formed
// on rows three past the tile (ring 3), T_K twice brings it back to ring 1.
template <int GEO, typename T, int MODE, int COL, int NS, int KB, int NOISE = 0> struct alignas(128) StencilSmem {
    using G = Geo<GEO>;
    static constexpr int TX = G::TX, TY = G::TY, TT = G::TT, HY = G::HY, HT = G::HT;
    static constexpr int HX = NOISE ? 4 : 2, SR = NOISE ? 3 : 1;
    static constexpr int PX = TX + 2 * HX, PY = TY + 2 * HY, PT = TT + 2 * HT;
    static constexpr int SX = TX + 2, SY = TY + HY, ST = TT + HT;
    static constexpr int SXW = TX + 2 * SR, SX2 = TX + 4;
    static constexpr int TN = TX * TY * TT, PN = PX * PY * PT, SN = SX * SY * ST;
    static constexpr int SNW = SXW * SY * ST, SN2 = SX2 * SY * ST;
    static constexpr int NB = MODE == M_APPLY ? 1 : NS;
    static constexpr int ND = MODE == M_CHEB ? NS : 1;
    static constexpr int NH = MODE == M_CHEB0 ? NS : 1, PH = MODE == M_CHEB0 ? PN : 1;
    static constexpr int NZ = MODE == M_PCG ? NS : 1, PZ = MODE == M_PCG ? PN : 1;
    // TMA destinations (p, b, d) first: every stage buffer starts on a
    // 128-byte boundary
    V4<T> p[NS][PN][KB];
    V4<T> b[NB][TN][KB];
    V4<T> d[ND][TN][KB];
    V4<T> z[NZ][PZ][KB];       // PCG: the preconditioned residual with halo
    T dinv[ND][TN];
    V4<T> s[SN][KB];
    V4<T> sw[NOISE ? SNW : 1][KB];     // NOISE: B_w p on ring 3
    V4<T> s2[NOISE ? SN2 : 1][KB];     // NOISE: T_K B_w p on ring 2
    V4<T> sj[COL ? SN : 1][KB];
    V4<T> qobs[TN][KB];        // A^T R^-1 A p at the tile's observed nodes
    T dinvh[NH][PH];           // CHEB0: D^-1 on the staged nodes
    T mu[(COL == 2 || COL == 4) ? NS : 1][(COL == 2 || COL == 4) ? PN : 1];
    static_assert((PN * sizeof(V4<T>)) % 128 == 0 && (TN * sizeof(V4<T>)) % 128 == 0,
                  "stage buffers of the TMA boxes keep 128-byte alignment");
};

// Tensor maps of one launch: the input tile with its halo, and the own tiles
// of the right-hand side and the direction (unused maps stay zero).
struct StencilMaps {
    CUtensorMap p, b, d;
};

// Flat shared-memory offsets of the taps: in the staged input (row r reads
// p at r + o) and in the s tile (node i gathers s at row i - o).
template <int PX, int PY> __host__ __device__ constexpr int poff(int o) { return (tap_dt(o) * PY + tap_dy(o)) * PX + tap_dx(o); }
template <int SX, int SY> __host__ __device__ constexpr int soff(int o) { return -((tap_dt(o) * SY + tap_dy(o)) * SX + tap_dx(o)); }

// Position of a work unit: tile coordinates (tx, ty, tt) in tile units and
// the block group.  Units are numbered group-major (u = grp * ntiles + tile);
// each CTA takes one contiguous chunk of units, so it crosses few group
// boundaries (where the dot partials are flushed), and steps through its
// chunk with carry-adds (no integer division inside the unit loop).
struct UnitPos {
    int tx, ty, tt, grp;
};
__device__ __forceinline__ UnitPos unit_decompose(long long u, int tiles_x, int tiles_y, int tiles_t) {
    UnitPos p;
    const long long ntiles = (long long)tiles_x * tiles_y * tiles_t;
    p.grp = (int)(u / ntiles);
    const long long tile = u - (long long)p.grp * ntiles;
    p.tx = (int)(tile % tiles_x);
    const long long r = tile / tiles_x;
    p.ty = (int)(r % tiles_y);
    p.tt = (int)(r / tiles_y);
    return p;
}
__device__ __forceinline__ void unit_next(UnitPos& p, int tiles_x, int tiles_y, int tiles_t) {
    if (++p.tx == tiles_x) {
        p.tx = 0;
        if (++p.ty == tiles_y) {
            p.ty = 0;
            if (++p.tt == tiles_t) { p.tt = 0; ++p.grp; }
        }
    }
}

// One work unit is (tile, group of KB consecutive blocks of four right-hand
// sides): all per-node index work, staging addresses and checks are shared
// by the 4 KB right-hand sides of the group.
// Set when a stencil CTA gave up waiting for a staged tile (bounded mbarrier
// wait); the solver checks and clears it after every solve.
__device__ int g_stencil_abort = 0;
constexpr int kMbarSpinCap = 1 << 22;
// polls before a staged-tile wait gives up (0: kMbarSpinCap; negative: give
// up without polling); a test hook
__device__ int g_stencil_wait_cap = 0;

template <int GEO, typename T, int MODE, int COL, int NS, int KB, int PER, int NOISE>
__global__ void __launch_bounds__(256) k_stencil(const StencilArgs<T> A, int nunits, const __grid_constant__ StencilMaps maps) {
    using SM = StencilSmem<GEO, T, MODE, COL, NS, KB, NOISE>;
    constexpr int TX = SM::TX, TY = SM::TY, TT = SM::TT, HY = SM::HY, HT = SM::HT;
    constexpr int PX = SM::PX, PY = SM::PY, PN = SM::PN, TN = SM::TN;
    constexpr int SX = SM::SX, SY = SM::SY, SN = SM::SN;
    constexpr int HX = SM::HX, SR = SM::SR, SXW = SM::SXW, SNW = SM::SNW, SX2 = SM::SX2, SN2 = SM::SN2;
    constexpr int HYS = HY / 2;
    constexpr int OC = ObsStencil<GEO>::OC;
    constexpr int KP = (PN + 255) / 256, KS = (SNW + 255) / 256;
    static_assert(!NOISE || (GEO == GEO_XT && HY == 0 && SY == 1), "Matern transition noise: 1D space-time tiles");
    static_assert(SN >= TN, "s tile covers the node tile");
    static_assert(NS >= 2, "the copy pipeline needs two stages");
    static_assert(KB == 1, "the input tile is one TMA box of one block");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem_base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);   // TMA destinations: 128 B
    SM& S = *reinterpret_cast<SM*>(smem_base);
    __shared__ uint64_t bars[NS];
    __shared__ int abort_unit;
    const int cap = g_stencil_wait_cap > 0 ? g_stencil_wait_cap : (g_stencil_wait_cap < 0 ? 0 : kMbarSpinCap);

    const LevelView<T>& L = A.L;
    const int nx = L.nx, ny = L.ny, nt = L.nt;
    const int N = (int)L.N;
    // a periodic level has no Dirichlet rows (App. B, N_k = 1) and its rows
    // extend one node past each end of the torus (rows of the wrapped halo)
    constexpr bool per = PER != 0;
    const int rlx = per ? -1 : 0, rhx = per ? nx + 1 : nx, rly = per ? -1 : 0, rhy = per ? ny + 1 : ny;
    auto dirich = [&](int x, int y) { return !per && is_dirichlet(x, y, nx, ny); };
    const int nblk = A.nblk;
    const int ntiles = L.tiles_x * L.tiles_y * L.tiles_t;
    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = (tid / TX) % TY, lt = tid / (TX * TY);
    const int G = gridDim.x;
    const bool has_obs = L.ocap > 0;
    const bool obs_staged = has_obs && !L.obs_direct;
    const int ostage = TN * 2 + L.ostride;     // bytes of one stage of observation tables
    unsigned char* obs_smem = smem_base + sizeof(SM);
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) mbar_init(&bars[i], 1);
        mbar_fence_init();
        abort_unit = 0;
    }
    __syncthreads();
    unsigned phbits = 0;                       // parity of the next completion of each stage's barrier
    unsigned pend = 0;                         // stages with copies issued and not yet waited for

    T c0[NTAP], c1[NTAP];
#pragma unroll
    for (int o = 0; o < NTAP; ++o) { c0[o] = L.cf[0][o]; c1[o] = L.cf[1][o]; }
    auto tap_used = [](int o) { return !(HY == 0 && tap_dy(o) != 0) && !(HT == 0 && tap_dt(o) != 0); };

    // per-thread geometry of the staged items and the s items (same every unit)
    int p_dx[KP], p_dy[KP], p_dt[KP], p_rel[KP];
    unsigned p_own = 0;     // bit k: staged item k is a node of the tile itself
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int e = tid + 256 * k;
        const int px = e % PX, py = (e / PX) % PY, pt = e / (PX * PY);
        p_dx[k] = px - HX; p_dy[k] = py - HY; p_dt[k] = pt - HT;
        p_rel[k] = (p_dt[k] * ny + p_dy[k]) * nx + p_dx[k];
        if (p_dx[k] >= 0 && p_dx[k] < TX && p_dy[k] >= 0 && p_dy[k] < TY && p_dt[k] >= 0 && p_dt[k] < TT) p_own |= 1u << k;
    }
    // s items: rows of B_w p on ring SR around the tile (s_e1: the item's
    // index in the ring-1 layout, -1 outside it)
    int s_dx[KS], s_dy[KS], s_dt[KS], s_base[KS], s_e1[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        const int e = tid + 256 * k;
        const int sx = e % SXW, sy = (e / SXW) % SY, stt = e / (SXW * SY);
        s_dx[k] = sx - SR; s_dy[k] = sy - HYS; s_dt[k] = stt;
        s_base[k] = ((stt + HT) * PY + (sy + HY - HYS)) * PX + (sx - SR + HX);
        const int x1 = sx - (SR - 1);
        s_e1[k] = (x1 >= 0 && x1 < SX) ? (stt * SY + sy) * SX + x1 : -1;
    }
    const int pbase = ((lt + HT) * PY + (ly + HY)) * PX + (lx + HX);
    const int sbase = (lt * SY + (ly + HYS)) * SX + (lx + 1);

    if (A.partial != nullptr)
        for (int i = tid; i < nblk * 4; i += 256) A.partial[((size_t)(i >> 2) * G + blockIdx.x) * 4 + (i & 3)] = 0.0;

    const int tiles_x = L.tiles_x, tiles_y = L.tiles_y, tiles_t = L.tiles_t;
    const long long chunk = ((long long)nunits + G - 1) / G;
    const long long u0 = (long long)blockIdx.x * chunk;
    const int count = (int)std::max<long long>(0, std::min<long long>(chunk, (long long)nunits - u0));

    auto issue = [&](const UnitPos& P, int st, bool valid) {
        if (valid) {
            const int grp = P.grp;
            const int tile = (P.tt * tiles_y + P.ty) * tiles_x + P.tx;
            const int tx0 = P.tx * TX, ty0 = P.ty * TY, tt0 = P.tt * TT;
            // TMA boxes (zero outside the grid): the input tile with its halo,
            // the own tiles of b, d and D^-1
            if (tid == 0) {
                const int row0 = HY > 0 ? ty0 : tt0, hrow = HY > 0 ? HY : HT;
                const bool with_d = MODE == M_CHEB && A.d != nullptr;
                const unsigned bytes = (unsigned)(PN * sizeof(V4<T>)) + (MODE != M_APPLY ? (unsigned)(TN * sizeof(V4<T>)) : 0u) +
                                       (with_d ? (unsigned)(TN * sizeof(V4<T>)) : 0u) +
                                       (MODE == M_PCG ? (unsigned)(PN * sizeof(V4<T>)) : 0u);
                mbar_expect_tx(&bars[st], bytes);
                pend |= 1u << st;
                tma_load_3d(&S.p[st][0][0], &maps.p, 4 * (tx0 - HX), row0 - hrow, grp, &bars[st]);
                if (MODE != M_APPLY) tma_load_3d(&S.b[MODE != M_APPLY ? st : 0][0][0], &maps.b, 4 * tx0, row0, grp, &bars[st]);
                if (with_d) tma_load_3d(&S.d[MODE == M_CHEB ? st : 0][0][0], &maps.d, 4 * tx0, row0, grp, &bars[st]);
                if (MODE == M_PCG) tma_load_3d(&S.z[MODE == M_PCG ? st : 0][0][0], &maps.d, 4 * (tx0 - HX), row0 - hrow, grp, &bars[st]);
            }
            // D^-1 is one value per node: its rows (4 nx bytes) need not be 16-byte
            // multiples, which a tensor map requires, so it is copied per thread
            if (MODE == M_CHEB) {
                const int gx = tx0 + lx, gy = ty0 + ly, gt = tt0 + lt;
                const bool own = gx < nx && gy < ny && gt < nt;
                cp_scalar<T>(&S.dinv[MODE == M_CHEB ? st : 0][tid], A.dinv + (own ? (gt * ny + gy) * nx + gx : 0), own);
            }
            const int tbase = (tt0 * ny + ty0) * nx + tx0;
            if (COL == 2 || COL == 4 || MODE == M_CHEB0) {      // per-node scalars of the tile and halo
#pragma unroll
                for (int k = 0; k < KP; ++k) {
                    const int e = tid + 256 * k;
                    if (KP * 256 > PN && e >= PN) break;
                    const int gx = tx0 + p_dx[k], gy = ty0 + p_dy[k], gt = tt0 + p_dt[k];
                    const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny && gt >= 0 && gt < nt;
                    const int node = in ? tbase + p_rel[k] : 0;
                    if (COL == 2 || COL == 4)
                        cp_scalar<T>(&S.mu[(COL == 2 || COL == 4) ? st : 0][(COL == 2 || COL == 4) ? e : 0], L.mu + node, in);
                    if (MODE == M_CHEB0) cp_scalar<T>(&S.dinvh[MODE == M_CHEB0 ? st : 0][MODE == M_CHEB0 ? e : 0], A.dinv + node, in);
                }
            }
            if (obs_staged) {
                unsigned char* dst = obs_smem + (size_t)st * ostage;
                const unsigned char* gmap = reinterpret_cast<const unsigned char*>(L.omap + (size_t)tile * TN);
                const unsigned char* gent = reinterpret_cast<const unsigned char*>(L.oent) + (size_t)tile * L.ostride;
                for (int c = tid; c < TN * 2 / 16; c += 256) cp_async16(dst + c * 16, gmap + c * 16, true);
                for (int c = tid; c < L.ostride / 16; c += 256) cp_async16(dst + TN * 2 + c * 16, gent + c * 16, true);
            }
        }
        cp_commit();
    };

    UnitPos cur = unit_decompose(u0 < nunits ? u0 : 0, tiles_x, tiles_y, tiles_t);
    UnitPos ahead = cur;
#pragma unroll 1
    for (int k = 0; k < NS - 1; ++k) {
        issue(ahead, k, k < count);
        unit_next(ahead, tiles_x, tiles_y, tiles_t);
    }

    T dacc[KB][4];
#pragma unroll
    for (int j = 0; j < KB; ++j) dacc[j][0] = dacc[j][1] = dacc[j][2] = dacc[j][3] = T(0);
    // PCG: alpha and beta of the unit's right-hand sides, reloaded when the
    // block group changes (a CTA's units are consecutive, so rarely)
    V4<T> pcg_a[KB], pcg_b[KB];
    int pcg_grp = -1;
    int st = 0;
#pragma unroll 1
    // Two barriers per unit: the first (after this unit's copies landed) also
    // orders every read of the previous unit (its stage buffer, the s tile,
    // qobs) before the refill of that buffer and the next writes.
    for (int done = 0; done < count; ++done) {
        fence_proxy_async();           // generic accesses of the last unit before the TMA refill below
        cp_wait<NS - 2>();
        if (mbar_wait_bounded(&bars[st], (phbits >> st) & 1u, cap)) {   // this unit's input tile
            phbits ^= 1u << st;
            pend &= ~(1u << st);
        } else {
            abort_unit = 1;
        }
        __syncthreads();
        if (abort_unit) break;
        issue(ahead, st == 0 ? NS - 1 : st - 1, done + NS - 1 < count);
        unit_next(ahead, tiles_x, tiles_y, tiles_t);
        if (GEO == GEO_XY && PER) {
            // torus: the tensor-map copy filled the halo past the grid with
            // zeros; the halo nodes within two of the torus take their
            // wrapped values (a tile at the seam only)
            const int ex0 = cur.tx * TX, ey0 = cur.ty * TY;
            if (ex0 < 2 || ex0 + TX + 2 > nx || ey0 < HY || ey0 + TY + HY > ny) {
                const T* src = MODE == M_CHEB0 ? A.b : A.x;
#pragma unroll
                for (int k = 0; k < KP; ++k) {
                    const int e = tid + 256 * k;
                    if (KP * 256 > PN && e >= PN) break;
                    const int gx = ex0 + p_dx[k], gy = ey0 + p_dy[k];
                    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) continue;
                    if (gx < -2 || gx > nx + 1 || gy < -2 || gy > ny + 1) continue;
                    const int node = wrap_idx(gy, ny) * nx + wrap_idx(gx, nx);
#pragma unroll
                    for (int j = 0; j < KB; ++j) {
                        const int blk = cur.grp * KB + j;
                        if (blk < nblk) S.p[st][e][j] = v4load(src + ((size_t)blk * N + node) * RW);
                    }
                    if (MODE == M_CHEB0) S.dinvh[MODE == M_CHEB0 ? st : 0][MODE == M_CHEB0 ? e : 0] = A.dinv[node];
                    if (MODE == M_PCG) {
#pragma unroll
                        for (int j = 0; j < KB; ++j) {
                            const int blk = cur.grp * KB + j;
                            if (blk < nblk) S.z[MODE == M_PCG ? st : 0][MODE == M_PCG ? e : 0][j] = v4load(A.d + ((size_t)blk * N + node) * RW);
                        }
                    }
                }
                if (MODE != M_CHEB0) __syncthreads();   // the in-place step below has its own barrier
            }
        }
        V4<T> pold[KB];             // PCG: the previous direction at the own node
        if (MODE == M_PCG) {        // staged p, z -> p' = z + beta p in place
            if (cur.grp != pcg_grp) {
                pcg_grp = cur.grp;
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    const int blk = min(cur.grp * KB + j, nblk - 1);
                    const double* ap = A.alpha + (size_t)blk * RW;
                    const double* bp = A.beta + (size_t)blk * RW;
                    pcg_a[j] = V4<T>{(T)ap[0], (T)ap[1], (T)ap[2], (T)ap[3]};
                    pcg_b[j] = V4<T>{(T)bp[0], (T)bp[1], (T)bp[2], (T)bp[3]};
                }
            }
            auto upd = [&](int e, int j) {
                const V4<T> pv = S.p[st][e][j], zv = S.z[MODE == M_PCG ? st : 0][MODE == M_PCG ? e : 0][j];
                S.p[st][e][j] = V4<T>{fma(pcg_b[j].a, pv.a, zv.a), fma(pcg_b[j].b, pv.b, zv.b), fma(pcg_b[j].c, pv.c, zv.c),
                                      fma(pcg_b[j].d, pv.d, zv.d)};
            };
            // the own node is updated by its own thread, which reads the old
            // direction there first; every halo item by the thread that stages
            // it (the two sets are disjoint, so no barrier before the update)
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                pold[j] = S.p[st][pbase][j];
                upd(pbase, j);
            }
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const int e = tid + 256 * k;
                if (KP * 256 > PN && e >= PN) break;
                if ((p_own >> k) & 1u) continue;
#pragma unroll
                for (int j = 0; j < KB; ++j) upd(e, j);
            }
            __syncthreads();
        }
        if (MODE == M_CHEB0) {      // staged b -> x1 = c0 D^-1 b in place
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const int e = tid + 256 * k;
                if (KP * 256 > PN && e >= PN) break;
                const T f = A.c0 * S.dinvh[MODE == M_CHEB0 ? st : 0][MODE == M_CHEB0 ? e : 0];
#pragma unroll
                for (int j = 0; j < KB; ++j) S.p[st][e][j] = f * S.p[st][e][j];
            }
            __syncthreads();
        }
        const int grp = cur.grp;
        const int tx0 = cur.tx * TX, ty0 = cur.ty * TY, tt0 = cur.tt * TT;
        const V4<T>(*sp)[KB] = S.p[st];
        auto smu = [&](int e) -> T {
            return (COL == 2 || COL == 4) ? S.mu[(COL == 2 || COL == 4) ? st : 0][(COL == 2 || COL == 4) ? e : 0] : T(0);
        };

        // s = B p on the rows of the tile plus a one-node ring (NOISE: B_w p on
        // ring 3).  Dirichlet rows are zero; rows next to the boundary skip the
        // Dirichlet columns (App. B column elimination), all other rows take
        // every tap.
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int e = tid + 256 * k;
            if (KS * 256 > SNW && e >= SNW) break;
            const int rx = tx0 + s_dx[k], ry = ty0 + s_dy[k], rt = tt0 + s_dt[k];
            const bool inrow = rx >= rlx && rx < rhx && ry >= rly && ry < rhy && rt < nt;
            const int base = s_base[k];
            V4<T> sv[KB];
#pragma unroll
            for (int j = 0; j < KB; ++j) sv[j] = v4zero<T>();
            if (inrow && !dirich(rx, ry)) {
                const bool first = HT > 0 && nt > 1 && rt == 0;
                // a tap of a non-Dirichlet row reaches a Dirichlet column only
                // from the second or second-last node of an axis
                const bool xl = !per && rx == 1, xr = !per && rx == nx - 2;
                const bool yl = !per && HY > 0 && ry == 1, yr = !per && HY > 0 && ry == ny - 2;
#pragma unroll
                for (int o = 0; o < NTAP; ++o) {
                    if (!tap_used(o)) continue;
                    const T c = first ? c1[o] : c0[o];
                    if (c == T(0)) continue;
                    const bool hit = (tap_dx(o) < 0 && xl) || (tap_dx(o) > 0 && xr) || (tap_dy(o) < 0 && yl) ||
                                     (tap_dy(o) > 0 && yr);
                    if (hit) continue;
#pragma unroll
                    for (int j = 0; j < KB; ++j) sv[j] = fma4(c, sp[base + poff<PX, PY>(o)][j], sv[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                if (NOISE) S.sw[NOISE ? e : 0][j] = sv[j];
                else S.s[e][j] = sv[j];
            }
            const int e1 = s_e1[k];        // collocation rows on ring 1 only
            if (COL && e1 < 0) continue;
            if (COL == 1 || COL == 2) {
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    V4<T> sjv = v4zero<T>();
                    if (inrow && rx >= 1 && rx <= nx - 2 && rt >= 1 && colloc_on(L.col, rx, rt)) {
                        T cC, cL, cR;
                        jcoef<T, COL>(L.col, smu(base), smu(base - 1), smu(base + 1), cC, cL, cR);
                        sjv = cC * sp[base][j];
                        sjv = fma4(cL, sp[base - 1][j], sjv);
                        sjv = fma4(cR, sp[base + 1][j], sjv);
                        sjv = fma4((T)(-L.col.inv_dt), sp[base - PY * PX][j], sjv);
                    }
                    S.sj[COL ? e1 : 0][j] = sjv;
                }
            } else if (COL >= 3) {
                // FEM Crank-Nicolson row: taps x-1, x, x+1 on this level and the one before
                constexpr int TP = PY * PX;           // one time level back in the staged tile
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    V4<T> sjv = v4zero<T>();
                    if (inrow && rx >= 1 && rx <= nx - 2 && rt >= 1 && colloc_on(L.col, rx, rt)) {
                        T dk[3], dp[3];
                        fem_cn_half_conv<T>(L.col, smu(base - 1), smu(base), smu(base + 1), dk);
                        fem_cn_half_conv<T>(L.col, smu(base - TP - 1), smu(base - TP), smu(base - TP + 1), dp);
#pragma unroll
                        for (int e3 = 0; e3 < 3; ++e3) {
                            sjv = fma4(fem_cn_fixed<T>(L.col, e3, T(1)) + dk[e3], sp[base + e3 - 1][j], sjv);
                            sjv = fma4(fem_cn_fixed<T>(L.col, e3, T(-1)) + dp[e3], sp[base - TP + e3 - 1][j], sjv);
                        }
                    }
                    S.sj[COL ? e1 : 0][j] = sjv;
                }
            }
        }
        // A^T R^-1 A p at the observed nodes of the tile: entry e (one node's
        // 3^k-point stencil) is evaluated by thread 255 - e, so only the last
        // ceil(entries / 32) warps run the loop
        // this tile's tables: the staged copy, or global memory when a level's
        // tables are too large to stage (small, heavily observed coarse levels)
        const int16_t* omap_t = nullptr;
        const unsigned char* oent_t = nullptr;
        if (has_obs) {
            if (obs_staged) {
                omap_t = reinterpret_cast<const int16_t*>(obs_smem + (size_t)st * ostage);
                oent_t = obs_smem + (size_t)st * ostage + TN * 2;
            } else {
                const int tile = (cur.tt * tiles_y + cur.ty) * tiles_x + cur.tx;
                omap_t = L.omap + (size_t)tile * TN;
                oent_t = reinterpret_cast<const unsigned char*>(L.oent) + (size_t)tile * L.ostride;
            }
        }
        const int oe = 255 - tid;      // entries go to the last warps (the first ones hold extra s rows)
        if (has_obs && oe < L.ocap) {
            const int nd = reinterpret_cast<const int16_t*>(oent_t + (size_t)L.ocap * OC * sizeof(T))[oe];
            if (nd >= 0) {
                const int ex = nd % TX, ey = (nd / TX) % TY, et = nd / (TX * TY);
                const int pb = ((et + HT) * PY + (ey + HY)) * PX + (ex + HX);
                const T* c = reinterpret_cast<const T*>(oent_t) + oe * OC;
                V4<T> v[KB];
#pragma unroll
                for (int j = 0; j < KB; ++j) v[j] = v4zero<T>();
#pragma unroll
                for (int a = 0; a < OC; ++a) {
                    const int po = pb + (obs_dt(GEO, a) * PY + obs_dy(GEO, a)) * PX + obs_dx(GEO, a);
#pragma unroll
                    for (int j = 0; j < KB; ++j) v[j] = fma4(c[a], sp[po][j], v[j]);
                }
#pragma unroll
                for (int j = 0; j < KB; ++j) S.qobs[nd][j] = v[j];
            }
        }
        __syncthreads();
        if (NOISE) {
            // s <- T_K T_K s: T_K = tk_c on the diagonal and tk_o to the two
            // x neighbours, between interior rows of levels t >= 1 (identity
            // on the boundary rows and the initial level)
            const T tc = (T)L.tk_c, to = (T)L.tk_o;
            auto tk = [&](const V4<T>* src, int i, int rx, int rt) -> V4<T> {
                V4<T> v = src[i];
                if (rt >= 1 && rt < nt && rx >= 1 && rx <= nx - 2) {
                    V4<T> w = tc * v;
                    if (rx - 1 >= 1) w = fma4(to, src[i - 1], w);
                    if (rx + 1 <= nx - 2) w = fma4(to, src[i + 1], w);
                    v = w;
                }
                return v;
            };
            for (int e = tid; e < (NOISE ? SN2 : 1); e += 256) {       // ring 3 -> ring 2
                const int sx = e % SX2, stt = e / SX2;
                const int rx = tx0 - 2 + sx, rt = tt0 + stt;
                S.s2[NOISE ? e : 0][0] = tk(reinterpret_cast<const V4<T>*>(S.sw), stt * SXW + sx + 1, rx, rt);
            }
            __syncthreads();
            for (int e = tid; e < SN; e += 256) {                       // ring 2 -> ring 1
                const int sx = e % SX, stt = e / SX;
                const int rx = tx0 - 1 + sx, rt = tt0 + stt;
                S.s[e][0] = tk(reinterpret_cast<const V4<T>*>(S.s2), stt * SX2 + sx + 1, rx, rt);
            }
            __syncthreads();
        }

        // q = B^T s (+ J^T Q_eps sj + A^T R^-1 A p) at the thread's own node
        const int gx = tx0 + lx, gy = ty0 + ly, gt = tt0 + lt;
        const bool own = gx < nx && gy < ny && gt < nt;
        const int node = own ? (gt * ny + gy) * nx + gx : 0;
        V4<T> q[KB], pown[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) { q[j] = v4zero<T>(); pown[j] = sp[pbase][j]; }
        if (own) {
            if (dirich(gx, gy)) {
#pragma unroll
                for (int j = 0; j < KB; ++j) q[j] = L.inv_eps2 * pown[j];
            } else {
#pragma unroll
                for (int o = 0; o < NTAP; ++o) {
                    if (!tap_used(o)) continue;
                    const bool first = HT > 0 && nt > 1 && gt - tap_dt(o) == 0;
                    const T c = first ? c1[o] : c0[o];
                    if (c == T(0)) continue;
#pragma unroll
                    for (int j = 0; j < KB; ++j) q[j] = fma4(c, S.s[sbase + soff<SX, SY>(o)][j], q[j]);
                }
            }
            if (COL >= 3) {
                // FEM Crank-Nicolson rows touching this column: (x+d, t) by their
                // tap -d on their own level, (x+d, t+1) by their tap -d on the
                // level before; both carry the half convection derivative of
                // row x+d at level t
                const int sb = lt * SX + (lx + 1);
                T dd[3][3];
#pragma unroll
                for (int d = -1; d <= 1; ++d)
                    fem_cn_half_conv<T>(L.col, smu(pbase + d - 1), smu(pbase + d), smu(pbase + d + 1), dd[d + 1]);
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    V4<T> acc = v4zero<T>();
#pragma unroll
                    for (int d = -1; d <= 1; ++d) {
                        const T hd = dd[d + 1][1 - d];
                        acc = fma4(fem_cn_fixed<T>(L.col, 1 - d, T(1)) + hd, S.sj[COL ? sb + d : 0][j], acc);
                        acc = fma4(fem_cn_fixed<T>(L.col, 1 - d, T(-1)) + hd, S.sj[COL ? sb + SX + d : 0][j], acc);
                    }
                    q[j] = fma4((T)L.col.qeps, acc, q[j]);
                }
            } else if (COL) {
                // rows touching this column: itself (centre), x-1 row (its x+1 tap),
                // x+1 row (its x-1 tap), t+1 row (its t-1 tap)
                const int sb = lt * SX + (lx + 1);
                T cC, cL, cR, tC, tL, tR, uC, uL, uR;
                const T m0 = smu(pbase), mm1 = smu(pbase - 1), mp1 = smu(pbase + 1);
                const T mm2 = smu(pbase - 2), mp2 = smu(pbase + 2);
                jcoef<T, COL>(L.col, m0, mm1, mp1, cC, cL, cR);
                jcoef<T, COL>(L.col, mm1, mm2, m0, tC, tL, tR);
                jcoef<T, COL>(L.col, mp1, m0, mp2, uC, uL, uR);
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    V4<T> acc = cC * S.sj[COL ? sb : 0][j];
                    acc = fma4(tR, S.sj[COL ? sb - 1 : 0][j], acc);
                    acc = fma4(uL, S.sj[COL ? sb + 1 : 0][j], acc);
                    acc = fma4((T)(-L.col.inv_dt), S.sj[COL ? sb + SX : 0][j], acc);
                    q[j] = fma4((T)L.col.qeps, acc, q[j]);
                }
            }
            if (has_obs) {
                if (omap_t[tid] >= 0) {
#pragma unroll
                    for (int j = 0; j < KB; ++j) q[j] = q[j] + S.qobs[tid][j];
                }
            }
        }

        // epilogue
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            const int blk = grp * KB + j;
            if (!own || blk >= nblk) continue;
            const size_t off = ((size_t)blk * N + node) * RW;
            if (MODE == M_APPLY || MODE == M_PCG) {
                v4store(A.out + off, q[j]);
                dacc[j][0] += pown[j].a * q[j].a; dacc[j][1] += pown[j].b * q[j].b;
                dacc[j][2] += pown[j].c * q[j].c; dacc[j][3] += pown[j].d * q[j].d;
                if (MODE == M_PCG) {
                    const V4<T> xo = S.b[MODE != M_APPLY ? st : 0][tid][j];
                    v4store(A.out2 + off, pown[j]);
                    v4store(A.out3 + off, V4<T>{fma(pcg_a[j].a, pold[j].a, xo.a), fma(pcg_a[j].b, pold[j].b, xo.b),
                                                fma(pcg_a[j].c, pold[j].c, xo.c), fma(pcg_a[j].d, pold[j].d, xo.d)});
                }
            } else if (MODE == M_RESID) {
                const V4<T> r = S.b[MODE != M_APPLY ? st : 0][tid][j] - q[j];
                v4store(A.out + off, r);
                const T w = A.rweight != nullptr ? A.rweight[node] : T(1);
                dacc[j][0] += w * r.a * r.a; dacc[j][1] += w * r.b * r.b;
                dacc[j][2] += w * r.c * r.c; dacc[j][3] += w * r.d * r.d;
            } else {
                const V4<T> bb = S.b[MODE != M_APPLY ? st : 0][tid][j];
                const V4<T> r = bb - q[j];
                const T di = MODE == M_CHEB0 ? S.dinvh[MODE == M_CHEB0 ? st : 0][MODE == M_CHEB0 ? pbase : 0]
                                             : S.dinv[MODE == M_CHEB ? st : 0][tid];
                V4<T> dn = (A.c2 * di) * r;
                if (MODE == M_CHEB0) dn = fma4(A.c1, pown[j], dn);          // d = x1
                else if (A.d != nullptr) dn = fma4(A.c1, S.d[MODE == M_CHEB ? st : 0][tid][j], dn);
                const V4<T> xn = pown[j] + dn;
                v4store(A.out + off, xn);
                v4store(A.out2 + off, dn);
                dacc[j][0] += bb.a * xn.a; dacc[j][1] += bb.b * xn.b; dacc[j][2] += bb.c * xn.c; dacc[j][3] += bb.d * xn.d;
            }
        }
        // dot partials: one entry per (block, CTA), flushed when the group changes
        UnitPos nxt = cur;
        unit_next(nxt, tiles_x, tiles_y, tiles_t);
        if (A.partial != nullptr) {
            if (nxt.grp != grp || done + 1 == count) {
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    const int blk = grp * KB + j;
                    if (blk < nblk) block_sum4<256, T>(dacc[j], A.partial + ((size_t)blk * G + blockIdx.x) * 4);
                    dacc[j][0] = dacc[j][1] = dacc[j][2] = dacc[j][3] = T(0);
                }
            }
        }
        cur = nxt;
        st = st + 1 == NS ? 0 : st + 1;
    }
    cp_wait<0>();
    if (tid == 0 && abort_unit) {
        mbar_drain(bars, NS, pend, phbits, kMbarSpinCap);
        atomicExch(&g_stencil_abort, 1);
    }
}

// Tensor map of a blocked vector [nblk][N][4] seen as a 3D array (4 nx
// values, rows, blocks) whose rows are y (2D) or t (1D space x time); the box
// is one tile's input with its halo.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiled encode_tiled() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        cuda_ok(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || f == nullptr) throw std::runtime_error("cuTensorMapEncodeTiled not available");
        fn = reinterpret_cast<EncodeTiled>(f);
    });
    return fn;
}

void encode_tensor_map(CUtensorMap* m, bool f64, int rank, const void* base, const cuuint64_t* dims,
                       const cuuint64_t* strides, const cuuint32_t* box) {
    std::memset(m, 0, sizeof(*m));
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = encode_tiled()(m, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                      (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, estr,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw std::runtime_error("tensor map of a stencil operand: error " + std::to_string((int)r));
}

template <int GEO, typename T, int NOISE = 0>
static CUtensorMap tile_map(const T* v, const LevelView<T>& L, int nblk, bool halo) {
    using G = Geo<GEO>;
    static_assert(G::HY == 0 || G::TT == 1, "2D tiles have one time level");
    constexpr int PX = G::TX + (NOISE ? 8 : 4), PR = G::HY > 0 ? G::TY + 2 * G::HY : G::TT + 2 * G::HT;
    constexpr int TR = G::HY > 0 ? G::TY : G::TT;
    const cuuint64_t rows = G::HY > 0 ? (cuuint64_t)L.ny : (cuuint64_t)L.nt;
    const cuuint64_t dims[3] = {(cuuint64_t)4 * L.nx, rows, (cuuint64_t)nblk};
    const cuuint64_t strides[2] = {(cuuint64_t)4 * L.nx * sizeof(T), (cuuint64_t)L.N * 4 * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)(4 * (halo ? PX : G::TX)), (cuuint32_t)(halo ? PR : TR), 1};
    CUtensorMap m;
    encode_tensor_map(&m, sizeof(T) == 8, 3, v, dims, strides, box);
    return m;
}

void set_wait_cap(int cap) {
    const int v = cap;
    cuda_ok(cudaMemcpyToSymbol(g_stencil_wait_cap, &v, sizeof(int)));
    march_set_wait_cap(v);
}

void stencil_abort_peek_async(int32_t* host2, cudaStream_t s) {
    cuda_ok(cudaMemcpyFromSymbolAsync(host2, g_stencil_abort, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    march_abort_peek_async(host2 + 1, s);
}

int stencil_abort_take(cudaStream_t s) {
    int v = 0;
    cuda_ok(cudaMemcpyFromSymbolAsync(&v, g_stencil_abort, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    cuda_ok(cudaStreamSynchronize(s));
    if (v) {
        static const int zero = 0;
        cuda_ok(cudaMemcpyToSymbolAsync(g_stencil_abort, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
        cuda_ok(cudaStreamSynchronize(s));
    }
    return v | march_abort_take(s);
}

// Largest persistent grid any stencil launch uses (sizes the partial buffers).
constexpr int kMaxStencilGrid = 4096;

#ifndef GMRF_STENCIL_STAGES
#define GMRF_STENCIL_STAGES 2
#endif
#ifndef GMRF_STENCIL_KB
#define GMRF_STENCIL_KB 1
#endif

static const char* mode_name(int m) {
    return m == M_APPLY ? "apply" : m == M_RESID ? "resid" : m == M_CHEB ? "cheb" : m == M_CHEB0 ? "cheb0" : "pcg";
}
template <int GEO, typename T, int MODE, int COL, int PER> static std::string stencil_name() {
    return std::string("stencil<") + (GEO == GEO_XY ? (PER ? "torus" : "xy") : "xt") + (sizeof(T) == 8 ? ",f64," : ",f32,") +
           mode_name(MODE) + ",col" + std::to_string(COL) + ">";
}

// dry: only the one-time set-up of this instantiation (function attributes,
// occupancy query, which also loads the kernel's code), no launch
template <int GEO, typename T, int MODE, int COL, int PER, int NOISE = 0>
static int launch_one(const StencilArgs<T>& a, cudaStream_t s, bool dry = false) {
    constexpr int NS = sizeof(T) == 8 ? 2 : GMRF_STENCIL_STAGES;
    constexpr int KB = sizeof(T) == 8 ? 1 : GMRF_STENCIL_KB;
    using SM = StencilSmem<GEO, T, MODE, COL, NS, KB, NOISE>;
    auto kern = k_stencil<GEO, T, MODE, COL, NS, KB, PER, NOISE>;
    static int attr_smem = 0;
    static int sms = 0, optin = 0;
    static std::map<size_t, int> per_sm;       // resident CTAs per SM by dynamic shared memory
    static std::mutex mu;                      // solves of independent posteriors may run on several host threads
    StencilArgs<T> args = a;
    size_t smem = sizeof(SM) + 128;            // + alignment slack of the TMA destinations
    int resident = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (sms == 0) {
            int dev = 0;
            cuda_ok(cudaGetDevice(&dev));
            cuda_ok(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            cuda_ok(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        }
        // stage the observation tables with the inputs when they fit beside
        // them (with the 1 KB the block reduction's static array may take)
        const size_t staged = sizeof(SM) + 128 + (size_t)NS * (SM::TN * 2 + a.L.ostride);
        args.L.obs_direct = 0;
        if (a.L.ocap > 0) {
            if (staged + 1024 <= (size_t)optin) smem = staged;
            else args.L.obs_direct = 1;
        }
        if (smem + 1024 > (size_t)optin) throw std::runtime_error("stencil kernel does not fit in shared memory");
        if ((int)smem > attr_smem) {
            cuda_ok(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr_smem = (int)smem;
        }
        auto itp = per_sm.find(smem);
        if (itp == per_sm.end()) {
            int per = 0;
            cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, smem));
            if (per <= 0) throw std::runtime_error("stencil kernel does not fit on an SM (shared memory)");
            itp = per_sm.emplace(smem, per).first;
        }
        resident = sms * itp->second;
    }
    if (dry) return 0;
    const long long ntiles = (long long)a.L.tiles_x * a.L.tiles_y * a.L.tiles_t;
    const long long nunits = ntiles * ((a.nblk + KB - 1) / KB);
    const int per = resident / sms;
    const int nsm = sms;
    auto grid_of = [nunits, nsm](int k) {
        return (int)std::min<long long>(std::min<long long>(nunits, (long long)nsm * k), kMaxStencilGrid);
    };
    auto run = [kern, smem, nunits](const StencilArgs<T>& aa, int grid, cudaStream_t st, bool count) {
        StencilMaps maps;
        std::memset(&maps, 0, sizeof(maps));
        maps.p = tile_map<GEO, T, NOISE>(MODE == M_CHEB0 ? aa.b : aa.x, aa.L, aa.nblk, true);
        if (MODE != M_APPLY) maps.b = tile_map<GEO, T, NOISE>(aa.b, aa.L, aa.nblk, false);
        if (MODE == M_CHEB && aa.d != nullptr) maps.d = tile_map<GEO, T, NOISE>(aa.d, aa.L, aa.nblk, false);
        if (MODE == M_PCG) maps.d = tile_map<GEO, T, NOISE>(aa.d, aa.L, aa.nblk, true);
        kern<<<(unsigned)grid, 256, smem, st>>>(aa, (int)nunits, maps);
        if (count) note_launch();
    };
    int grid = grid_of(per);
    // launch shape: measured once per key when there is more than one unit per SM
    if (nunits > nsm && per > 1) {
        const TuneKey key{stencil_name<GEO, T, MODE, COL, PER>() + (NOISE ? "+noise" : ""), args.nblk, tune_units_bucket(nunits),
                          tune_obs_bucket(args.L.ostride, args.L.ocap > 0)};
        auto measure = [key, args, per, grid_of, run](cudaStream_t st) {
            TuneChoice c;
            if (tune_lookup(key, &c)) return c;
            TuneScratch sc;
            StencilArgs<T> t = args;
            const size_t vb = (size_t)args.nblk * args.L.N * 4 * sizeof(T);
            t.x = (const T*)sc.zeros(vb, st);
            t.b = (const T*)sc.zeros(vb, st);
            if (args.d) t.d = (const T*)sc.zeros(vb, st);
            t.out = (T*)sc.zeros(vb, st);
            if (args.out2) t.out2 = (T*)sc.zeros(vb, st);
            if (args.out3) t.out3 = (T*)sc.zeros(vb, st);
            if (args.alpha) t.alpha = (const double*)sc.zeros(sizeof(double) * 4 * args.nblk, st);
            if (args.beta) t.beta = (const double*)sc.zeros(sizeof(double) * 4 * args.nblk, st);
            if (args.partial) t.partial = (double*)sc.zeros(sizeof(double) * 4 * args.nblk * kMaxStencilGrid, st);
            std::vector<TuneChoice> cands;
            for (int k = per; k >= 1; --k) cands.push_back(TuneChoice{k, 0});
            return tune_measure(key, cands, [&](const TuneChoice& cc, cudaStream_t s2) { run(t, grid_of(cc.ctas_per_sm), s2, false); }, st);
        };
        TuneChoice c;
        if (tune_lookup(key, &c)) grid = grid_of(c.ctas_per_sm);
        else if (tune_now(s)) grid = grid_of(measure(s).ctas_per_sm);
        else tune_defer([measure](cudaStream_t st) { measure(st); });
    }
    run(args, grid, s, true);
    return grid;
}

template <int GEO, typename T, int MODE>
static int launch_geo_mode(const StencilArgs<T>& a, cudaStream_t s, bool dry) {
    if (GEO == GEO_XT && a.L.noise) {       // Matern transition noise: point data or Burgers rows
        constexpr int NZ = GEO == GEO_XT ? 1 : 0;
        if (a.L.col.kind == 0) return launch_one<GEO, T, MODE, 0, 0, NZ>(a, s, dry);
        if (a.L.col.kind == 2) return launch_one<GEO, T, MODE, (GEO == GEO_XT ? 2 : 0), 0, NZ>(a, s, dry);
        if (a.L.col.kind == 4) return launch_one<GEO, T, MODE, (GEO == GEO_XT ? 4 : 0), 0, NZ>(a, s, dry);
        throw std::runtime_error("Matern transition noise: point data or Burgers rows only");
    }
    if (GEO == GEO_XT && a.L.col.kind == 1) return launch_one<GEO, T, MODE, (GEO == GEO_XT ? 1 : 0), 0>(a, s, dry);
    if (GEO == GEO_XT && a.L.col.kind == 2) return launch_one<GEO, T, MODE, (GEO == GEO_XT ? 2 : 0), 0>(a, s, dry);
    if (GEO == GEO_XT && a.L.col.kind == 3) return launch_one<GEO, T, MODE, (GEO == GEO_XT ? 3 : 0), 0>(a, s, dry);
    if (GEO == GEO_XT && a.L.col.kind == 4) return launch_one<GEO, T, MODE, (GEO == GEO_XT ? 4 : 0), 0>(a, s, dry);
    if (GEO == GEO_XY && a.L.periodic) return launch_one<GEO, T, MODE, 0, (GEO == GEO_XY ? 1 : 0)>(a, s, dry);
    return launch_one<GEO, T, MODE, 0, 0>(a, s, dry);
}

template <typename T, int GEO>
static int launch_geo(int mode, const StencilArgs<T>& a, cudaStream_t s, bool dry = false) {
    if (mode == M_APPLY) return launch_geo_mode<GEO, T, M_APPLY>(a, s, dry);
    if (mode == M_RESID) return launch_geo_mode<GEO, T, M_RESID>(a, s, dry);
    if (mode == M_CHEB0) return launch_geo_mode<GEO, T, M_CHEB0>(a, s, dry);
    if (mode == M_PCG) return launch_geo_mode<GEO, T, M_PCG>(a, s, dry);
    return launch_geo_mode<GEO, T, M_CHEB>(a, s, dry);
}

template <typename T> void stencil_check_args(int mode, int col, const StencilArgs<T>& a) {
    auto need = [&](const void* p, const char* what) {
        if (p == nullptr) throw std::runtime_error(std::string("stencil launch: ") + what + " is required for mode " + mode_name(mode));
    };
    if (mode != M_APPLY && mode != M_RESID && mode != M_CHEB && mode != M_CHEB0 && mode != M_PCG)
        throw std::runtime_error("stencil launch: unknown mode");
    if (a.nblk <= 0 || a.L.N <= 0) throw std::runtime_error("stencil launch: empty batch or level");
    need(a.out, "out");
    if (mode != M_CHEB0) need(a.x, "x");
    if (mode != M_APPLY) need(a.b, "b");
    if (mode == M_CHEB || mode == M_CHEB0) { need(a.dinv, "dinv"); need(a.out2, "out2"); }
    if (mode == M_PCG) {
        need(a.d, "d (z)"); need(a.out2, "out2 (p')"); need(a.out3, "out3 (iterate)");
        need(a.alpha, "alpha"); need(a.beta, "beta");
    }
    if (col == 2 || col == 4) need(a.L.mu, "the linearisation point");
    if (a.L.ocap > 0) { need(a.L.omap, "observation map"); need(a.L.oent, "observation entries"); }
}
template void stencil_check_args<float>(int, int, const StencilArgs<float>&);
template void stencil_check_args<double>(int, int, const StencilArgs<double>&);

template <typename T> int launch_stencil(int geo, int mode, const StencilArgs<T>& a, cudaStream_t s) {
    stencil_check_args<T>(mode, a.L.col.kind, a);
    if (geo == GEO_XY) return launch_geo<T, GEO_XY>(mode, a, s);
    if (geo == GEO_XT) return launch_geo<T, GEO_XT>(mode, a, s);
    return launch_march<T>(mode, a, s);
}
template int launch_stencil<float>(int, int, const StencilArgs<float>&, cudaStream_t);
template int launch_stencil<double>(int, int, const StencilArgs<double>&, cudaStream_t);

template <typename T> void stencil_prepare(int geo, int mode, const StencilArgs<T>& a) {
    if (geo == GEO_XY) launch_geo<T, GEO_XY>(mode, a, 0, true);
    else if (geo == GEO_XT) launch_geo<T, GEO_XT>(mode, a, 0, true);
    else march_prepare<T>(mode, a);
}
template void stencil_prepare<float>(int, int, const StencilArgs<float>&);
template void stencil_prepare<double>(int, int, const StencilArgs<double>&);
int stencil_max_grid() { return kMaxStencilGrid; }

}  // namespace gmrf
