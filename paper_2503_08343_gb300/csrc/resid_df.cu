// Refinement residual r = b - Q_u|y x in double-float arithmetic.
//
// The iterative refinement needs b - Q x to about 1e-14 relative accuracy
// (its target is a relative residual of 1e-10).  GB300 issues FP64 at about
// 1/64 of the FP32 rate, so the FP64 form of the fused stencil is compute-
// bound at ~1 ms for the 512^2, 65-RHS workload.  Here every value is a pair
// of floats (hi + lo, about 48 significant bits): staged FP64 inputs are split
// with integer operations, products and sums use the error-free FMA-based
// transformations (Dekker / Knuth two-product and two-sum), and the residual
// is stored as the pair (hi, lo) in the 8 bytes of the FP64 slot.  The inner
// FP32 solve only reads hi; the weighted norm is accumulated from hi.  The
// tiling, staging and unit order follow the 2D / 1D-space-time kernel
// (GEO_XY and GEO_XT without collocation rows).
#include <algorithm>
#include <map>
#include <mutex>
#include <stdexcept>
#include <string>

#include "kernels.h"

namespace gmrf {

namespace {

struct alignas(8) dfl {
    float hi, lo;
};
static_assert(sizeof(dfl) == sizeof(double), "a pair fills an FP64 slot");

// d = hi + lo to about 2^-48 relative: hi is d truncated to 24 significant
// bits, lo the remaining 29 bits rounded to 24 (scaled in two steps below
// 2^-74).  Integer and FP32 operations only, no FP64 instructions; magnitudes
// below the FP32 normal range (2^-126) become zero.
__device__ __forceinline__ dfl split_double(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned sign = (unsigned)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7ff) - 1023;          // unbiased exponent
    const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    dfl r;
    if (e < -126) { r.hi = 0.f; r.lo = 0.f; return r; }    // below the FP32 normal range
    if (e > 127) { r.hi = __int_as_float((int)(sign | 0x7f800000u)); r.lo = 0.f; return r; }
    r.hi = __int_as_float((int)(sign | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29)));
    const unsigned rem = (unsigned)(m & ((1ull << 29) - 1));
    if (rem == 0) { r.lo = 0.f; return r; }
    const int es = e - 52 + 127;                             // biased exponent of 2^(e - 52)
    float lo = es >= 1 ? (float)rem * __int_as_float(es << 23)
                       : ((float)rem * __int_as_float((es + 64) << 23)) * __int_as_float((127 - 64) << 23);
    r.lo = __int_as_float(__float_as_int(lo) | (int)sign);
    return r;
}

// acc + c * x with c, x, acc pairs
__device__ __forceinline__ dfl df_fma(dfl c, dfl x, dfl acc) {
    const float p = c.hi * x.hi;
    float e = fmaf(c.hi, x.hi, -p);                          // exact error of the product
    e = fmaf(c.hi, x.lo, e);
    e = fmaf(c.lo, x.hi, e);
    const float s = acc.hi + p;                              // two-sum of acc.hi and p
    const float bv = s - acc.hi;
    float t = (acc.hi - (s - bv)) + (p - bv);
    t += acc.lo + e;
    dfl r;
    r.hi = s + t;                                            // renormalise
    r.lo = t - (r.hi - s);
    return r;
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    const float s = a.hi + b.hi;
    const float bv = s - a.hi;
    float t = (a.hi - (s - bv)) + (b.hi - bv);
    t += a.lo + b.lo;
    dfl r;
    r.hi = s + t;
    r.lo = t - (r.hi - s);
    return r;
}

__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.hi, -a.lo}; }

struct alignas(16) V4d {
    dfl a, b, c, d;
};
__device__ __forceinline__ V4d v4d_zero() { return V4d{{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ V4d v4d_fma(dfl c, const V4d& x, const V4d& acc) {
    return V4d{df_fma(c, x.a, acc.a), df_fma(c, x.b, acc.b), df_fma(c, x.c, acc.c), df_fma(c, x.d, acc.d)};
}
__device__ __forceinline__ V4d v4d_add(const V4d& x, const V4d& y) {
    return V4d{df_add(x.a, y.a), df_add(x.b, y.b), df_add(x.c, y.c), df_add(x.d, y.d)};
}

template <int GEO> struct DfSmem {
    using G = Geo<GEO>;
    static constexpr int TX = G::TX, TY = G::TY, TT = G::TT, HY = G::HY, HT = G::HT;
    static constexpr int PX = TX + 4, PY = TY + 2 * HY, PT = TT + 2 * HT;
    static constexpr int SX = TX + 2, SY = TY + HY, ST = TT + HT;
    static constexpr int TN = TX * TY * TT, PN = PX * PY * PT, SN = SX * SY * ST;
    V4d p[2][PN];              // staged as FP64, converted in place to pairs
    V4d b[2][TN];              // FP64
    V4d s[SN];
    V4d qobs[TN];
};

void ok(cudaError_t e) {
    if (e != cudaSuccess) throw std::runtime_error(std::string("kernel setup: ") + cudaGetErrorString(e));
}

template <int GEO>
__global__ void __launch_bounds__(256) k_resid_df(const LevelView<double> L, const double* __restrict__ x,
                                                  const double* __restrict__ bvec, double* __restrict__ out,
                                                  const double* __restrict__ rweight, double* __restrict__ partial,
                                                  int nblk, int nunits) {
    using SM = DfSmem<GEO>;
    constexpr int TX = SM::TX, TY = SM::TY, TT = SM::TT, HY = SM::HY, HT = SM::HT;
    constexpr int PX = SM::PX, PY = SM::PY, PN = SM::PN, TN = SM::TN;
    constexpr int SX = SM::SX, SY = SM::SY, SN = SM::SN;
    constexpr int HYS = HY / 2;
    constexpr int OC = ObsStencil<GEO>::OC;
    constexpr int KP = (PN + 255) / 256, KS = (SN + 255) / 256;
    static_assert(TN == 256, "one thread per node of the tile");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM& S = *reinterpret_cast<SM*>(smem_raw);
    const int nx = L.nx, ny = L.ny, nt = L.nt;
    const long long N = L.N;
    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = (tid / TX) % TY, lt = tid / (TX * TY);
    const int G = gridDim.x;
    const bool has_obs = L.ocap > 0;
    const bool obs_staged = has_obs && !L.obs_direct;
    const int ostage = TN * 2 + L.ostride;
    unsigned char* obs_smem = smem_raw + sizeof(SM);
    auto tap_used = [](int o) { return !(HY == 0 && tap_dy(o) != 0) && !(HT == 0 && tap_dt(o) != 0); };

    dfl c0[NTAP], c1[NTAP];
#pragma unroll
    for (int o = 0; o < NTAP; ++o) { c0[o] = split_double(L.cf[0][o]); c1[o] = split_double(L.cf[1][o]); }
    const dfl eps2 = split_double(L.inv_eps2);

    int p_dx[KP], p_dy[KP], p_dt[KP], p_rel[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int e = tid + 256 * k;
        const int px = e % PX, py = (e / PX) % PY, pt = e / (PX * PY);
        p_dx[k] = px - 2; p_dy[k] = py - HY; p_dt[k] = pt - HT;
        p_rel[k] = (p_dt[k] * ny + p_dy[k]) * nx + p_dx[k];
    }
    int s_dx[KS], s_dy[KS], s_dt[KS], s_base[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        const int e = tid + 256 * k;
        const int sx = e % SX, sy = (e / SX) % SY, stt = e / (SX * SY);
        s_dx[k] = sx - 1; s_dy[k] = sy - HYS; s_dt[k] = stt;
        s_base[k] = ((stt + HT) * PY + (sy + HY - HYS)) * PX + (sx + 1);
    }
    const int pbase = ((lt + HT) * PY + (ly + HY)) * PX + (lx + 2);
    const int sbase = (lt * SY + (ly + HYS)) * SX + (lx + 1);

    for (int i = tid; i < nblk * 4; i += 256) partial[((size_t)(i >> 2) * G + blockIdx.x) * 4 + (i & 3)] = 0.0;

    const int tiles_x = L.tiles_x, tiles_y = L.tiles_y, tiles_t = L.tiles_t;
    const long long ntiles = (long long)tiles_x * tiles_y * tiles_t;
    const long long chunk = ((long long)nunits + G - 1) / G;
    const long long u0 = (long long)blockIdx.x * chunk;
    const int count = (int)std::max<long long>(0, std::min<long long>(chunk, (long long)nunits - u0));
    auto unit_at = [&](long long u, int& tx, int& ty, int& tt, int& grp) {
        grp = (int)(u / ntiles);
        long long tile = u - (long long)grp * ntiles;
        tx = (int)(tile % tiles_x); tile /= tiles_x;
        ty = (int)(tile % tiles_y); tt = (int)(tile / tiles_y);
    };

    auto issue = [&](long long u, int st, bool valid) {
        if (valid) {
            int tx, ty, tt, grp;
            unit_at(u, tx, ty, tt, grp);
            const int tx0 = tx * TX, ty0 = ty * TY, tt0 = tt * TT;
            const int tbase = (tt0 * ny + ty0) * nx + tx0;
            const double* xb = x + (size_t)grp * N * RW;
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const int e = tid + 256 * k;
                if (KP * 256 > PN && e >= PN) break;
                const int gx = tx0 + p_dx[k], gy = ty0 + p_dy[k], gt = tt0 + p_dt[k];
                bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny && gt >= 0 && gt < nt;
                int node = in ? tbase + p_rel[k] : 0;
                if (L.periodic && !in && gt >= 0 && gt < nt && gx >= -2 && gx <= nx + 1 && gy >= -2 && gy <= ny + 1) {
                    in = true;      // torus: the halo wraps
                    node = (gt * ny + wrap_idx(gy, ny)) * nx + wrap_idx(gx, nx);
                }
                cp_v4<double>(reinterpret_cast<V4<double>*>(&S.p[st][e]), xb + (size_t)node * RW, in);
            }
            const int gx = tx0 + lx, gy = ty0 + ly, gt = tt0 + lt;
            const bool own = gx < nx && gy < ny && gt < nt;
            const size_t node = own ? ((size_t)gt * ny + gy) * nx + gx : 0;
            cp_v4<double>(reinterpret_cast<V4<double>*>(&S.b[st][tid]), bvec + ((size_t)grp * N + node) * RW, own);
            if (obs_staged) {
                const long long tile = ((long long)tt * tiles_y + ty) * tiles_x + tx;
                unsigned char* dst = obs_smem + (size_t)st * ostage;
                const unsigned char* gmap = reinterpret_cast<const unsigned char*>(L.omap + (size_t)tile * TN);
                const unsigned char* gent = reinterpret_cast<const unsigned char*>(L.oent) + (size_t)tile * L.ostride;
                for (int c = tid; c < TN * 2 / 16; c += 256) cp_async16(dst + c * 16, gmap + c * 16, true);
                for (int c = tid; c < L.ostride / 16; c += 256) cp_async16(dst + TN * 2 + c * 16, gent + c * 16, true);
            }
        }
        cp_commit();
    };

    float wacc[4] = {0.f, 0.f, 0.f, 0.f};
    issue(u0, 0, count > 0);
    int st = 0;
#pragma unroll 1
    for (int done = 0; done < count; ++done) {
        const long long u = u0 + done;
        cp_wait<0>();
        __syncthreads();                   // unit done landed; everyone finished unit done - 1
        issue(u + 1, st ^ 1, done + 1 < count);
        int tx, ty, tt, grp;
        unit_at(u, tx, ty, tt, grp);
        const int tx0 = tx * TX, ty0 = ty * TY, tt0 = tt * TT;
        // FP64 -> pairs in place
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int e = tid + 256 * k;
            if (KP * 256 > PN && e >= PN) break;
            const V4<double> v = *reinterpret_cast<const V4<double>*>(&S.p[st][e]);
            S.p[st][e] = V4d{split_double(v.a), split_double(v.b), split_double(v.c), split_double(v.d)};
        }
        __syncthreads();
        const V4d* sp = S.p[st];
        // s = B p on the tile plus a one-node ring (Dirichlet handling as in the FP32 kernel)
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int e = tid + 256 * k;
            if (KS * 256 > SN && e >= SN) break;
            const int rx = tx0 + s_dx[k], ry = ty0 + s_dy[k], rt = tt0 + s_dt[k];
            const bool per = L.periodic != 0;     // torus: rows one past each end wrap, no Dirichlet rows
            const bool inrow = per ? (rx >= -1 && rx <= nx && ry >= -1 && ry <= ny && rt < nt)
                                   : (rx >= 0 && rx < nx && ry >= 0 && ry < ny && rt < nt);
            V4d sv = v4d_zero();
            if (inrow && (per || !is_dirichlet(rx, ry, nx, ny))) {
                const bool first = HT > 0 && nt > 1 && rt == 0;
                const bool xl = !per && rx == 1, xr = !per && rx == nx - 2;
                const bool yl = !per && HY > 0 && ry == 1, yr = !per && HY > 0 && ry == ny - 2;
#pragma unroll
                for (int o = 0; o < NTAP; ++o) {
                    if (!tap_used(o)) continue;
                    const dfl c = first ? c1[o] : c0[o];
                    if (c.hi == 0.f) continue;
                    const bool hit = (tap_dx(o) < 0 && xl) || (tap_dx(o) > 0 && xr) || (tap_dy(o) < 0 && yl) ||
                                     (tap_dy(o) > 0 && yr);
                    if (hit) continue;
                    sv = v4d_fma(c, sp[s_base[k] + (tap_dt(o) * PY + tap_dy(o)) * PX + tap_dx(o)], sv);
                }
            }
            S.s[e] = sv;
        }
        // observation entries (thread 255 - e evaluates entry e)
        const int16_t* omap_t = nullptr;
        const unsigned char* oent_t = nullptr;
        if (has_obs) {
            if (obs_staged) {
                omap_t = reinterpret_cast<const int16_t*>(obs_smem + (size_t)st * ostage);
                oent_t = obs_smem + (size_t)st * ostage + TN * 2;
            } else {
                const long long tile = ((long long)tt * tiles_y + ty) * tiles_x + tx;
                omap_t = L.omap + (size_t)tile * TN;
                oent_t = reinterpret_cast<const unsigned char*>(L.oent) + (size_t)tile * L.ostride;
            }
        }
        const int oe = 255 - tid;
        if (has_obs && oe < L.ocap) {
            const int nd = reinterpret_cast<const int16_t*>(oent_t + (size_t)L.ocap * OC * sizeof(double))[oe];
            if (nd >= 0) {
                const int ex = nd % TX, ey = (nd / TX) % TY, et = nd / (TX * TY);
                const int pb = ((et + HT) * PY + (ey + HY)) * PX + (ex + 2);
                const double* c = reinterpret_cast<const double*>(oent_t) + oe * OC;
                V4d v = v4d_zero();
#pragma unroll
                for (int a = 0; a < OC; ++a)
                    v = v4d_fma(split_double(c[a]), sp[pb + (obs_dt(GEO, a) * PY + obs_dy(GEO, a)) * PX + obs_dx(GEO, a)], v);
                S.qobs[nd] = v;
            }
        }
        __syncthreads();
        // q = B^T s (+ A^T R^-1 A p); r = b - q
        const int gx = tx0 + lx, gy = ty0 + ly, gt = tt0 + lt;
        if (gx < nx && gy < ny && gt < nt) {
            V4d q = v4d_zero();
            if (!L.periodic && is_dirichlet(gx, gy, nx, ny)) {
                q = v4d_fma(eps2, sp[pbase], q);
            } else {
#pragma unroll
                for (int o = 0; o < NTAP; ++o) {
                    if (!tap_used(o)) continue;
                    const bool first = HT > 0 && nt > 1 && gt - tap_dt(o) == 0;
                    const dfl c = first ? c1[o] : c0[o];
                    if (c.hi == 0.f) continue;
                    q = v4d_fma(c, S.s[sbase - ((tap_dt(o) * SY + tap_dy(o)) * SX + tap_dx(o))], q);
                }
            }
            if (has_obs && omap_t[tid] >= 0) q = v4d_add(q, S.qobs[tid]);
            const V4<double> bd = *reinterpret_cast<const V4<double>*>(&S.b[st][tid]);
            const V4d r = V4d{df_add(split_double(bd.a), df_neg(q.a)), df_add(split_double(bd.b), df_neg(q.b)),
                              df_add(split_double(bd.c), df_neg(q.c)), df_add(split_double(bd.d), df_neg(q.d))};
            const size_t node = ((size_t)gt * ny + gy) * nx + gx;
            *reinterpret_cast<V4d*>(out + ((size_t)grp * N + node) * RW) = r;
            const float w = rweight != nullptr ? (float)__double2float_rn(rweight[node]) : 1.f;
            wacc[0] += w * r.a.hi * r.a.hi; wacc[1] += w * r.b.hi * r.b.hi;
            wacc[2] += w * r.c.hi * r.c.hi; wacc[3] += w * r.d.hi * r.d.hi;
        }
        // dot partials: flushed when the block changes
        int ntx, nty, ntt, ngrp;
        unit_at(u + 1, ntx, nty, ntt, ngrp);
        if (ngrp != grp || done + 1 == count) {
            block_sum4<256, float>(wacc, partial + ((size_t)grp * G + blockIdx.x) * 4);
            wacc[0] = wacc[1] = wacc[2] = wacc[3] = 0.f;
        }
        st ^= 1;
    }
    cp_wait<0>();
}

constexpr int kMaxDfGrid = 4096;

template <int GEO>
int launch_geo(const LevelView<double>& Lv, const double* x, const double* b, double* out, const double* rweight,
               double* partial, int nblk, cudaStream_t s) {
    using SM = DfSmem<GEO>;
    auto kern = k_resid_df<GEO>;
    static int sms = 0, optin = 0, attr = 0;
    static std::map<size_t, int> per_sm;
    static std::mutex mu;
    LevelView<double> L = Lv;
    size_t smem = sizeof(SM);
    int resident = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (sms == 0) {
            int dev = 0;
            ok(cudaGetDevice(&dev));
            ok(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            ok(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        }
        const size_t staged = sizeof(SM) + 2 * (size_t)(SM::TN * 2 + L.ostride);
        L.obs_direct = 0;
        if (L.ocap > 0) {
            if (staged + 1024 <= (size_t)optin) smem = staged;
            else L.obs_direct = 1;
        }
        if (smem + 1024 > (size_t)optin) throw std::runtime_error("double-float residual does not fit in shared memory");
        if ((int)smem > attr) {
            ok(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr = (int)smem;
        }
        auto it = per_sm.find(smem);
        if (it == per_sm.end()) {
            int per = 0;
            ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, smem));
            if (per <= 0) throw std::runtime_error("double-float residual does not fit on an SM");
            it = per_sm.emplace(smem, per).first;
        }
        resident = sms * it->second;
    }
    const long long nunits = (long long)L.tiles_x * L.tiles_y * L.tiles_t * nblk;
    const int grid = (int)std::min<long long>(std::min<long long>(nunits, resident), kMaxDfGrid);
    { kern<<<(unsigned)grid, 256, smem, s>>>(L, x, b, out, rweight, partial, nblk, (int)nunits); note_launch(); }
    return grid;
}

__global__ void k_norm2_df(const double* __restrict__ r, long long N, double* __restrict__ partial, int nparts) {
    const int blk = blockIdx.y;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const V4d v = *reinterpret_cast<const V4d*>(r + ((size_t)blk * N + n) * RW);
        acc[0] += v.a.hi * v.a.hi; acc[1] += v.b.hi * v.b.hi; acc[2] += v.c.hi * v.c.hi; acc[3] += v.d.hi * v.d.hi;
    }
    block_sum4<256, float>(acc, partial + ((size_t)blk * nparts + blockIdx.x) * 4);
}

__global__ void k_scale_cast_df(const double* __restrict__ r, const double* __restrict__ norms, float* __restrict__ r32,
                                long long N) {
    const int blk = blockIdx.y;
    const double* nm = norms + blk * RW;
    float sc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) sc[c] = nm[c] > 0 ? __double2float_rn(nm[c]) : 0.f;
    for (int k = 0; k < EPT; ++k) {
        const long long n = (long long)blockIdx.x * ECHUNK + k * 256 + threadIdx.x;
        if (n >= N) break;
        const size_t off = ((size_t)blk * N + n) * RW;
        const V4d v = *reinterpret_cast<const V4d*>(r + off);
        v4store(r32 + off, V4<float>{sc[0] > 0 ? (v.a.hi + v.a.lo) / sc[0] : 0.f, sc[1] > 0 ? (v.b.hi + v.b.lo) / sc[1] : 0.f,
                                     sc[2] > 0 ? (v.c.hi + v.c.lo) / sc[2] : 0.f, sc[3] > 0 ? (v.d.hi + v.d.lo) / sc[3] : 0.f});
    }
}

}  // namespace

bool resid_df_applicable(const Level& L) { return (L.geo == GEO_XY || L.geo == GEO_XT) && L.col.kind == 0 && !L.noise; }

int launch_resid_df(const Level& Lv, const double* x, const double* b, double* out, const double* rweight,
                    double* partial, int nblk, cudaStream_t s) {
    const LevelView<double> L = Lv.view<double>();
    if (Lv.geo == GEO_XY) return launch_geo<GEO_XY>(L, x, b, out, rweight, partial, nblk, s);
    return launch_geo<GEO_XT>(L, x, b, out, rweight, partial, nblk, s);
}

void launch_norm2_df(const double* r, long long N, int nblk, double* partial, int nparts, cudaStream_t s) {
    { k_norm2_df<<<dim3(nparts, nblk), 256, 0, s>>>(r, N, partial, nparts); note_launch(); }
}

void launch_scale_cast_df(const double* r, const double* norms, float* r32, long long N, int nblk, cudaStream_t s) {
    { k_scale_cast_df<<<dim3(elem_parts(N), nblk), 256, 0, s>>>(r, norms, r32, N); note_launch(); }
}

}  // namespace gmrf
