// Posterior-precision stencil for 2D space x time (GEO_XYT), 2.5D-blocked.
//
// Q_u|y = B^T B + A^T R^-1 A with B the implicit-Euler space-time root
// (Sec. 2.4, App. A eq. block-tridiag-prec): row (x, y, t) of B couples the
// 7 space taps of level t and the node (x, y, t - 1).  A CTA owns a 32 x 8
// tile of the (x, y) plane and marches through a range of time levels.  It
// keeps four planes of the input (levels t - 1, t, t + 1 and t + 2 in
// flight; halo 2) and two planes of s = B p (levels t, t + 1; ring 1) in
// shared memory.  Each level then stages one input plane (1.69 entries per
// owned node) and forms one s plane (1.33 rows per owned node), the same
// ratios as the 2D kernel, where a 3D tile with a time halo needs 3.75 and
// 2.1.  Level t's output q_t = B^T s needs s_t and s_{t+1}:
//   step t:  wait for plane t + 1;  issue plane t + 2 (and level t + 1's
//            right-hand side, direction, diagonal and observation tables)
//            into the slots of level t - 2 / t - 1;  s_{t+1} from planes
//            t + 1 and t;  observation entries of level t from planes
//            t - 1 .. t + 1;  barrier;  q_t from s_t, s_{t+1};  epilogue.
// Two barriers per level; modes and epilogues as in the 2D/1D kernel.
#include <algorithm>
#include <map>
#include <mutex>
#include <stdexcept>
#include <string>

#include "kernels.h"

namespace gmrf {

namespace {

constexpr int MX = Geo<GEO_XYT>::TX, MY = Geo<GEO_XYT>::TY;
constexpr int PX = MX + 4, PY = MY + 4, PP = PX * PY;    // input plane, halo 2
constexpr int SX = MX + 2, SY = MY + 2, SP = SX * SY;    // s plane, ring 1
constexpr int KP = (PP + 255) / 256, KS = (SP + 255) / 256;
constexpr int OC = ObsStencil<GEO_XYT>::OC;
static_assert(MX * MY == 256 && Geo<GEO_XYT>::TT == 1, "one thread per node of a 32 x 8 plane tile");
static_assert(tap_dt(7) == -1 && tap_dx(7) == 0 && tap_dy(7) == 0, "tap 7 is the previous time level");

template <typename T, int MODE> struct MarchSmem {
    V4<T> p[4][PP];
    V4<T> s[2][SP];
    V4<T> b[MODE != M_APPLY ? 2 : 1][256];
    V4<T> d[MODE == M_CHEB ? 2 : 1][256];
    T dinv[MODE == M_CHEB ? 2 : 1][256];
    T dinvh[MODE == M_CHEB0 ? 4 : 1][MODE == M_CHEB0 ? PP : 1];
    V4<T> qobs[256];
};

void ok(cudaError_t e) {
    if (e != cudaSuccess) throw std::runtime_error(std::string("kernel setup: ") + cudaGetErrorString(e));
}

// Work unit u = ((grp * nchunks + chunk) * tiles_y + ty) * tiles_x + tx.  CTA
// c takes units c, c + G, ...: at any time the grid works on G consecutive
// tiles at about the same time level, so the halo planes a tile shares with
// its neighbours are read from L2 (a unit spans many levels, so flushing the
// dot partials after every unit costs little).
struct MUnit {
    int tx, ty, chunk, grp;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_march(const StencilArgs<T> A, int nunits, int tc, int nchunks) {
    using SM = MarchSmem<T, MODE>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM& S = *reinterpret_cast<SM*>(smem_raw);
    const LevelView<T>& L = A.L;
    const int nx = L.nx, ny = L.ny, nt = L.nt;
    const long long N = L.N;
    const size_t plane = (size_t)nx * ny;
    const int nblk = A.nblk;
    const int tid = threadIdx.x, lx = tid % MX, ly = tid / MX;
    const int G = gridDim.x;
    const int tiles_x = L.tiles_x, tiles_y = L.tiles_y;
    const bool has_obs = L.ocap > 0;
    const bool obs_staged = has_obs && !L.obs_direct;
    const int ostage = 256 * 2 + L.ostride;
    unsigned char* obs_smem = smem_raw + sizeof(SM);

    T c0[NTAP], c1[NTAP];
#pragma unroll
    for (int o = 0; o < NTAP; ++o) { c0[o] = L.cf[0][o]; c1[o] = L.cf[1][o]; }

    int p_dx[KP], p_dy[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int e = tid + 256 * k;
        p_dx[k] = e % PX - 2;
        p_dy[k] = e / PX - 2;
    }
    int s_dx[KS], s_dy[KS], s_base[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        const int e = tid + 256 * k;
        const int sx = e % SX, sy = e / SX;
        s_dx[k] = sx - 1;
        s_dy[k] = sy - 1;
        s_base[k] = (sy + 1) * PX + (sx + 1);
    }
    const int pown = (ly + 2) * PX + (lx + 2);
    const int sown = (ly + 1) * SX + (lx + 1);

    if (A.partial != nullptr)
        for (int i = tid; i < nblk * 4; i += 256) A.partial[((size_t)(i >> 2) * G + blockIdx.x) * 4 + (i & 3)] = 0.0;

    auto unit_at = [&](long long u) {
        MUnit m;
        m.tx = (int)(u % tiles_x); u /= tiles_x;
        m.ty = (int)(u % tiles_y); u /= tiles_y;
        m.chunk = (int)(u % nchunks);
        m.grp = (int)(u / nchunks);
        return m;
    };

    // input plane of level tau into slot tau & 3 (zero outside the grid)
    auto stage_p = [&](int grp, int tx0, int ty0, int tau) {
        const int slot = tau & 3;
        const bool lv = tau >= 0 && tau < nt;
        const size_t lvl = (size_t)(lv ? tau : 0) * plane;
        const T* src = (MODE == M_CHEB0 ? A.b : A.x) + ((size_t)grp * N + lvl) * RW;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int e = tid + 256 * k;
            if (KP * 256 > PP && e >= PP) break;
            const int gx = tx0 + p_dx[k], gy = ty0 + p_dy[k];
            const bool in = lv && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
            const int node = in ? gy * nx + gx : 0;
            cp_v4<T>(&S.p[slot][e], src + (size_t)node * RW, in);
            if (MODE == M_CHEB0)
                cp_scalar<T>(&S.dinvh[MODE == M_CHEB0 ? slot : 0][MODE == M_CHEB0 ? e : 0], A.dinv + lvl + node, in);
        }
    };
    // right-hand side, direction, diagonal and observation tables of level
    // tau into slot tau & 1
    auto stage_own = [&](int grp, const MUnit& u, int tau) {
        const int slot = tau & 1;
        const int gx = u.tx * MX + lx, gy = u.ty * MY + ly;
        const bool own = gx < nx && gy < ny;
        const size_t node = own ? (size_t)tau * plane + (size_t)gy * nx + gx : 0;
        const size_t off = ((size_t)grp * N + node) * RW;
        if (MODE != M_APPLY) cp_v4<T>(&S.b[MODE != M_APPLY ? slot : 0][tid], A.b + off, own);
        if (MODE == M_CHEB && A.d != nullptr) cp_v4<T>(&S.d[MODE == M_CHEB ? slot : 0][tid], A.d + off, own);
        if (MODE == M_CHEB) cp_scalar<T>(&S.dinv[MODE == M_CHEB ? slot : 0][tid], A.dinv + node, own);
        if (obs_staged) {
            const int tile = (tau * tiles_y + u.ty) * tiles_x + u.tx;
            unsigned char* dst = obs_smem + (size_t)slot * ostage;
            const unsigned char* gmap = reinterpret_cast<const unsigned char*>(L.omap + (size_t)tile * 256);
            const unsigned char* gent = reinterpret_cast<const unsigned char*>(L.oent) + (size_t)tile * L.ostride;
            for (int c = tid; c < 256 * 2 / 16; c += 256) cp_async16(dst + c * 16, gmap + c * 16, true);
            for (int c = tid; c < L.ostride / 16; c += 256) cp_async16(dst + 256 * 2 + c * 16, gent + c * 16, true);
        }
    };
    // CHEB0: staged b -> x1 = c0 D^-1 b in place (after the plane landed)
    auto scale_plane = [&](int tau) {
        if (MODE != M_CHEB0) return;
        const int slot = tau & 3;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int e = tid + 256 * k;
            if (KP * 256 > PP && e >= PP) break;
            S.p[slot][e] = (A.c0 * S.dinvh[MODE == M_CHEB0 ? slot : 0][MODE == M_CHEB0 ? e : 0]) * S.p[slot][e];
        }
    };
    // s = B p on level tau (tile plus ring) into slot tau & 1
    auto spass = [&](int tx0, int ty0, int tau) {
        const V4<T>* pc = S.p[tau & 3];
        const V4<T>* pm = S.p[(tau - 1) & 3];
        V4<T>* sd = S.s[tau & 1];
        const bool first = nt > 1 && tau == 0;
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int e = tid + 256 * k;
            if (KS * 256 > SP && e >= SP) break;
            const int rx = tx0 + s_dx[k], ry = ty0 + s_dy[k];
            const bool inrow = rx >= 0 && rx < nx && ry >= 0 && ry < ny && tau < nt;
            const int base = s_base[k];
            V4<T> sv = v4zero<T>();
            if (inrow && !is_dirichlet(rx, ry, nx, ny)) {
                const bool xl = rx == 1, xr = rx == nx - 2, yl = ry == 1, yr = ry == ny - 2;
#pragma unroll
                for (int o = 0; o < NTAP; ++o) {
                    const T c = first ? c1[o] : c0[o];
                    if (c == T(0)) continue;
                    if (o == 7) { sv = fma4(c, pm[base], sv); continue; }
                    const bool hit = (tap_dx(o) < 0 && xl) || (tap_dx(o) > 0 && xr) || (tap_dy(o) < 0 && yl) ||
                                     (tap_dy(o) > 0 && yr);
                    if (hit) continue;
                    sv = fma4(c, pc[base + tap_dy(o) * PX + tap_dx(o)], sv);
                }
            }
            sd[e] = sv;
        }
    };

    T dacc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 1
    for (long long u = blockIdx.x; u < nunits; u += G) {
        const MUnit cur = unit_at(u);
        const int grp = cur.grp;
        const int tx0 = cur.tx * MX, ty0 = cur.ty * MY;
        const int ta = cur.chunk * tc, tb = min(ta + tc, nt);
        // prologue: planes ta - 1, ta (s_ta) and ta + 1 with level ta's own data
        __syncthreads();                       // the previous unit's reads are done
        stage_p(grp, tx0, ty0, ta - 1);
        cp_commit();
        stage_p(grp, tx0, ty0, ta);
        cp_commit();
        stage_p(grp, tx0, ty0, ta + 1);
        stage_own(grp, cur, ta);
        cp_commit();
        cp_wait<1>();
        __syncthreads();
        if (MODE == M_CHEB0) {
            scale_plane(ta - 1);
            scale_plane(ta);
            __syncthreads();
        }
        spass(tx0, ty0, ta);
#pragma unroll 1
        for (int t = ta; t < tb; ++t) {
            cp_wait<0>();                      // plane t + 1 and level t's own data landed
            __syncthreads();
            if (t + 2 <= tb) stage_p(grp, tx0, ty0, t + 2);
            if (t + 1 < tb) stage_own(grp, cur, t + 1);
            cp_commit();
            if (MODE == M_CHEB0) {
                scale_plane(t + 1);
                __syncthreads();
            }
            spass(tx0, ty0, t + 1);
            // observation tables of level t
            const int16_t* omap_t = nullptr;
            const unsigned char* oent_t = nullptr;
            if (has_obs) {
                if (obs_staged) {
                    omap_t = reinterpret_cast<const int16_t*>(obs_smem + (size_t)(t & 1) * ostage);
                    oent_t = obs_smem + (size_t)(t & 1) * ostage + 256 * 2;
                } else {
                    const int tile = (t * tiles_y + cur.ty) * tiles_x + cur.tx;
                    omap_t = L.omap + (size_t)tile * 256;
                    oent_t = reinterpret_cast<const unsigned char*>(L.oent) + (size_t)tile * L.ostride;
                }
            }
            const int oe = 255 - tid;          // entries on the last warps
            if (has_obs && oe < L.ocap) {
                const int nd = reinterpret_cast<const int16_t*>(oent_t + (size_t)L.ocap * OC * sizeof(T))[oe];
                if (nd >= 0) {
                    const int pb = (nd / MX + 2) * PX + (nd % MX + 2);
                    const T* c = reinterpret_cast<const T*>(oent_t) + oe * OC;
                    V4<T> v = v4zero<T>();
#pragma unroll
                    for (int a = 0; a < OC; ++a)
                        v = fma4(c[a], S.p[(t + obs_dt(GEO_XYT, a)) & 3][pb + obs_dy(GEO_XYT, a) * PX + obs_dx(GEO_XYT, a)], v);
                    S.qobs[nd] = v;
                }
            }
            __syncthreads();
            // q_t = B^T s (+ A^T R^-1 A p) at the thread's node
            const int gx = tx0 + lx, gy = ty0 + ly;
            const bool own = gx < nx && gy < ny;
            const V4<T> pv = S.p[t & 3][pown];
            V4<T> q = v4zero<T>();
            if (own) {
                if (is_dirichlet(gx, gy, nx, ny)) {
                    q = L.inv_eps2 * pv;
                } else {
                    const V4<T>* sc = S.s[t & 1];
                    const bool first = nt > 1 && t == 0;
#pragma unroll
                    for (int o = 0; o < 7; ++o) {
                        const T c = first ? c1[o] : c0[o];
                        if (c == T(0)) continue;
                        q = fma4(c, sc[sown - (tap_dy(o) * SX + tap_dx(o))], q);
                    }
                    if (c0[7] != T(0)) q = fma4(c0[7], S.s[(t + 1) & 1][sown], q);
                }
                if (has_obs && omap_t[tid] >= 0) q = q + S.qobs[tid];
                const size_t node = (size_t)t * plane + (size_t)gy * nx + gx;
                const size_t off = ((size_t)grp * N + node) * RW;
                if (MODE == M_APPLY) {
                    v4store(A.out + off, q);
                    dacc[0] += pv.a * q.a; dacc[1] += pv.b * q.b; dacc[2] += pv.c * q.c; dacc[3] += pv.d * q.d;
                } else if (MODE == M_RESID) {
                    const V4<T> r = S.b[MODE != M_APPLY ? (t & 1) : 0][tid] - q;
                    v4store(A.out + off, r);
                    const T w = A.rweight != nullptr ? A.rweight[node] : T(1);
                    dacc[0] += w * r.a * r.a; dacc[1] += w * r.b * r.b; dacc[2] += w * r.c * r.c; dacc[3] += w * r.d * r.d;
                } else {
                    const V4<T> bb = S.b[MODE != M_APPLY ? (t & 1) : 0][tid];
                    const V4<T> r = bb - q;
                    const T di = MODE == M_CHEB0 ? S.dinvh[MODE == M_CHEB0 ? (t & 3) : 0][MODE == M_CHEB0 ? pown : 0]
                                                 : S.dinv[MODE == M_CHEB ? (t & 1) : 0][tid];
                    V4<T> dn = (A.c2 * di) * r;
                    if (MODE == M_CHEB0) dn = fma4(A.c1, pv, dn);
                    else if (A.d != nullptr) dn = fma4(A.c1, S.d[MODE == M_CHEB ? (t & 1) : 0][tid], dn);
                    const V4<T> xn = pv + dn;
                    v4store(A.out + off, xn);
                    v4store(A.out2 + off, dn);
                    dacc[0] += bb.a * xn.a; dacc[1] += bb.b * xn.b; dacc[2] += bb.c * xn.c; dacc[3] += bb.d * xn.d;
                }
            }
        }
        // dot partials of this unit's block: add to the CTA's entry
        if (A.partial != nullptr) {
            double* dst = A.partial + ((size_t)grp * G + blockIdx.x) * 4;
            __shared__ double prev[4];
            if (tid < 4) prev[tid] = dst[tid];       // this CTA's running sum for the block
            block_sum4<256, T>(dacc, dst);
            if (tid < 4) dst[tid] += prev[tid];
            dacc[0] = dacc[1] = dacc[2] = dacc[3] = T(0);
        }
    }
    cp_wait<0>();
}

// Largest persistent grid (the dot-partial buffers are sized for it).
constexpr int kMaxMarchGrid = 4096;

template <typename T, int MODE>
int launch_march_mode(const StencilArgs<T>& a, cudaStream_t s) {
    using SM = MarchSmem<T, MODE>;
    auto kern = k_march<T, MODE>;
    static int sms = 0, optin = 0, attr = 0;
    static std::map<size_t, int> per_sm;
    static std::mutex mu;
    StencilArgs<T> args = a;
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
        const size_t staged = sizeof(SM) + 2 * (size_t)(256 * 2 + a.L.ostride);
        args.L.obs_direct = 0;
        if (a.L.ocap > 0) {
            if (staged + 1024 <= (size_t)optin) smem = staged;
            else args.L.obs_direct = 1;
        }
        if (smem + 1024 > (size_t)optin) throw std::runtime_error("space-time stencil does not fit in shared memory");
        if ((int)smem > attr) {
            ok(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr = (int)smem;
        }
        auto it = per_sm.find(smem);
        if (it == per_sm.end()) {
            int per = 0;
            ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, smem));
            if (per <= 0) throw std::runtime_error("space-time stencil does not fit on an SM");
            it = per_sm.emplace(smem, per).first;
        }
        resident = sms * it->second;
    }
    if (a.L.col.kind != 0) throw std::runtime_error("space-time stencil: collocation rows are 1D space only");
    // split time into chunks when tiles x blocks alone do not fill the grid twice
    const long long tiles = (long long)a.L.tiles_x * a.L.tiles_y;
    const long long base = tiles * a.nblk;
    const int nt = a.L.nt;
    int nchunks = (int)std::min<long long>(std::max<long long>(1, (2LL * resident + base - 1) / base), std::max(1, nt / 8));
    const int tc = (nt + nchunks - 1) / nchunks;
    nchunks = (nt + tc - 1) / tc;
    const long long nunits = base * nchunks;
    const int grid = (int)std::min<long long>(std::min<long long>(nunits, resident), kMaxMarchGrid);
    { kern<<<(unsigned)grid, 256, smem, s>>>(args, (int)nunits, tc, nchunks); note_launch(); }
    return grid;
}

}  // namespace

template <typename T> int launch_march(int mode, const StencilArgs<T>& a, cudaStream_t s) {
    if (mode == M_APPLY) return launch_march_mode<T, M_APPLY>(a, s);
    if (mode == M_RESID) return launch_march_mode<T, M_RESID>(a, s);
    if (mode == M_CHEB0) return launch_march_mode<T, M_CHEB0>(a, s);
    return launch_march_mode<T, M_CHEB>(a, s);
}
template int launch_march<float>(int, const StencilArgs<float>&, cudaStream_t);
template int launch_march<double>(int, const StencilArgs<double>&, cudaStream_t);

}  // namespace gmrf
