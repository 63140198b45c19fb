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

#include <cstring>

#include <cuda.h>

#include "autotune.h"
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

// TMA destinations (input planes, own b and d) first, each stage buffer on a
// 128-byte boundary.
template <typename T, int MODE> struct alignas(128) MarchSmem {
    V4<T> p[4][PP];
    V4<T> b[MODE != M_APPLY ? 2 : 1][256];
    V4<T> d[MODE == M_CHEB ? 2 : 1][256];
    V4<T> s[2][SP];
    T dinv[MODE == M_CHEB ? 2 : 1][256];
    T dinvh[MODE == M_CHEB0 ? 4 : 1][MODE == M_CHEB0 ? PP : 1];
    V4<T> qobs[256];
    static_assert((PP * sizeof(V4<T>)) % 128 == 0 && (256 * sizeof(V4<T>)) % 128 == 0, "128-byte stage buffers");
};

// Tensor maps of a blocked space-time vector seen as (4 nx values, ny, nt,
// blocks): the input plane with its halo, and the own plane tile.
struct MarchMaps {
    CUtensorMap p, b, d;
};

__device__ int g_march_abort = 0;
constexpr int kSpinCap = 1 << 22;
// polls before a staged-plane wait gives up (0: kSpinCap; negative: give up
// without polling); a test hook
__device__ int g_march_wait_cap = 0;

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
__global__ void __launch_bounds__(256) k_march(const StencilArgs<T> A, int nunits, int tc, int nchunks,
                                                const __grid_constant__ MarchMaps maps) {
    using SM = MarchSmem<T, MODE>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem_base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    SM& S = *reinterpret_cast<SM*>(smem_base);
    __shared__ uint64_t bars[4];               // one per input-plane slot
    __shared__ int aborted;
    const int cap = g_march_wait_cap > 0 ? g_march_wait_cap : (g_march_wait_cap < 0 ? 0 : kSpinCap);
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
    unsigned char* obs_smem = smem_base + sizeof(SM);
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
        mbar_fence_init();
        aborted = 0;
    }
    __syncthreads();
    unsigned phbits = 0;                       // parity of the next completion of each slot's barrier
    unsigned pend = 0;                         // slots with copies issued and not yet waited for (thread 0)

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

    // Input plane of level tau into slot tau & 3 (TMA, zero outside the grid),
    // with level tau - 1's own tiles of b and d when with_own; both complete
    // on the slot's barrier.  The per-node scalars (D^-1 for CHEB0 with halo,
    // D^-1 and the observation tables of level tau - 1) go by cp.async.
    auto stage = [&](int grp, const MUnit& u, int tau, bool with_own) {
        const int slot = tau & 3;
        const int tx0 = u.tx * MX, ty0 = u.ty * MY;
        if (tid == 0) {
            const bool with_b = with_own && MODE != M_APPLY;
            const bool with_d = with_own && MODE == M_CHEB && A.d != nullptr;
            const unsigned bytes = (unsigned)(PP * sizeof(V4<T>)) + (with_b ? 256u * (unsigned)sizeof(V4<T>) : 0u) +
                                   (with_d ? 256u * (unsigned)sizeof(V4<T>) : 0u);
            mbar_expect_tx(&bars[slot], bytes);
            pend |= 1u << slot;
            tma_load_4d(&S.p[slot][0], &maps.p, 4 * (tx0 - 2), ty0 - 2, tau, grp, &bars[slot]);
            if (with_b) tma_load_4d(&S.b[MODE != M_APPLY ? (tau - 1) & 1 : 0][0], &maps.b, 4 * tx0, ty0, tau - 1, grp, &bars[slot]);
            if (with_d) tma_load_4d(&S.d[MODE == M_CHEB ? (tau - 1) & 1 : 0][0], &maps.d, 4 * tx0, ty0, tau - 1, grp, &bars[slot]);
        }
        if (MODE == M_CHEB0) {
            const bool lv = tau >= 0 && tau < nt;
            const size_t lvl = (size_t)(lv ? tau : 0) * plane;
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const int e = tid + 256 * k;
                if (KP * 256 > PP && e >= PP) break;
                const int gx = tx0 + p_dx[k], gy = ty0 + p_dy[k];
                const bool in = lv && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
                cp_scalar<T>(&S.dinvh[MODE == M_CHEB0 ? slot : 0][MODE == M_CHEB0 ? e : 0], A.dinv + lvl + (in ? gy * nx + gx : 0), in);
            }
        }
        if (with_own) {
            const int lvo = tau - 1, oslot = lvo & 1;
            const int gx = tx0 + lx, gy = ty0 + ly;
            const bool own = gx < nx && gy < ny;
            if (MODE == M_CHEB)
                cp_scalar<T>(&S.dinv[MODE == M_CHEB ? oslot : 0][tid], A.dinv + (own ? (size_t)lvo * plane + (size_t)gy * nx + gx : 0), own);
            if (obs_staged) {
                const int tile = (lvo * tiles_y + u.ty) * tiles_x + u.tx;
                unsigned char* dst = obs_smem + (size_t)oslot * ostage;
                const unsigned char* gmap = reinterpret_cast<const unsigned char*>(L.omap + (size_t)tile * 256);
                const unsigned char* gent = reinterpret_cast<const unsigned char*>(L.oent) + (size_t)tile * L.ostride;
                for (int c = tid; c < 256 * 2 / 16; c += 256) cp_async16(dst + c * 16, gmap + c * 16, true);
                for (int c = tid; c < L.ostride / 16; c += 256) cp_async16(dst + 256 * 2 + c * 16, gent + c * 16, true);
            }
        }
    };
    // bounded wait for the plane of level tau (and what rides on its barrier)
    auto wait_plane = [&](int tau) {
        const int slot = tau & 3;
        if (mbar_wait_bounded(&bars[slot], (phbits >> slot) & 1u, cap)) {
            phbits ^= 1u << slot;
            pend &= ~(1u << slot);
        } else {
            aborted = 1;
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
        fence_proxy_async();                   // this thread's accesses of the last unit before the TMA refills
        __syncthreads();                       // the previous unit's reads are done
        stage(grp, cur, ta - 1, false);
        cp_commit();
        stage(grp, cur, ta, false);
        cp_commit();
        stage(grp, cur, ta + 1, true);
        cp_commit();
        cp_wait<1>();
        wait_plane(ta - 1);
        wait_plane(ta);
        __syncthreads();
        if (aborted) break;
        if (MODE == M_CHEB0) {
            scale_plane(ta - 1);
            scale_plane(ta);
            __syncthreads();
        }
        spass(tx0, ty0, ta);
#pragma unroll 1
        for (int t = ta; t < tb; ++t) {
            fence_proxy_async();
            cp_wait<0>();                      // plane t + 1 and level t's own data landed
            wait_plane(t + 1);
            __syncthreads();
            if (aborted) break;
            if (t + 2 <= tb) stage(grp, cur, t + 2, t + 1 < tb);
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
        if (aborted) break;
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
    if (tid == 0 && aborted) {
        mbar_drain(bars, 4, pend, phbits, kSpinCap);
        atomicExch(&g_march_abort, 1);
    }
}

// Tensor map of a blocked space-time vector [nblk][nt][ny][nx][4] as the 4D
// array (4 nx values, ny, nt, nblk); the box is one 32 x 8 plane tile, with
// the 2-node halo when `halo` (zero outside the grid and outside [0, nt)).
template <typename T>
CUtensorMap march_map(const T* v, const LevelView<T>& L, int nblk, bool halo) {
    const cuuint64_t dims[4] = {(cuuint64_t)4 * L.nx, (cuuint64_t)L.ny, (cuuint64_t)L.nt, (cuuint64_t)nblk};
    const cuuint64_t strides[3] = {(cuuint64_t)4 * L.nx * sizeof(T), (cuuint64_t)L.nx * L.ny * 4 * sizeof(T),
                                   (cuuint64_t)L.N * 4 * sizeof(T)};
    const cuuint32_t box[4] = {(cuuint32_t)(4 * (halo ? PX : MX)), (cuuint32_t)(halo ? PY : MY), 1, 1};
    CUtensorMap m;
    encode_tensor_map(&m, sizeof(T) == 8, 4, v, dims, strides, box);
    return m;
}

}  // namespace

void march_set_wait_cap(int cap) { ok(cudaMemcpyToSymbol(g_march_wait_cap, &cap, sizeof(int))); }

void march_abort_peek_async(int32_t* host1, cudaStream_t s) {
    ok(cudaMemcpyFromSymbolAsync(host1, g_march_abort, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
}

int march_abort_take(cudaStream_t s) {
    int v = 0;
    ok(cudaMemcpyFromSymbolAsync(&v, g_march_abort, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    ok(cudaStreamSynchronize(s));
    if (v) {
        static const int zero = 0;
        ok(cudaMemcpyToSymbolAsync(g_march_abort, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
        ok(cudaStreamSynchronize(s));
    }
    return v;
}

namespace {

// Largest persistent grid (the dot-partial buffers are sized for it).
constexpr int kMaxMarchGrid = 4096;

template <typename T, int MODE>
int launch_march_mode(const StencilArgs<T>& a, cudaStream_t s, bool dry = false) {
    using SM = MarchSmem<T, MODE>;
    auto kern = k_march<T, MODE>;
    static int sms = 0, optin = 0, attr = 0;
    static std::map<size_t, int> per_sm;
    static std::mutex mu;
    StencilArgs<T> args = a;
    size_t smem = sizeof(SM) + 128;            // + slack to put the stage buffers on 128 bytes
    int resident = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (sms == 0) {
            int dev = 0;
            ok(cudaGetDevice(&dev));
            ok(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            ok(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        }
        const size_t staged = smem + 2 * (size_t)(256 * 2 + a.L.ostride);
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
    if (dry) return 0;
    if (a.L.col.kind != 0) throw std::runtime_error("space-time stencil: collocation rows are 1D space only");
    // time is cut into chunks when tiles x blocks alone do not fill the grid:
    // about `mult` units per resident CTA, at least 8 time levels per chunk
    const long long tiles = (long long)a.L.tiles_x * a.L.tiles_y;
    const long long base = tiles * a.nblk;
    const int nt = a.L.nt;
    const int nsm = sms, per = resident / sms;
    struct Shape { int grid, tc, nchunks; long long nunits; };
    auto shape_of = [base, nt, nsm](int k, int mult) {
        const long long res = (long long)nsm * k;
        int nchunks = (int)std::min<long long>(std::max<long long>(1, (mult * res + base - 1) / base), std::max(1, nt / 8));
        const int tc = (nt + nchunks - 1) / nchunks;
        nchunks = (nt + tc - 1) / tc;
        const long long nunits = base * nchunks;
        return Shape{(int)std::min<long long>(std::min<long long>(nunits, res), kMaxMarchGrid), tc, nchunks, nunits};
    };
    auto run = [kern, smem](const StencilArgs<T>& aa, const Shape& sh, cudaStream_t st, bool count) {
        MarchMaps maps;
        std::memset(&maps, 0, sizeof(maps));
        maps.p = march_map<T>(MODE == M_CHEB0 ? aa.b : aa.x, aa.L, aa.nblk, true);
        if (MODE != M_APPLY) maps.b = march_map<T>(aa.b, aa.L, aa.nblk, false);
        if (MODE == M_CHEB && aa.d != nullptr) maps.d = march_map<T>(aa.d, aa.L, aa.nblk, false);
        kern<<<(unsigned)sh.grid, 256, smem, st>>>(aa, (int)sh.nunits, sh.tc, sh.nchunks, maps);
        if (count) note_launch();
    };
    Shape sh = shape_of(per, 2);
    // launch shape (CTAs per SM, units per resident CTA): measured once per key
    if (base * std::max(1, nt / 8) > nsm) {
        const TuneKey key{std::string("march<") + (sizeof(T) == 8 ? "f64," : "f32,") +
                              (MODE == M_APPLY ? "apply" : MODE == M_RESID ? "resid" : MODE == M_CHEB ? "cheb" : "cheb0") + ">",
                          args.nblk, tune_units_bucket(base * nt), tune_obs_bucket(args.L.ostride, args.L.ocap > 0)};
        auto measure = [key, args, per, shape_of, run](cudaStream_t st) {
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
            if (args.partial) t.partial = (double*)sc.zeros(sizeof(double) * 4 * args.nblk * kMaxMarchGrid, st);
            std::vector<TuneChoice> cands;
            std::vector<Shape> seen;
            for (int k = per; k >= 1; --k)
                for (int m : {2, 1, 4}) {
                    const Shape q = shape_of(k, m);
                    bool dup = false;
                    for (const Shape& o : seen) dup |= o.grid == q.grid && o.nchunks == q.nchunks;
                    if (dup) continue;
                    seen.push_back(q);
                    cands.push_back(TuneChoice{k, m});
                }
            return tune_measure(key, cands, [&](const TuneChoice& cc, cudaStream_t s2) { run(t, shape_of(cc.ctas_per_sm, cc.aux), s2, false); }, st);
        };
        TuneChoice c;
        if (tune_lookup(key, &c)) sh = shape_of(c.ctas_per_sm, c.aux);
        else if (tune_now(s)) { c = measure(s); sh = shape_of(c.ctas_per_sm, c.aux); }
        else tune_defer([measure](cudaStream_t st) { measure(st); });
    }
    run(args, sh, s, true);
    return sh.grid;
}

}  // namespace

template <typename T> int launch_march(int mode, const StencilArgs<T>& a, cudaStream_t s) {
    if (mode == M_PCG) throw std::runtime_error("space-time stencil: no fused conjugate-gradient mode");
    if (mode == M_APPLY) return launch_march_mode<T, M_APPLY>(a, s);
    if (mode == M_RESID) return launch_march_mode<T, M_RESID>(a, s);
    if (mode == M_CHEB0) return launch_march_mode<T, M_CHEB0>(a, s);
    return launch_march_mode<T, M_CHEB>(a, s);
}
template int launch_march<float>(int, const StencilArgs<float>&, cudaStream_t);
template int launch_march<double>(int, const StencilArgs<double>&, cudaStream_t);

template <typename T> void march_prepare(int mode, const StencilArgs<T>& a) {
    if (mode == M_PCG) throw std::runtime_error("space-time stencil: no fused conjugate-gradient mode");
    if (mode == M_APPLY) launch_march_mode<T, M_APPLY>(a, 0, true);
    else if (mode == M_RESID) launch_march_mode<T, M_RESID>(a, 0, true);
    else if (mode == M_CHEB0) launch_march_mode<T, M_CHEB0>(a, 0, true);
    else launch_march_mode<T, M_CHEB>(a, 0, true);
}
template void march_prepare<float>(int, const StencilArgs<float>&);
template void march_prepare<double>(int, const StencilArgs<double>&);
int march_max_grid() { return kMaxMarchGrid; }

}  // namespace gmrf
