// Device helpers shared by the GMRF kernels: the 4-wide right-hand-side
// vector type, tile geometries, Philox4x32-10 normals and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gmrf {

// Right-hand sides are stored in blocks of four: element (rhs r, node n) of a
// batch lives at ((r / 4) * N + n) * 4 + r % 4.  One thread owns one node of
// one block and moves 16 B (FP32) or 32 B (FP64) per access.
constexpr int RW = 4;

template <typename T> struct alignas(sizeof(T) * 4) V4 { T a, b, c, d; };

template <typename T> __device__ __forceinline__ V4<T> v4zero() { return V4<T>{T(0), T(0), T(0), T(0)}; }
template <typename T> __device__ __forceinline__ V4<T> v4load(const T* p) { return *reinterpret_cast<const V4<T>*>(p); }
template <typename T> __device__ __forceinline__ void v4store(T* p, V4<T> v) { *reinterpret_cast<V4<T>*>(p) = v; }
template <typename T> __device__ __forceinline__ V4<T> operator+(V4<T> x, V4<T> y) { return {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; }
template <typename T> __device__ __forceinline__ V4<T> operator-(V4<T> x, V4<T> y) { return {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; }
template <typename T> __device__ __forceinline__ V4<T> operator*(T s, V4<T> x) { return {s * x.a, s * x.b, s * x.c, s * x.d}; }
template <typename T> __device__ __forceinline__ V4<T> operator*(V4<T> x, V4<T> y) { return {x.a * y.a, x.b * y.b, x.c * y.c, x.d * y.d}; }
template <typename T> __device__ __forceinline__ V4<T> fma4(T s, V4<T> x, V4<T> acc) {
    return {fma(s, x.a, acc.a), fma(s, x.b, acc.b), fma(s, x.c, acc.c), fma(s, x.d, acc.d)};
}
// FP32: two packed f32x2 instructions per 4-wide operation (sm_100 and
// later); each lane rounds exactly like the scalar fma.rn / add.rn / mul.rn,
// so results are bit-identical to the generic form above while the FP32
// pipe issues half the instructions.
template <> __device__ __forceinline__ V4<float> fma4<float>(float s, V4<float> x, V4<float> acc) {
    V4<float> r;
    asm("{\n\t.reg .b64 s2, x0, x1, a0, a1, r0, r1;\n\t"
        "mov.b64 s2, {%8, %8};\n\t"
        "mov.b64 x0, {%9, %10};\n\tmov.b64 x1, {%11, %12};\n\t"
        "mov.b64 a0, {%4, %5};\n\tmov.b64 a1, {%6, %7};\n\t"
        "fma.rn.f32x2 r0, s2, x0, a0;\n\tfma.rn.f32x2 r1, s2, x1, a1;\n\t"
        "mov.b64 {%0, %1}, r0;\n\tmov.b64 {%2, %3}, r1;\n\t}"
        : "=f"(r.a), "=f"(r.b), "=f"(r.c), "=f"(r.d)
        : "f"(acc.a), "f"(acc.b), "f"(acc.c), "f"(acc.d), "f"(s), "f"(x.a), "f"(x.b), "f"(x.c), "f"(x.d));
    return r;
}
template <> __device__ __forceinline__ V4<float> operator*<float>(float s, V4<float> x) {
    V4<float> r;
    asm("{\n\t.reg .b64 s2, x0, x1, r0, r1;\n\t"
        "mov.b64 s2, {%4, %4};\n\t"
        "mov.b64 x0, {%5, %6};\n\tmov.b64 x1, {%7, %8};\n\t"
        "mul.rn.f32x2 r0, s2, x0;\n\tmul.rn.f32x2 r1, s2, x1;\n\t"
        "mov.b64 {%0, %1}, r0;\n\tmov.b64 {%2, %3}, r1;\n\t}"
        : "=f"(r.a), "=f"(r.b), "=f"(r.c), "=f"(r.d)
        : "f"(s), "f"(x.a), "f"(x.b), "f"(x.c), "f"(x.d));
    return r;
}
template <> __device__ __forceinline__ V4<float> operator+<float>(V4<float> x, V4<float> y) {
    V4<float> r;
    asm("{\n\t.reg .b64 x0, x1, y0, y1, r0, r1;\n\t"
        "mov.b64 x0, {%4, %5};\n\tmov.b64 x1, {%6, %7};\n\t"
        "mov.b64 y0, {%8, %9};\n\tmov.b64 y1, {%10, %11};\n\t"
        "add.rn.f32x2 r0, x0, y0;\n\tadd.rn.f32x2 r1, x1, y1;\n\t"
        "mov.b64 {%0, %1}, r0;\n\tmov.b64 {%2, %3}, r1;\n\t}"
        : "=f"(r.a), "=f"(r.b), "=f"(r.c), "=f"(r.d)
        : "f"(x.a), "f"(x.b), "f"(x.c), "f"(x.d), "f"(y.a), "f"(y.b), "f"(y.c), "f"(y.d));
    return r;
}
template <> __device__ __forceinline__ V4<float> operator-<float>(V4<float> x, V4<float> y) {
    V4<float> r;
    asm("{\n\t.reg .b64 x0, x1, y0, y1, r0, r1;\n\t"
        "mov.b64 x0, {%4, %5};\n\tmov.b64 x1, {%6, %7};\n\t"
        "mov.b64 y0, {%8, %9};\n\tmov.b64 y1, {%10, %11};\n\t"
        "sub.rn.f32x2 r0, x0, y0;\n\tsub.rn.f32x2 r1, x1, y1;\n\t"
        "mov.b64 {%0, %1}, r0;\n\tmov.b64 {%2, %3}, r1;\n\t}"
        : "=f"(r.a), "=f"(r.b), "=f"(r.c), "=f"(r.d)
        : "f"(x.a), "f"(x.b), "f"(x.c), "f"(x.d), "f"(y.a), "f"(y.b), "f"(y.c), "f"(y.d));
    return r;
}

template <typename T> __device__ __forceinline__ T comp(const V4<T>& v, int i) {
    return i == 0 ? v.a : (i == 1 ? v.b : (i == 2 ? v.c : v.d));
}

// Tile geometries.  GEO_XY: 2D space; GEO_XT: 1D space x time (the y axis is
// absent, ny = 1); GEO_XYT: 2D space x time.  A CTA of 256 threads owns one
// TX x TY x TT tile of nodes for one block of four right-hand sides.  The
// input vector is staged with a halo of 2 in x and y (the stacked stencil
// B^T B reaches two nodes) and 1 in t.  GEO_XYT tiles are single time levels
// of a 32 x 8 plane tile: its stencil kernel marches through time with
// rolling planes in shared memory, and the observation tables and tile lists
// are kept per plane tile.
enum Geometry { GEO_XY = 0, GEO_XT = 1, GEO_XYT = 2 };

template <int GEO> struct Geo;
template <> struct Geo<GEO_XY>  { static constexpr int TX = 32, TY = 8, TT = 1, HY = 2, HT = 0; };
template <> struct Geo<GEO_XT>  { static constexpr int TX = 32, TY = 1, TT = 8, HY = 0, HT = 1; };
template <> struct Geo<GEO_XYT> { static constexpr int TX = 32, TY = 8, TT = 1, HY = 2, HT = 1; };

// Offsets of the observation stencil A^T R^-1 A: all (dx, dy, dt) in
// {-1, 0, 1} over the axes the geometry has (9 points in 2D, 27 in 3D).
template <int GEO> struct ObsStencil;
template <> struct ObsStencil<GEO_XY>  { static constexpr int OC = 9; };
template <> struct ObsStencil<GEO_XT>  { static constexpr int OC = 9; };
template <> struct ObsStencil<GEO_XYT> { static constexpr int OC = 27; };
__host__ __device__ constexpr int obs_dx(int, int a) { return a % 3 - 1; }
__host__ __device__ constexpr int obs_dy(int geo, int a) { return geo == GEO_XT ? 0 : (a / 3) % 3 - 1; }
__host__ __device__ constexpr int obs_dt(int geo, int a) { return geo == GEO_XY ? 0 : (geo == GEO_XT ? a / 3 - 1 : a / 9 - 1); }
inline int obs_oc(int g) { return g == GEO_XYT ? 27 : 9; }

inline int geo_tx(int) { return 32; }
inline int geo_ty(int g) { return g == GEO_XT ? 1 : 8; }
inline int geo_tt(int g) { return g == GEO_XT ? 8 : 1; }

// Stencil taps of the root B (dx, dy, dt): 0 centre, 1 x-1, 2 x+1, 3 y-1,
// 4 y+1, 5 (x-1, y-1), 6 (x+1, y+1), 7 t-1.
constexpr int NTAP = 8;
__host__ __device__ constexpr int tap_dx(int o) { return o == 1 || o == 5 ? -1 : (o == 2 || o == 6 ? 1 : 0); }
__host__ __device__ constexpr int tap_dy(int o) { return o == 3 || o == 5 ? -1 : (o == 4 || o == 6 ? 1 : 0); }
__host__ __device__ constexpr int tap_dt(int o) { return o == 7 ? -1 : 0; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products
// with a Weyl-sequence key schedule.

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Uniform in (0, 1]: RN(k + 1/2) 2^-53 with k the 53-bit integer
// (a >> 5) 2^26 + (b >> 6).  Formed with integer operations and one exact
// integer-to-double conversion: below 2^52, k + 1/2 is exact; from 2^52 on it
// is a tie that rounds to the even neighbour of k; w = 2 RN(k + 1/2) is an
// exact integer and the result is w 2^-54 (exponent lowered by 54).
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
    const unsigned long long k = ((unsigned long long)(a >> 5) << 26) | (unsigned long long)(b >> 6);
    const unsigned long long w = k < (1ull << 52) ? 2 * k + 1 : 2 * k + 2 * (k & 1);
    const long long bits = __double_as_longlong((double)w) - (54ll << 52);
    return __longlong_as_double(bits);
}

__device__ __forceinline__ double philox_rademacher(uint64_t seed, uint32_t sample, uint64_t idx) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(idx >> 2), sample, 2u, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const uint32_t word = (idx & 3) == 0 ? w.x : ((idx & 3) == 1 ? w.y : ((idx & 3) == 2 ? w.z : w.w));
    return (word & 1u) ? -1.0 : 1.0;
}

// ---------------------------------------------------------------------------
// Block reduction of four partial sums (one per right-hand side of the
// block) over a 256-thread CTA; threads 0..3 write the totals as FP64.
// Every thread of the CTA must call it.  Each thread's own partial stays in
// the kernel's precision (an FP32 kernel sums a few dozen FP32 terms per
// thread: the FP64 pipe of GB300 is too narrow for one FP64 add per node);
// everything above it -- the warp shuffles, the sum over warps and the sum
// over CTAs -- runs in FP64.

template <typename A> __device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int NT, typename A>
__device__ __forceinline__ void block_sum4(A v[4], double* out /* 4 doubles, global */) {
    __shared__ double red[NT / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = warp_sum((double)v[i]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) red[warp][i] = w[i];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) s += red[k][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();   // the scratch may be reused by the next call
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async; a false predicate copies
// zero bytes and zero-fills the destination) and the Dirichlet test of the
// space boundary (App. B).

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gmem), "r"(pred ? 16 : 0));
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, bool pred) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(gmem), "r"(pred ? 4 : 0));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool pred) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gmem), "r"(pred ? 8 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename T> __device__ __forceinline__ void cp_v4(V4<T>* smem, const T* gmem, bool pred) {
    cp_async16(smem, gmem, pred);
    if (sizeof(T) == 8) cp_async16(reinterpret_cast<char*>(smem) + 16, reinterpret_cast<const char*>(gmem) + 16, pred);
}
template <typename T> __device__ __forceinline__ void cp_scalar(T* smem, const T* gmem, bool pred) {
    if (sizeof(T) == 8) cp_async8(smem, gmem, pred);
    else cp_async4(smem, gmem, pred);
}

// Tensor-memory-accelerator (TMA) loads completing on an mbarrier.  A load
// whose box leaves the tensor zero-fills the outside part; its innermost
// start coordinate times the element size must be a multiple of 16 bytes and
// the shared-memory destination 128-byte aligned.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
                 ::"r"(smem_u32(dst)), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)) : "memory");
}
// Bounded wait for the completion of phase `parity` of a barrier: false when
// it did not come within `cap` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int cap) {
    for (int i = 0; i < cap; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Before a CTA that gave up on a wait returns: wait (bounded again) for the
// copies still in flight on the barriers whose bits are set in `pending`, so
// that no bulk copy writes shared memory after the CTA ended.
__device__ __forceinline__ void mbar_drain(uint64_t* bars, int nbars, unsigned pending, unsigned phbits, int cap) {
    for (int i = 0; i < nbars; ++i)
        if ((pending >> i) & 1u) mbar_wait_bounded(&bars[i], (phbits >> i) & 1u, cap);
}
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, int c0, int c1, int c2, int c3, uint64_t* bar) {
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];\n"
                 ::"r"(smem_u32(dst)), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar)) : "memory");
}
// orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses to the same buffers
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ bool is_dirichlet(int x, int y, int nx, int ny) {
    return x == 0 || x == nx - 1 || (ny > 1 && (y == 0 || y == ny - 1));
}

// index on a torus axis of n nodes, for offsets within one period
__host__ __device__ __forceinline__ int wrap_idx(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

}  // namespace gmrf
