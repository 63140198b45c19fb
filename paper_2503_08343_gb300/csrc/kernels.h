// Host-callable launchers of the GMRF kernels (stencil.cu, stencil_march.cu,
// resid_df.cu and kernels.cu).
#pragma once

#include <cuda.h>

#include "impl.h"

namespace gmrf {

void note_launch();
void capture_begin();
unsigned long long capture_end();
void note_graph_launch(unsigned long long kernels);
unsigned long long launch_count();

// CHEB0: the first two Chebyshev steps from x = 0 in one pass; x1 = c0 D^-1 b
// is formed in shared memory from the staged b, then one CHEB step with d = x1
enum StencilMode { M_APPLY = 0, M_RESID = 1, M_CHEB = 2, M_CHEB0 = 3, M_PCG = 4 };

template <typename T>
struct StencilArgs {
    LevelView<T> L;
    const T* x;        // input vector, staged with halo
    const T* b;        // RESID / CHEB right-hand side
    const T* d;        // CHEB previous direction (null on the first step)
    const T* dinv;     // CHEB inverse diagonal [N]
    T* out;            // APPLY: Q x; RESID: b - Q x; CHEB: x + d_new
    T* out2;           // CHEB: d_new
    T c1, c2;          // CHEB: d_new = c1 d + c2 D^-1 (b - Q x)
    T c0;              // CHEB0: x = c0 D^-1 b before the step (x is not read)
    double* partial;   // per-CTA dot partials [nblk][grid][4] or null
    int nblk;
    const T* rweight;  // RESID: if set, the dot is sum r^2 * rweight[node] (D^-1-weighted norm)
    // PCG (one conjugate-gradient iteration's vector work around the apply):
    // x = previous direction p (staged with halo), d = preconditioned
    // residual z (staged with halo), b = iterate (own nodes); per right-hand
    // side alpha, beta ([nblk][4]);  p' = z + beta p, out = Q p', out2 = p',
    // out3 = b + alpha p (the iterate's update of the previous iteration)
    T* out3;
    const double* alpha;
    const double* beta;
};

// Dot partials written to `partial` as [nblk][grid][4] (APPLY x.Qx, RESID
// |r|^2, CHEB b.x_new); returns the grid size, i.e. the partial count per block.
template <typename T> int launch_stencil(int geo, int mode, const StencilArgs<T>& a, cudaStream_t s);
// the pointers a mode reads and writes are all set (host check before every
// launch; throws std::runtime_error naming the missing one)
template <typename T> void stencil_check_args(int mode, int col, const StencilArgs<T>& a);
// 2D space x time: the 2.5D-blocked kernel of stencil_march.cu (called by launch_stencil)
template <typename T> int launch_march(int mode, const StencilArgs<T>& a, cudaStream_t s);
int stencil_max_grid();
int march_max_grid();
// One-time set-up of the stencil instantiation that launch_stencil would use
// for (geo, mode, a): function attributes and occupancy, which also load the
// kernel's code on the current device.  Launches nothing.
template <typename T> void stencil_prepare(int geo, int mode, const StencilArgs<T>& a);
template <typename T> void march_prepare(int mode, const StencilArgs<T>& a);
// loads the code of the partial-sum reduction kernel on the current device
void reduce_prepare();
// 1 if a stencil CTA gave up waiting for a staged input tile since the last
// call (the flags of both stencil kernels are cleared)
int stencil_abort_take(cudaStream_t s);
int march_abort_take(cudaStream_t s);
// queue copies of both abort flags into host memory (2 ints, pinned) on s;
// valid after the next synchronisation of s
void stencil_abort_peek_async(int32_t* host2, cudaStream_t s);
void march_abort_peek_async(int32_t* host1, cudaStream_t s);
// test hook: poll cap of the staged-tile waits of both stencil kernels
// (0: the default 2^22; negative: give up without polling), a device variable
// read by every CTA (so captured graphs follow it); the drain of in-flight
// copies keeps the default
void set_wait_cap(int cap);
void march_set_wait_cap(int cap);
// cuTensorMapEncodeTiled of a dense FP32 (f64 = false) or FP64 array of
// `rank` dimensions (innermost first; strides of dimensions 1.. in bytes),
// no interleave or swizzle, zero fill outside; throws on an error.
void encode_tensor_map(CUtensorMap* m, bool f64, int rank, const void* base, const cuuint64_t* dims,
                       const cuuint64_t* strides, const cuuint32_t* box);

// reduce [nblk][nparts][4] partials into out[nblk * 4]
void launch_reduce(const double* partial, int nparts, int nblk, double* out, cudaStream_t s);

// elementwise vector kernels over blocked batches ([nblk][N][4])
template <typename T> void launch_cheb_first(const T* b, const T* dinv, T c2, T* x, T* d, long long N, int nblk, cudaStream_t s);
template <typename T> void launch_restrict_axis(const T* in, T* out, int nx, int ny, int nt, int axis, int ncoarse,
                                                const int32_t* rs, const int32_t* rc, const int32_t* pj, const T* pw,
                                                int nblk, cudaStream_t s);
template <typename T> void launch_restrict_xy(const T* in, T* out, int nx, int ny, int nt, int cx, int cy,
                                              const int32_t* const rs[2], const int32_t* const rc[2],
                                              const int32_t* const pj[2], const T* const pw[2], bool p1,
                                              const int span[2], int nblk, cudaStream_t s);
template <typename T> void launch_prolong_add(T* xf, const T* xc, const Level& f, const Level& c, bool p1, int nblk, cudaStream_t s);
// restriction between periodic (torus) levels, the transpose of launch_prolong_add
template <typename T> void launch_restrict_torus(const T* in, T* out, const Level& f, const Level& c, bool p1, int nblk, cudaStream_t s);
template <typename T> void launch_dense_solve(const T* Ainv, const T* b, T* x, int n, int nblk, cudaStream_t s);

// PCG scalar and vector steps.  Per-RHS scalars live in `sc` (FP64):
//   sc[0*P + r] = rz, sc[1*P + r] = pq, sc[2*P + r] = alpha, sc[3*P + r] = beta,
//   sc[4*P + r] = rr, sc[5*P + r] = rr0, sc[6*P + r] = active (0/1), sc[7*P + r] = breakdown
// with P = nblk * 4.
// r -= alpha q; then, after z = M r and beta: x += alpha p, p = z + beta p
template <typename T> void launch_pcg_update_r(T* r, const T* q, const double* sc, long long N, int nblk, cudaStream_t s);
template <typename T> void launch_pcg_update_xp(T* x, T* p, const T* z, const double* sc, long long N, int nblk,
                                                cudaStream_t s);
// x += alpha p (the last iterate update after fused iterations)
template <typename T> void launch_pcg_update_x(T* x, const T* p, const double* sc, long long N, int nblk, cudaStream_t s);
void launch_pcg_scalar(int kind, const double* red, double* sc, int nblk, double tol2, cudaStream_t s);
// launch_reduce into `red` followed by launch_pcg_scalar on it, as one kernel
void launch_reduce_scalar(int kind, const double* partial, int nparts, int nblk, double* red, double* sc, double tol2,
                          cudaStream_t s);
constexpr int EPT = 4;                  // nodes per thread in elementwise kernels
constexpr int ECHUNK = 256 * EPT;       // nodes per CTA
int elem_parts(long long N);

// Refinement residual r = b - Q x in double-float arithmetic (resid_df.cu),
// for 2D and 1D space-time levels without collocation rows: r is stored as
// float pairs (hi, lo) in the FP64 slots of `out`; the partials hold the
// rweight-weighted |r|^2 ([nblk][grid][4]); returns the grid size.
bool resid_df_applicable(const Level& L);
int launch_resid_df(const Level& L, const double* x, const double* b, double* out, const double* rweight,
                    double* partial, int nblk, cudaStream_t s);
// |r|^2 per right-hand side of a pair-stored residual, and r / norm as FP32
void launch_norm2_df(const double* r, long long N, int nblk, double* partial, int nparts, cudaStream_t s);
void launch_scale_cast_df(const double* r, const double* norms, float* r32, long long N, int nblk, cudaStream_t s);

// mixed precision refinement
void launch_scale_cast(const double* r64, const double* norms, float* r32, long long N, int nblk, cudaStream_t s);
void launch_axpy_mixed(double* x64, const double* norms, const float* d32, long long N, int nblk, double* partial, cudaStream_t s);
void launch_axpy_scaled64(double* x64, const double* norms, const double* d64, long long N, int nblk, double* partial, cudaStream_t s);
void launch_scale64(const double* r64, const double* norms, double* out, long long N, int nblk, cudaStream_t s);

// right-hand sides, layout conversion, variances
// b64 slots: sample RHS, data RHS or zero by slot id; z1 ([nblk][N][4] FP64
// scratch) receives the prior-row normals and z2 ([nblk][rows][4]) those of
// the observation rows (point, initial-condition and collocation rows,
// numbered as in the posterior); both NULL when no slot draws a sample
void launch_sample_rhs(int geo, const LevelView<double>& L, uint64_t seed, const int32_t* slot_sample,
                       const double* bdata, double* b64, double* z1, double* z2, long long rows, int nblk,
                       cudaStream_t s);
// data right-hand side A^T R^-1 y of the point rows (row index < nrows_y),
// added into b; deterministic per-tile gather
void launch_obs_data_rhs(const Level& L, int nrows_y, const double* y, double* b, cudaStream_t s);
void launch_pack(const double* src, double* dst, const int32_t* slot_src, long long N, int nblk, cudaStream_t s);
void launch_unpack(const double* src, double* dst, const int32_t* slot_dst, long long N, int nblk, cudaStream_t s);
template <typename QT>
void launch_rbmc(const QT* Qx, const double* x, const double* diag, const int32_t* slot_sample, long long N,
                 int nblk, int ns, double* var, double* se, cudaStream_t s);
template <typename T> void launch_diag(int geo, const LevelView<T>& L, double* diag64, cudaStream_t s);
// observation part of the diagonal, added into diag; deterministic per-tile gather
void launch_obs_diag(const Level& L, double* diag, cudaStream_t s);
void launch_max_share(const double* prior, const double* total, long long N, unsigned long long* out, cudaStream_t s);
void launch_finish_diag(const double* diag, float* dinv32, double* dinv64, long long N, cudaStream_t s);
void launch_normals(uint64_t seed, int stream, int sample0, int count, long long n, double* out, cudaStream_t s);
template <typename T> void launch_cast(const double* in, T* out, long long n, cudaStream_t s);
template <typename T> void launch_widen(const T* in, double* out, long long n, cudaStream_t s);
void launch_rademacher_fill(uint64_t seed, const int32_t* slot_sample, double* b64, long long N, int nblk, cudaStream_t s);
void launch_dot_blocked(const double* a, const double* b, long long N, int nblk, double* partial, int nparts, cudaStream_t s);

}  // namespace gmrf

namespace gmrf {
template <typename T> void launch_dot(const T* a, const T* b, long long N, int nblk, double* partial, int nparts, cudaStream_t s);
void launch_norm2w(const double* v, const double* w, long long N, int nblk, double* partial, int nparts, cudaStream_t s);
template <typename T> void launch_norm2(const T* v, long long N, int nblk, double* partial, int nparts, cudaStream_t s);
void launch_power_scale(float* q, const float* dinv, long long N, double* partial, int nparts, cudaStream_t s);
void launch_scale_comp(float* v, const float* w, const double* nrm2, long long N, cudaStream_t s);
void launch_fill_random(float* v, long long N, uint64_t seed, cudaStream_t s, const float* dinv = nullptr);
}  // namespace gmrf
