// Host-side helpers shared by the setup, solver and C ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "kernels.h"

namespace gmrf {

// Errors inside the library are thrown as Error and turned into a status at
// the C boundary (nothing crosses extern "C" as an exception).
struct Error : std::runtime_error {
    gmrf_status status;
    Error(gmrf_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

inline void cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) throw Error(GMRF_E_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    throw Error(GMRF_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define GCK(call) ::gmrf::cuda_check((call), #call)

template <typename T> T* dev_alloc(size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    cuda_check(cudaMalloc(&p, n * sizeof(T)), "cudaMalloc");
    return static_cast<T*>(p);
}

template <typename T> void dev_upload(T** dst, const std::vector<T>& v) {
    if (*dst) cudaFree(*dst);
    *dst = dev_alloc<T>(v.size());
    if (!v.empty()) cuda_check(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
}

inline void dev_free(void* p) {
    if (p) cudaFree(p);
}

// setup.cu
int geometry_of(const gmrf_prior_desc& d);
void level_coefficients(const gmrf_prior_desc& d, Level& L);
void build_hierarchy(const gmrf_prior_desc& d, std::vector<Level>& levels);
void build_level_obs(const gmrf_prior_desc& d, const Posterior& P, const std::vector<double>& coords,
                     const std::vector<double>& rinv, Level& L, bool fine);
void build_transfer(Level& f, const Level& c);
void build_obs_stencil(Level& L);
std::vector<double> dense_operator(const Level& L, const double* mu);
bool spd_inverse(std::vector<double>& A, int n);

// solver.cu
struct SolveStats {
    int refinements = 0;
    int inner = 0;
    bool converged = false;
    double max_rel = 0.0;
    bool breakdown = false;
};

void level_free(Level& L);
void posterior_setup_levels(Posterior& P, cudaStream_t s);     // diag, Chebyshev bounds, transfers, dense inverse
void posterior_refresh_operator(Posterior& P, cudaStream_t s); // after the linearisation point changed
// Solve Q_u|y X = B for a blocked FP64 batch b64 (nblk blocks) into x64;
// x64 holds the starting guess (x_zero: it is zero, so r = b needs no apply).
SolveStats solve_blocked(Posterior& P, int nblk, const double* b64, double* x64, const gmrf_solve_opts& o,
                         cudaStream_t s, bool x_zero = false);
void apply64(Posterior& P, int nblk, const double* x64, double* y64, cudaStream_t s);
// the device-driven solve (one CUDA graph per batch size with the refinement
// and PCG loops as conditional while nodes): usable for the batched FP32
// refinement path without a wall-clock limit; launch enqueues it without
// waiting, collect reads its statistics once the stream has finished
bool device_loop_usable(const gmrf_solve_opts& o);
void solve_graph_launch(Posterior& P, int nblk, const double* b64, double* x64, const gmrf_solve_opts& o, cudaStream_t s);
SolveStats solve_graph_collect(Posterior& P, int nblk, cudaStream_t s);
Workspace& workspace(Posterior& P, int nblk);
void solve_graph_free(SolveGraph* g);
void workspace_free(Workspace* w);
double time_stencil(Posterior& P, int mode, int nblk, int iters, cudaStream_t s);
// One launch of the fused stencil on `level` in FP32 (prec 0) or FP64 (1):
// device FP64 [k][N_level] inputs x (unused by mode 3), b (modes 1-3),
// d (mode 2, may be null) and outputs out, out2 (modes 2-3); dots[k] (host)
// receives the kernel's per-RHS dot products.
// stencil_step mode that applies the solve's preconditioner (level 0)
constexpr int kStepPrecond = 5;
void stencil_step(Posterior& P, int level, int prec, int mode, int k, const double* x, const double* b, const double* d,
                  double c0, double c1, double c2, double* out, double* out2, double* out3, double* dots, cudaStream_t s);

// noalloc.cu: loads what gmrf_apply_posterior_noalloc uses for this posterior
void noalloc_prepare(const Posterior& P);

// tsp.cu
bool tsp_applicable(const Level& L, int nic);
bool tsp_mixed_weights(const Level& L);
// the inner PCG of this posterior's solves must run in FP64 (see tsp_mixed_weights)
bool inner_needs_fp64(const Posterior& P);
// o with its automatic fields resolved for P (max_inner <= 0: 60 with the
// multigrid preconditioner, 200 with the time-stepping one; FP64 inner solve
// where inner_needs_fp64)
gmrf_solve_opts solve_opts_for(const Posterior& P, const gmrf_solve_opts& o);
// the application kernel's shared memory fits for precision T
template <typename T> bool tsp_fits(const Level& L);
void tsp_prepare(Level& L, int nic, cudaStream_t s);
template <typename T>
void launch_tsp(const Level& L, double w_ic, double w_bnd, const T* r, T* y, T* z, int nblk, cudaStream_t s);

// gn.cu
struct GnResult {
    SolveStats stats;
    double decrement = 0.0;
    double alpha = 0.0;
};
void linearise(Posterior& P, const double* u, cudaStream_t s);
GnResult gauss_newton_step(Posterior& P, double* u_io, double* d_io, bool u_dev, bool d_dev, const gmrf_solve_opts& o,
                           cudaStream_t s);

// grad.cu
// dB/dtheta taps of the prior root per row class (0 interior / t >= 1,
// 1 t = 0) for theta = (log kappa, log tau, cx, nu)
struct DerivTaps {
    double d[4][2][NTAP];
};
DerivTaps derivative_taps(const gmrf_prior_desc& d, const Level& L);

// prior_det.cu: exact log det Q and 1/2 tr(Q^-1 dQ/dtheta) from the
// diagonal blocks of the root (interior 7-point operators)
struct Stencil7 {
    double c[7];
};
struct InteriorDet {
    double logabsdet = 0.0;
    int sign = 1;
    std::vector<double> tr;    // tr(A^-1 X_p)
};
InteriorDet interior_logdet(int mx, int my, const double a[7], const std::vector<Stencil7>& X);
struct PriorDet {
    double logdet = 0.0;
    double tr[4] = {0, 0, 0, 0};   // 1/2 tr(Q^-1 dQ/dtheta), theta = (log kappa, log tau, cx, nu)
};
PriorDet prior_logdet(const gmrf_prior_desc& d, const Level& F);

struct LoglikOut {
    double loglik = 0.0, loglik_se = 0.0;
    double logdet_prior = 0.0, logdet_post = 0.0;
    int lanczos_steps = 0;
    bool lanczos_converged = false;
};
// ll == nullptr: gradient only (no Lanczos quadrature)
SolveStats loglik_grad(Posterior& P, int S, uint64_t seed, const gmrf_solve_opts& o, int max_lanczos, LoglikOut* ll,
                       double grad[5], double gse[5], cudaStream_t s);

// slq.cu: log det Q_u|y by stochastic Lanczos quadrature over S Rademacher probes
struct SlqResult {
    double logdet = 0.0, stderr_ = 0.0;
    int steps = 0;
    bool converged = false;
};
SlqResult slq_logdet(Posterior& P, int S, uint64_t seed, int max_steps, cudaStream_t s);
double gauss_log_quadrature(const std::vector<double>& a, const std::vector<double>& b);

// scratch of one batch size
struct Workspace {
    int nblk = 0;
    // FP64 refinement vectors (blocked)
    double *b64 = nullptr, *x64 = nullptr, *r64 = nullptr, *t64 = nullptr;
    // observation-row normals of the drawn samples [nblk][rows][4], sized on first use
    double* z2 = nullptr;
    size_t z2_n = 0;
    // partial sums and per-RHS scalars
    double* partial = nullptr;
    size_t npartial = 0;
    double* red = nullptr;
    double* red2 = nullptr;        // second reduction target (nblk * 4)
    double* norms = nullptr;       // device, nblk * 4
    double* sc32 = nullptr;        // PCG scalars of the FP32 inner solve
    double* sc64 = nullptr;
    double* h_red = nullptr;       // pinned host mirror of `red`
    double* h_active = nullptr;    // pinned host mirror of the active flags
    int32_t* h_abort = nullptr;    // pinned copies of the two stencil abort flags
    SolveGraph* sgraph = nullptr;  // device-driven solve of this batch size (solver.cu)
    int32_t* slot_a = nullptr;     // per-slot ids (device)
    int32_t* slot_b = nullptr;
    // per-level vectors for each precision
    struct Vecs {
        bool ready = false;
        void* pcg[6] = {};             // x, r, p, q, z, p' (fine level; p and p' alternate in the fused iteration)
        std::vector<void*> xa, xb, d, res, b, t1, t2;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        double graph_tol = -1.0;   // inner tolerance baked into the captured graph
        unsigned long long graph_kernels = 0;
    } v32, v64;
};

}  // namespace gmrf
