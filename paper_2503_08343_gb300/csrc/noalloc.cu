// Allocation-free variant of the FP64 posterior-precision apply.
//
// Some callers cannot allocate device memory at the point where they need
// Q_u|y x: code running inside a custom allocator or memory-pool callback
// (a cudaMalloc there would re-enter the allocator), latency-critical loops
// that must not take cudaMalloc's implicit device synchronisation, and
// processes whose device memory is fully reserved by a pool at start-up.
// gmrf_apply_posterior_noalloc serves them: the caller passes the input and
// output vectors, and the scratch the computation needs (the vectors in the
// library's blocked four-wide layout and the per-CTA partial sums of
// x^T Q_u|y x) lives in one file-scope device array of fixed size.  The call
// makes no cudaMalloc, cudaFree or other allocating call.
#include <algorithm>
#include <mutex>
#include <string>

#include "autotune.h"
#include "handles.h"

namespace {

// Largest system accepted: 262 144 unknowns (a 512 x 512 grid).
constexpr long long kNoAllocMaxN = 262144;
// Room for the CTA partial sums of the persistent stencil grid.
constexpr long long kNoAllocMaxParts = 4096;
// Layout in doubles: blocked input [N][4] | blocked output [N][4] |
// partial sums [parts][4] | the reduced sums [4].  16.1 MB per device,
// held by every GPU that loads the library until the process exits.
constexpr long long kOffX = 0;
constexpr long long kOffY = kNoAllocMaxN * 4;
constexpr long long kOffPart = 2 * kNoAllocMaxN * 4;
constexpr long long kOffSum = kOffPart + kNoAllocMaxParts * 4;
constexpr long long kScratchDoubles = kOffSum + 4;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// In host code the symbol above is only a host-side stand-in; the device
// address is looked up with cudaGetSymbolAddress, once per device, while that
// device is current.
std::mutex g_mu;
double* g_addr[1024] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the first lookup loads this file's module, whose load is what
// places the array in device memory).
double* scratch_address() {
    int dev = 0;
    gmrf::cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 1024) throw gmrf::Error(GMRF_E_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_addr[dev] == nullptr) {
        void* p = nullptr;
        gmrf::cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
        g_addr[dev] = static_cast<double*>(p);
    }
    return g_addr[dev];
}

bool is_device_memory(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// x [N] -> blocked [N][4] with the three unused slots cleared (they are
// stale from the previous call otherwise).
__global__ void k_pack_one(const double* __restrict__ x, double* __restrict__ xb, long long N) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n >= N) return;
    xb[n * 4 + 0] = x[n];
    xb[n * 4 + 1] = 0.0;
    xb[n * 4 + 2] = 0.0;
    xb[n * 4 + 3] = 0.0;
}

__global__ void k_unpack_one(const double* __restrict__ yb, double* __restrict__ y, long long N) {
    const long long n = (long long)blockIdx.x * 256 + threadIdx.x;
    if (n < N) y[n] = yb[n * 4];
}

// The CTA-partial region holds the largest grid either stencil kernel launches.
static_assert(kNoAllocMaxParts >= 4096, "partial-sum scratch below the stencil grid caps");

}  // namespace

namespace gmrf {
void set_last_error(const std::string& msg);

// Set-up of the allocation-free apply for one posterior, run by
// gmrf_condition on the posterior's device: loads everything the entry point
// will touch (this file's module with the scratch array, the pack/unpack
// kernels, the FP64 apply instantiation of the posterior's stencil and the
// reduction kernel), so that gmrf_apply_posterior_noalloc itself loads and
// allocates nothing.  Posteriors above the size limit skip it.
void noalloc_prepare(const Posterior& P) {
    const Level& L = P.levels[0];
    if (L.N > kNoAllocMaxN) return;
    scratch_address();
    cudaFuncAttributes fa;
    cuda_check(cudaFuncGetAttributes(&fa, k_pack_one), "loading the allocation-free apply");
    cuda_check(cudaFuncGetAttributes(&fa, k_unpack_one), "loading the allocation-free apply");
    StencilArgs<double> a{};
    a.L = L.view<double>();
    a.nblk = 1;
    stencil_prepare<double>(L.geo, M_APPLY, a);
    reduce_prepare();
}
}  // namespace gmrf

extern "C" gmrf_status gmrf_apply_posterior_noalloc(gmrf_posterior* post, const double* x, double* y, double* xQx) {
    try {
        gmrf::TuneSuppress no_measuring;          // launch shapes: cached or default, never measured here
        if (!post || !x || !y) throw gmrf::Error(GMRF_E_INVALID, "gmrf_apply_posterior_noalloc: null argument");
        gmrf::Posterior& P = post->impl;
        const gmrf::Level& L = P.levels[0];
        const long long N = L.N;
        if (N > kNoAllocMaxN)
            throw gmrf::Error(GMRF_E_INVALID, "gmrf_apply_posterior_noalloc: " + std::to_string(N) +
                                                  " unknowns exceed the fixed scratch limit of " +
                                                  std::to_string(kNoAllocMaxN));
        if (std::max(gmrf::stencil_max_grid(), gmrf::march_max_grid()) > kNoAllocMaxParts)
            throw gmrf::Error(GMRF_E_INVALID, "gmrf_apply_posterior_noalloc: partial-sum scratch too small");
        if (!is_device_memory(x) || !is_device_memory(y))
            throw gmrf::Error(GMRF_E_INVALID, "gmrf_apply_posterior_noalloc: x and y must be device memory");
        const cudaStream_t s = P.prior->stream;
        double* scr = scratch_address();
        double* xb = scr + kOffX;
        double* yb = scr + kOffY;
        double* part = scr + kOffPart;
        double* sum = scr + kOffSum;
        const unsigned g = (unsigned)((N + 255) / 256);
        k_pack_one<<<g, 256, 0, s>>>(x, xb, N);
        gmrf::note_launch();
        gmrf::StencilArgs<double> a{};
        a.L = L.view<double>();
        a.nblk = 1;
        a.x = xb;
        a.out = yb;
        a.partial = part;     // every CTA clears its own entries before use
        const int nparts = gmrf::launch_stencil<double>(L.geo, gmrf::M_APPLY, a, s);
        if (nparts > kNoAllocMaxParts)
            throw gmrf::Error(GMRF_E_CUDA, "gmrf_apply_posterior_noalloc: stencil grid beyond the partial-sum scratch");
        gmrf::launch_reduce(part, nparts, 1, sum, s);
        k_unpack_one<<<g, 256, 0, s>>>(yb, y, N);
        gmrf::note_launch();
        gmrf::cuda_check(cudaGetLastError(), "gmrf_apply_posterior_noalloc launch");
        if (xQx) gmrf::cuda_check(cudaMemcpyAsync(xQx, sum, sizeof(double), cudaMemcpyDefault, s), "copy x^T Q x");
        gmrf::cuda_check(cudaStreamSynchronize(s), "gmrf_apply_posterior_noalloc");
        // a CTA that gave up its bounded wait for a staged tile left y and
        // x^T Q x incomplete: report it (this also clears the flag, so the
        // next solve does not inherit it)
        if (gmrf::stencil_abort_take(s))
            throw gmrf::Error(GMRF_E_CUDA, "gmrf_apply_posterior_noalloc: staged input tile did not arrive (bounded wait)");
        return GMRF_OK;
    } catch (const gmrf::Error& e) {
        gmrf::set_last_error(e.what());
        return e.status;
    } catch (const std::exception& e) {
        gmrf::set_last_error(e.what());
        return GMRF_E_INVALID;
    }
}
