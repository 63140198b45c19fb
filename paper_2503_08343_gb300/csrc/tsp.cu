// Time-stepping preconditioner for collocation systems (1D space x time).
//
// With near-exact collocation (Sec. 3.1, 3.3) the posterior precision is
// dominated by Jt^T W Jt, where Jt stacks the initial-condition rows (t = 0),
// the Dirichlet rows of the prior at the spatial boundary and the
// collocation rows at interior nodes of levels k >= 1, with W their
// precisions.  Jt is square and block lower-bidiagonal in time (implicit
// Euler): level k reads level k (a tridiagonal stencil in x) and level k-1
// (-1/dt at the same x).  Its inverse is one forward time sweep and Jt^-T one
// backward sweep, each level a tridiagonal solve, so
//     z = M r = Jt^-1 W^-1 Jt^-T r
// costs two sweeps and leaves the prior's interior part and the point data,
// both orders of magnitude smaller, to the outer conjugate gradients.
// Tridiagonal systems are solved by parallel cyclic reduction in shared
// memory, one CTA per right-hand side and one thread per node of a level.
#include "handles.h"

namespace gmrf {

namespace {

constexpr int kTspMaxNx = 1024;

// Row coefficients of level k at node x: lower (x-1), diagonal, upper (x+1),
// plus the weight of the row.  Boundary x and level 0 are identity rows.
template <typename T>
__device__ __forceinline__ void tsp_row(const LevelView<T>& L, T w_ic, T w_bnd, int x, int k, T& lo, T& di, T& up, T& w) {
    const int nx = L.nx;
    if (k == 0) { lo = T(0); di = T(1); up = T(0); w = w_ic; return; }
    if (x == 0 || x == nx - 1) { lo = T(0); di = T(1); up = T(0); w = w_bnd; return; }
    const Colloc& c = L.col;
    T a, da;
    if (c.kind == 1) { a = (T)c.c; da = T(0); }
    else {
        const T* mu = L.mu + (long long)k * nx;
        a = mu[x];
        da = (mu[x + 1] - mu[x - 1]) * (T)c.inv_2h;
    }
    di = (T)c.inv_dt + da + T(2) * (T)c.nu_h2;
    lo = -a * (T)c.inv_2h - (T)c.nu_h2;
    up = a * (T)c.inv_2h - (T)c.nu_h2;
    w = (T)c.qeps;
}

// Parallel cyclic reduction on n <= blockDim.x equations held in shared
// memory (a: sub-diagonal, b: diagonal, c: super-diagonal, d: right-hand
// side); returns x_i for thread i < n.
template <typename T>
__device__ T pcr_solve(T* a, T* b, T* c, T* d, int n) {
    const int i = threadIdx.x;
    for (int s = 1; s < n; s <<= 1) {
        T an = T(0), bn = T(1), cn = T(0), dn = T(0);
        if (i < n) {
            const T ai = a[i], bi = b[i], ci = c[i], di = d[i];
            T k1 = T(0), k2 = T(0);
            bn = bi;
            dn = di;
            if (i - s >= 0) {
                k1 = ai / b[i - s];
                an = -a[i - s] * k1;
                bn -= c[i - s] * k1;
                dn -= d[i - s] * k1;
            }
            if (i + s < n) {
                k2 = ci / b[i + s];
                cn = -c[i + s] * k2;
                bn -= a[i + s] * k2;
                dn -= d[i + s] * k2;
            }
        }
        __syncthreads();
        if (i < n) { a[i] = an; b[i] = bn; c[i] = cn; d[i] = dn; }
        __syncthreads();
    }
    return i < n ? d[i] / b[i] : T(0);
}

// One CTA per right-hand side slot (block blk, component comp).  y is scratch
// of the blocked layout; r and z are blocked vectors.
template <typename T>
__global__ void __launch_bounds__(kTspMaxNx) k_tsp(const LevelView<T> L, T w_ic, T w_bnd, const T* __restrict__ r,
                                                  T* __restrict__ y, T* __restrict__ z) {
    __shared__ T sa[kTspMaxNx], sb[kTspMaxNx], sc[kTspMaxNx], sd[kTspMaxNx];
    const int nx = L.nx, nt = L.nt;
    const long long N = L.N;
    const int blk = blockIdx.x >> 2, comp = blockIdx.x & 3;
    const int x = threadIdx.x;
    const bool on = x < nx;
    auto at = [&](const T* v, int k) -> T { return v[(((size_t)blk * N) + (size_t)k * nx + x) * RW + comp]; };
    auto put = [&](T* v, int k, T val) { v[(((size_t)blk * N) + (size_t)k * nx + x) * RW + comp] = val; };
    const T inv_dt = (T)L.col.inv_dt;
    // backward sweep: Jt^T y = r, from the last level to the first.  Level k's
    // block is D_k^T; level k+1 reaches level k through C_{k+1}^T = -(1/dt) on
    // interior nodes.
    T ynext = T(0);       // y at (x, k+1)
    for (int k = nt - 1; k >= 0; --k) {
        T lo = T(0), di = T(1), up = T(0), w = T(1);
        if (on) tsp_row<T>(L, w_ic, w_bnd, x, k, lo, di, up, w);
        // D_k^T: sub-diagonal of row x is up(x-1), super-diagonal is lo(x+1)
        if (on) { sb[x] = di; sa[x] = T(0); sc[x] = T(0); }
        __syncthreads();
        if (on) {
            if (x + 1 < nx) sa[x + 1] = up;     // (D^T)_{x+1,x} = D_{x,x+1}
            if (x - 1 >= 0) sc[x - 1] = lo;     // (D^T)_{x-1,x} = D_{x,x-1}
        }
        __syncthreads();
        T rhs = on ? at(r, k) : T(0);
        const bool interior_next = k + 1 < nt && x > 0 && x < nx - 1;
        if (on && interior_next) rhs += inv_dt * ynext;
        if (on) sd[x] = rhs;
        __syncthreads();
        const T yk = pcr_solve<T>(sa, sb, sc, sd, nx);
        if (on) put(y, k, yk / w);               // store W^-1 y for the forward sweep
        ynext = yk;
        __syncthreads();
    }
    // forward sweep: Jt z = W^-1 y, from the first level to the last
    T zprev = T(0);
    for (int k = 0; k < nt; ++k) {
        T lo = T(0), di = T(1), up = T(0), w = T(1);
        if (on) tsp_row<T>(L, w_ic, w_bnd, x, k, lo, di, up, w);
        if (on) { sa[x] = lo; sb[x] = di; sc[x] = up; }
        T rhs = on ? at(y, k) : T(0);
        if (on && k > 0 && x > 0 && x < nx - 1) rhs += inv_dt * zprev;
        if (on) sd[x] = rhs;
        __syncthreads();
        const T zk = pcr_solve<T>(sa, sb, sc, sd, nx);
        if (on) put(z, k, zk);
        zprev = zk;
        __syncthreads();
    }
}

}  // namespace

bool tsp_applicable(const Level& L, int nic) {
    return L.geo == GEO_XT && L.col.kind != 0 && nic > 0 && L.nx <= kTspMaxNx;
}

template <typename T>
void launch_tsp(const Level& L, double w_ic, double w_bnd, const T* r, T* y, T* z, int nblk, cudaStream_t s) {
    int threads = 32;
    while (threads < L.nx) threads <<= 1;
    k_tsp<T><<<nblk * 4, threads, 0, s>>>(L.view<T>(), (T)w_ic, (T)w_bnd, r, y, z);
    note_launch();
}
template void launch_tsp<float>(const Level&, double, double, const float*, float*, float*, int, cudaStream_t);
template void launch_tsp<double>(const Level&, double, double, const double*, double*, double*, int, cudaStream_t);

}  // namespace gmrf
