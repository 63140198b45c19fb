// C ABI of the GMRF solver (declared in include/gmrf.h).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <map>
#include <thread>

#include "autotune.h"
#include "handles.h"

using namespace gmrf;

static void prior_release(gmrf_prior* p) {
    if (p->refs.fetch_sub(1) != 1) return;
    if (p->own && p->impl.stream) cudaStreamDestroy(p->impl.stream);
    delete p;
}

static thread_local std::string g_err;

namespace gmrf {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace gmrf

template <typename F> static gmrf_status guard(F&& f) {
    try {
        f();
        return GMRF_OK;
    } catch (const Error& e) {
        g_err = e.what();
        return e.status;
    } catch (const std::bad_alloc&) {
        g_err = "host allocation failed";
        return GMRF_E_OOM;
    } catch (const std::exception& e) {
        g_err = e.what();
        return GMRF_E_INVALID;
    }
}

static void require(bool ok, const std::string& msg) {
    if (!ok) throw Error(GMRF_E_INVALID, msg);
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void copy_out(double* dst, const double* dev_src, size_t n, cudaStream_t s) {
    GCK(cudaMemcpyAsync(dst, dev_src, n * sizeof(double),
                        is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
}

static void copy_in(double* dev_dst, const double* src, size_t n, cudaStream_t s) {
    GCK(cudaMemcpyAsync(dev_dst, src, n * sizeof(double),
                        is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

static void enter(gmrf_prior* pr) {
    if (pr->user) GCK(cudaStreamSynchronize(pr->user));
}

static gmrf_solve_opts resolve_opts(const gmrf_solve_opts* o) {
    gmrf_solve_opts d;
    gmrf_default_opts(&d);
    if (!o) return d;
    gmrf_solve_opts r = *o;
    if (!(r.rtol > 0)) r.rtol = d.rtol;
    if (r.max_refine <= 0) r.max_refine = d.max_refine;
    if (r.max_inner < 0) r.max_inner = 0;      // automatic, resolved per posterior
    if (!(r.inner_rtol > 0)) r.inner_rtol = d.inner_rtol;
    return r;
}

static gmrf_status finish(const SolveStats& st, gmrf_solve_info* info, int nrhs, double seconds) {
    if (info) {
        info->nrhs = nrhs;
        info->refinements = st.refinements;
        info->inner_iterations = st.inner;
        info->converged = st.converged ? 1 : 0;
        info->max_rel_residual = st.max_rel;
        info->seconds = seconds;
    }
    if (st.converged) return GMRF_OK;
    if (st.breakdown) {
        g_err = "conjugate gradients broke down (p^T Q p <= 0) before reaching rtol";
        return GMRF_E_NOT_SPD;
    }
    g_err = "iteration caps reached before rtol; max relative residual " + std::to_string(st.max_rel);
    return GMRF_E_NO_CONVERGENCE;
}

extern "C" {

void gmrf_default_opts(gmrf_solve_opts* o) {
    if (!o) return;
    o->rtol = 1e-10;
    o->max_refine = 12;
    o->max_inner = 0;
    o->inner_rtol = 1e-5;
    o->precision = 0;
    o->batched = 1;
    o->timeout_s = 0.0;
}

const char* gmrf_status_string(gmrf_status s) {
    switch (s) {
        case GMRF_OK: return "ok";
        case GMRF_E_INVALID: return "invalid argument";
        case GMRF_E_NOT_SPD: return "operator not positive definite";
        case GMRF_E_NO_CONVERGENCE: return "no convergence";
        case GMRF_E_CUDA: return "CUDA error";
        case GMRF_E_OOM: return "out of device memory";
        case GMRF_E_TIMEOUT: return "timeout";
    }
    return "unknown status";
}

const char* gmrf_last_error(void) { return g_err.c_str(); }

gmrf_status gmrf_build_prior(const gmrf_prior_desc* desc, void* stream, gmrf_prior** out) {
    return guard([&] {
        require(desc && out, "null argument");
        const gmrf_prior_desc& d = *desc;
        require(d.kind >= 0 && d.kind <= 3, "unknown prior kind");
        const bool st = d.kind == GMRF_ADVDIFF_ST_1D || d.kind == GMRF_ADVDIFF_ST_2D;
        require(d.nx >= 3, "nx must be >= 3");
        if (d.kind == GMRF_ADVDIFF_ST_1D) require(d.ny == 1, "1D space-time needs ny = 1");
        else require(d.ny >= 3, "2D priors need ny >= 3");
        if (st) require(d.nt >= 2, "space-time priors need nt >= 2");
        else require(d.nt == 1, "spatial priors need nt = 1");
        require(d.eps2 > 0 && d.tau > 0, "eps2 and tau must be positive");
        require(d.hi[0] > d.lo[0] && (d.ny == 1 || d.hi[1] > d.lo[1]) && (d.nt == 1 || d.hi[2] > d.lo[2]), "empty domain");
        if (st) require(d.kappa0 > 0 && d.nu >= 0, "space-time priors need kappa0 > 0, nu >= 0");
        else require(d.kappa > 0, "kappa must be positive");
        require((long long)d.nx * d.ny * d.nt < (1LL << 31), "grid too large for 32-bit node indices");
        require(d.nx < 32768 && d.ny < 32768 && d.nt < 32768, "axes are limited to 32767 nodes");
        require(d.bc == GMRF_BC_DIRICHLET || d.bc == GMRF_BC_PERIODIC, "unknown boundary");
        require(d.noise_kappa >= 0.0 && (d.noise_kappa == 0.0 || d.kind == GMRF_ADVDIFF_ST_1D),
                "Matern transition noise: the 1D space-time prior");
        require(d.decay >= 0.0 && d.decay < 1.0 && (d.decay == 0.0 || st), "decay: in [0, 1), space-time priors");
        if (d.bc == GMRF_BC_PERIODIC)
            require(!st && d.nx >= 5 && d.ny >= 5, "periodic boundary: spatial priors with at least 5 nodes per axis");
        gmrf_prior* p = new gmrf_prior();
        p->impl.desc = d;
        p->impl.geo = geometry_of(d);
        // a caller stream is used as is; otherwise the handle owns a
        // non-blocking stream (graph capture needs a stream other than 0)
        p->user = nullptr;
        p->own = stream == nullptr;
        if (stream) {
            p->impl.stream = (cudaStream_t)stream;
        } else {
            cudaError_t e = cudaStreamCreateWithFlags(&p->impl.stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                delete p;
                cuda_check(e, "cudaStreamCreateWithFlags");
            }
        }
        build_hierarchy(d, p->impl.levels);
        *out = p;
    });
}

gmrf_status gmrf_level_info(const gmrf_posterior* post, int32_t level, int32_t* dims, double* lmax) {
    return guard([&] {
        require(post && dims && level >= 0 && level < (int32_t)post->impl.levels.size(), "bad argument");
        const Level& L = post->impl.levels[(size_t)level];
        dims[0] = L.nx;
        dims[1] = L.ny;
        dims[2] = L.nt;
        if (lmax) *lmax = L.lmax;
    });
}

gmrf_status gmrf_transfer_info(const gmrf_posterior* post, int32_t* p1, double* data_share) {
    return guard([&] {
        require(post && p1, "bad argument");
        *p1 = post->impl.transfer_p1 ? 1 : 0;
        if (data_share) *data_share = post->impl.data_share;
    });
}

int64_t gmrf_num_unknowns(const gmrf_prior* p) { return p ? (int64_t)p->impl.levels[0].N : 0; }
int32_t gmrf_num_levels(const gmrf_prior* p) { return p ? (int32_t)p->impl.levels.size() : 0; }

void gmrf_prior_destroy(gmrf_prior* p) {
    if (p) prior_release(p);
}

static void rebuild_bdata(Posterior& P, cudaStream_t s) {
    const Level& L = P.levels[0];
    GCK(cudaMemcpyAsync(P.d_bdata, P.d_bstatic, sizeof(double) * L.N, cudaMemcpyDeviceToDevice, s));
    launch_obs_data_rhs(L, (int)P.m, P.d_ypoint, P.d_bdata, s);
}

gmrf_status gmrf_condition(gmrf_prior* prior, const gmrf_obs_desc* obs, gmrf_posterior** out) {
    gmrf_posterior* post = nullptr;
    const gmrf_status st = guard([&] {
        require(prior && obs && out, "null argument");
        enter(prior);
        const gmrf_prior_desc& d = prior->impl.desc;
        const cudaStream_t s = prior->impl.stream;
        require(obs->m >= 0, "negative observation count");
        require(obs->m == 0 || (obs->coords && obs->y), "coords and y are required");
        require(obs->m < (1LL << 30), "too many observations");
        post = new gmrf_posterior();
        post->prior = prior;
        prior->refs.fetch_add(1);
        Posterior& P = post->impl;
        P.prior = &prior->impl;
        P.levels = prior->impl.levels;
        for (Level& L : P.levels) {   // device members are per posterior
            L.d_obs = nullptr; L.d_tile_ptr = nullptr; L.d_tile_idx = nullptr;
            L.d_omap = nullptr; L.d_oent32 = nullptr; L.d_oent64 = nullptr;
            L.d_tsp32 = nullptr; L.d_tsp64 = nullptr;
            L.d_tspc32 = nullptr; L.d_tspc64 = nullptr;
        }
        const int dimc = d.kind == GMRF_ADVDIFF_ST_2D ? 3 : 2;
        P.m = obs->m;
        std::vector<double> coords((size_t)P.m * dimc);
        if (P.m) std::memcpy(coords.data(), obs->coords, coords.size() * sizeof(double));
        for (int64_t k = 0; k < P.m; ++k)
            for (int a = 0; a < dimc; ++a) require(std::isfinite(coords[(size_t)k * dimc + a]), "non-finite coordinate");
        P.y_point.assign(obs->y, obs->y + P.m);
        std::vector<double> rinv;
        for (int64_t k = 0; k < P.m; ++k) {
            const double sg = obs->sigma ? obs->sigma[k] : obs->sigma_all;
            require(sg > 0 && std::isfinite(sg), "observation sigma must be positive");
            require(std::isfinite(P.y_point[(size_t)k]), "non-finite observation value");
            rinv.push_back(1.0 / (sg * sg));
        }
        const Level& F = P.levels[0];
        std::vector<double> bstatic((size_t)F.N, 0.0);
        P.nic = 0;
        if (obs->ic) {
            require(d.kind == GMRF_ADVDIFF_ST_1D || d.kind == GMRF_ADVDIFF_ST_2D, "initial-condition rows need a space-time prior");
            require(obs->ic_sigma > 0, "ic_sigma must be positive");
            P.nic = (int64_t)d.nx * d.ny;
            P.ic_values.resize((size_t)P.nic);
            for (int64_t k = 0; k < P.nic; ++k) {
                const double x = d.lo[0] + (double)(k % d.nx) * F.hx;
                P.ic_values[(size_t)k] = obs->ic_values ? obs->ic_values[k] : -std::sin(3.14159265358979323846 * x);
                rinv.push_back(1.0 / (obs->ic_sigma * obs->ic_sigma));
                bstatic[(size_t)k] += P.ic_values[(size_t)k] / (obs->ic_sigma * obs->ic_sigma);
            }
        }
        P.colloc_kind = obs->colloc;
        P.ncol = 0;
        if (obs->colloc) {
            require(d.kind == GMRF_ADVDIFF_ST_1D, "collocation rows need the 1D space-time prior");
            require(obs->colloc >= 1 && obs->colloc <= 4, "colloc must be 0 .. 4");
            require(obs->colloc_sigma > 0, "colloc_sigma must be positive");
            P.ncol = (int64_t)(d.nx - 2) * (d.nt - 1);
            P.colloc_qeps = 1.0 / (obs->colloc_sigma * obs->colloc_sigma);
            P.colloc_nu = obs->colloc_nu;
            P.colloc_c = obs->colloc_c;
            const bool fem_rows = obs->colloc >= 3;
            const double hf = P.levels[0].hx;
            // rows observing the PDE: x % sx == 0 and t % st == 0 (strides halve on coarser levels)
            const int sx0 = std::max(1, (int)obs->colloc_stride_x), st0 = std::max(1, (int)obs->colloc_stride_t);
            auto active = [](int nx, int nt, int sx, int st) {
                long long cx = 0, ct = 0;
                for (int x = 1; x <= nx - 2; ++x) cx += x % sx == 0;
                for (int t = 1; t <= nt - 1; ++t) ct += t % st == 0;
                return (double)(cx * ct);
            };
            const double nfine = active(P.levels[0].nx, P.levels[0].nt, sx0, st0);
            for (size_t l = 0; l < P.levels.size(); ++l) {
                Level& L = P.levels[l];
                L.col.sx = std::max(1, sx0 >> (int)l);
                L.col.st = std::max(1, st0 >> (int)l);
                const double ncl = active(L.nx, L.nt, L.col.sx, L.col.st);
                // Burgers rows (2, 4) enter once linearised
                L.col.kind = (obs->colloc == 1 || obs->colloc == 3) ? obs->colloc : 0;
                // coarse levels: the row-count ratio keeps J^T Q_eps J of the same size;
                // FEM rows carry a factor h (int phi_i), which the ratio already covers
                L.col.qeps = ncl > 0 ? P.colloc_qeps * nfine / ncl * (fem_rows ? (hf * hf) / (L.hx * L.hx) : 1.0) : 0.0;
                L.col.inv_dt = 1.0 / L.dt;
                L.col.inv_2h = 1.0 / (2.0 * L.hx);
                L.col.nu_h2 = obs->colloc_nu / (L.hx * L.hx);
                L.col.c = obs->colloc_c;
                L.col.m6_dt = L.hx / (6.0 * L.dt);
                L.col.nu_2h = obs->colloc_nu / (2.0 * L.hx);
                L.col.row0 = (int32_t)(P.m + P.nic);
            }
            if (obs->colloc == 3) {
                // b += J^T Q_eps f on the fine level (FEM rows: f = int phi_i f, given per row)
                const Level& L = P.levels[0];
                auto none = [](int, int) { return 0.0; };
                for (int t = 1; t < L.nt; ++t)
                    for (int x = 1; x < L.nx - 1; ++x) {
                        if (!colloc_on(L.col, x, t)) continue;
                        const size_t r = (size_t)(t - 1) * (L.nx - 2) + (x - 1);
                        const double v = L.col.qeps * (obs->colloc_f ? obs->colloc_f[r] : 0.0);
                        double a[3], b[3];
                        fem_cn_row(L.col, x, t, none, a, b);
                        for (int e = 0; e < 3; ++e) {
                            bstatic[(size_t)t * L.nx + x + e - 1] += a[e] * v;
                            bstatic[(size_t)(t - 1) * L.nx + x + e - 1] += b[e] * v;
                        }
                    }
            }
            if (obs->colloc == 1) {
                // b += J^T Q_eps f on the fine level
                const Level& L = P.levels[0];
                for (int t = 1; t < L.nt; ++t)
                    for (int x = 1; x < L.nx - 1; ++x) {
                        if (!colloc_on(L.col, x, t)) continue;
                        const size_t r = (size_t)(t - 1) * (L.nx - 2) + (x - 1);
                        const double f = obs->colloc_f ? obs->colloc_f[r] : 0.0;
                        const double a = L.col.c;
                        const double cC = L.col.inv_dt + 2.0 * L.col.nu_h2, cL = -a * L.col.inv_2h - L.col.nu_h2,
                                     cR = a * L.col.inv_2h - L.col.nu_h2;
                        const double v = L.col.qeps * f;
                        bstatic[(size_t)t * L.nx + x] += cC * v;
                        bstatic[(size_t)t * L.nx + x - 1] += cL * v;
                        bstatic[(size_t)t * L.nx + x + 1] += cR * v;
                        bstatic[(size_t)(t - 1) * L.nx + x] += -L.col.inv_dt * v;
                    }
            }
        }
        P.nrows = P.m + P.nic + P.ncol;
        for (size_t l = 0; l < P.levels.size(); ++l) build_level_obs(d, P, coords, rinv, P.levels[l], l == 0);
        if (obs->colloc == 2 || obs->colloc == 4) {
            for (Level& L : P.levels) {
                L.d_mu32 = dev_alloc<float>((size_t)L.N);
                L.d_mu64 = dev_alloc<double>((size_t)L.N);
                GCK(cudaMemsetAsync(L.d_mu32, 0, sizeof(float) * L.N, s));
                GCK(cudaMemsetAsync(L.d_mu64, 0, sizeof(double) * L.N, s));
            }
        }
        posterior_setup_levels(P, s);
        if (obs->ic) P.ic_rinv = 1.0 / (obs->ic_sigma * obs->ic_sigma);
        P.use_tsp = tsp_applicable(P.levels[0], (int)P.nic);
        if (P.use_tsp) tsp_prepare(P.levels[0], (int)P.nic, s);
        dev_upload(&P.d_bstatic, bstatic);
        if (P.nic) dev_upload(&P.d_icvals, P.ic_values);
        P.d_bdata = dev_alloc<double>((size_t)F.N);
        P.d_ypoint = dev_alloc<double>((size_t)std::max<int64_t>(P.m, 1));
        if (P.m) GCK(cudaMemcpyAsync(P.d_ypoint, P.y_point.data(), sizeof(double) * P.m, cudaMemcpyHostToDevice, s));
        rebuild_bdata(P, s);
        noalloc_prepare(P);
        GCK(cudaStreamSynchronize(s));
        *out = post;
    });
    if (st != GMRF_OK && post) gmrf_posterior_destroy(post);
    return st;
}

void gmrf_posterior_destroy(gmrf_posterior* post) {
    if (!post) return;
    Posterior& P = post->impl;
    cudaStreamSynchronize(P.prior->stream);
    for (auto& kv : P.ws) workspace_free(kv.second);
    P.ws.clear();
    for (Level& L : P.levels) level_free(L);
    dev_free(P.d_bdata);
    dev_free(P.d_ypoint);
    dev_free(P.d_bstatic);
    dev_free(P.d_icvals);
    dev_free(P.d_blin);
    dev_free(P.d_gn);
    dev_free(P.d_grad_part);
    gmrf_prior* pr = post->prior;
    delete post;
    if (pr) prior_release(pr);
}

gmrf_status gmrf_update_data(gmrf_posterior* post, const double* y) {
    return guard([&] {
        require(post && (y || post->impl.m == 0), "null argument");
        enter(post->prior);
        Posterior& P = post->impl;
        const cudaStream_t s = P.prior->stream;
        if (P.m) copy_in(P.d_ypoint, y, (size_t)P.m, s);
        rebuild_bdata(P, s);
        GCK(cudaStreamSynchronize(s));
    });
}

// Batch of right-hand sides: optional data slot (the mean) followed by
// `ns` sample slots, padded to blocks of four.
struct Batch {
    int nrhs, nblk, off;
    std::vector<int32_t> sample, mean_row, samp_row;
};

static Batch make_batch(int ns, bool with_mean) {
    Batch b;
    b.off = with_mean ? 1 : 0;
    b.nrhs = ns + b.off;
    b.nblk = (b.nrhs + 3) / 4;
    const int P4 = b.nblk * 4;
    b.sample.assign((size_t)P4, -2);
    b.mean_row.assign((size_t)P4, -1);
    b.samp_row.assign((size_t)P4, -1);
    for (int i = 0; i < b.nrhs; ++i) {
        if (with_mean && i == 0) {
            b.sample[0] = -1;
            b.mean_row[0] = 0;
        } else {
            b.sample[(size_t)i] = i - b.off;
            b.samp_row[(size_t)i] = i - b.off;
        }
    }
    return b;
}

static SolveStats run_batch(Posterior& P, const Batch& b, uint64_t seed, const gmrf_solve_opts& o, cudaStream_t s) {
    Workspace& W = workspace(P, b.nblk);
    GCK(cudaMemcpyAsync(W.slot_a, b.sample.data(), sizeof(int32_t) * b.sample.size(), cudaMemcpyHostToDevice, s));
    const bool draws = b.nrhs > b.off;     // any sample slot (t64 is free until the solve ends)
    const long long orows = std::max<long long>(P.nrows, 1);    // observation rows (stream-1 normals)
    if (draws && W.z2_n < (size_t)b.nblk * orows * 4) {
        dev_free(W.z2);
        W.z2_n = (size_t)b.nblk * orows * 4;
        W.z2 = dev_alloc<double>(W.z2_n);
    }
    launch_sample_rhs(P.levels[0].geo, P.levels[0].view<double>(), seed, W.slot_a, P.linearised ? P.d_blin : P.d_bdata,
                      W.b64, draws ? W.t64 : nullptr, draws ? W.z2 : nullptr, orows, b.nblk, s);
    GCK(cudaMemsetAsync(W.x64, 0, sizeof(double) * b.nblk * P.levels[0].N * 4, s));
    if (o.batched || b.nblk == 1) return solve_blocked(P, b.nblk, W.b64, W.x64, o, s, true);
    // one right-hand side per solve (the comparison path): the batch is
    // spread to dense rows, each row solved alone, and the solutions packed back
    SolveStats tot;
    tot.converged = true;
    Workspace& W1 = workspace(P, 1);
    const long long N = P.levels[0].N;
    std::vector<int32_t> rows((size_t)b.nblk * 4, -1);
    for (int k = 0; k < b.nrhs; ++k) rows[(size_t)k] = k;
    GCK(cudaMemcpyAsync(W.slot_b, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice, s));
    launch_unpack(W.b64, W.t64, W.slot_b, N, b.nblk, s);
    for (int i = 0; i < b.nrhs; ++i) {
        std::vector<int32_t> one(4, -1);
        one[0] = i;
        GCK(cudaMemcpyAsync(W1.slot_b, one.data(), sizeof(int32_t) * 4, cudaMemcpyHostToDevice, s));
        launch_pack(W.t64, W1.b64, W1.slot_b, N, 1, s);
        GCK(cudaMemsetAsync(W1.x64, 0, sizeof(double) * N * 4, s));
        SolveStats st = solve_blocked(P, 1, W1.b64, W1.x64, o, s, true);
        tot.refinements += st.refinements;
        tot.inner += st.inner;
        tot.converged &= st.converged;
        tot.breakdown |= st.breakdown;
        tot.max_rel = std::max(tot.max_rel, st.max_rel);
        launch_unpack(W1.x64, W.r64, W1.slot_b, N, 1, s);
        GCK(cudaStreamSynchronize(s));
    }
    launch_pack(W.r64, W.x64, W.slot_b, N, b.nblk, s);
    GCK(cudaStreamSynchronize(s));
    return tot;
}

static void write_rows(Posterior& P, Workspace& W, const std::vector<int32_t>& rows, int count, double* dst,
                       cudaStream_t s) {
    if (!dst || count == 0) return;
    const long long N = P.levels[0].N;
    GCK(cudaMemcpyAsync(W.slot_b, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice, s));
    if (is_device_ptr(dst)) {
        launch_unpack(W.x64, dst, W.slot_b, N, W.nblk, s);
    } else {
        launch_unpack(W.x64, W.t64, W.slot_b, N, W.nblk, s);
        GCK(cudaMemcpyAsync(dst, W.t64, sizeof(double) * N * count, cudaMemcpyDeviceToHost, s));
    }
    GCK(cudaStreamSynchronize(s));
}

gmrf_status gmrf_reserve(gmrf_posterior* post, int32_t nrhs, const gmrf_solve_opts* opts) {
    return guard([&] {
        require(post && nrhs >= 1, "bad argument");
        enter(post->prior);
        Posterior& P = post->impl;
        const cudaStream_t s = P.prior->stream;
        const gmrf_solve_opts o = resolve_opts(opts);
        // one pass of the batch (mean + nrhs - 1 samples) creates every buffer
        // and CUDA graph of this batch size; its results are discarded
        const Batch b = make_batch(nrhs - 1, true);
        run_batch(P, b, 0, o, s);
        GCK(cudaStreamSynchronize(s));
    });
}

gmrf_status gmrf_solve_mean(gmrf_posterior* post, double* mu, const gmrf_solve_opts* opts, gmrf_solve_info* info) {
    gmrf_status rc = GMRF_OK;
    const gmrf_status st = guard([&] {
        require(post && mu, "null argument");
        enter(post->prior);
        Posterior& P = post->impl;
        const cudaStream_t s = P.prior->stream;
        const gmrf_solve_opts o = resolve_opts(opts);
        const auto t0 = std::chrono::steady_clock::now();
        const Batch b = make_batch(0, true);
        const SolveStats ss = run_batch(P, b, 0, o, s);
        write_rows(P, workspace(P, b.nblk), b.mean_row, 1, mu, s);
        rc = finish(ss, info, 1, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    });
    return st != GMRF_OK ? st : rc;
}

gmrf_status gmrf_sample(gmrf_posterior* post, int32_t ns, uint64_t seed, double* mean, double* x,
                        const gmrf_solve_opts* opts, gmrf_solve_info* info) {
    gmrf_status rc = GMRF_OK;
    const gmrf_status st = guard([&] {
        require(post && ns >= 0 && (ns == 0 || x), "bad argument");
        require(ns > 0 || mean, "nothing to compute");
        enter(post->prior);
        Posterior& P = post->impl;
        const cudaStream_t s = P.prior->stream;
        const gmrf_solve_opts o = resolve_opts(opts);
        const auto t0 = std::chrono::steady_clock::now();
        const Batch b = make_batch(ns, mean != nullptr);
        const SolveStats ss = run_batch(P, b, seed, o, s);
        Workspace& W = workspace(P, b.nblk);
        write_rows(P, W, b.mean_row, 1, mean, s);
        write_rows(P, W, b.samp_row, ns, x, s);
        rc = finish(ss, info, b.nrhs, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    });
    return st != GMRF_OK ? st : rc;
}

gmrf_status gmrf_marginal_var(gmrf_posterior* post, int32_t ns, uint64_t seed, double* mean, double* var,
                              double* stderr_, const gmrf_solve_opts* opts, gmrf_solve_info* info) {
    gmrf_status rc = GMRF_OK;
    const gmrf_status st = guard([&] {
        require(post && ns >= 1 && var, "bad argument");
        enter(post->prior);
        Posterior& P = post->impl;
        const cudaStream_t s = P.prior->stream;
        const gmrf_solve_opts o = resolve_opts(opts);
        const auto t0 = std::chrono::steady_clock::now();
        const Batch b = make_batch(ns, mean != nullptr);
        const SolveStats ss = run_batch(P, b, seed, o, s);
        Workspace& W = workspace(P, b.nblk);
        const long long N = P.levels[0].N;
        write_rows(P, W, b.mean_row, 1, mean, s);
        GCK(cudaMemcpyAsync(W.slot_a, b.sample.data(), sizeof(int32_t) * b.sample.size(), cudaMemcpyHostToDevice, s));
        if (W.v32.ready) {
            // Q x of the FP64 samples by the FP32 apply: each term carries a
            // relative error of about 1e-7, and the off-diagonal sum e_i is of
            // the size of x_i (no cancellation), far inside the Monte Carlo
            // error of the estimator
            float* x32 = static_cast<float*>(W.v32.pcg[0]);
            float* q32 = static_cast<float*>(W.v32.pcg[3]);
            launch_cast<float>(W.x64, x32, (long long)b.nblk * N * 4, s);
            StencilArgs<float> a{};
            a.L = P.levels[0].view<float>();
            a.nblk = b.nblk;
            a.x = x32;
            a.out = q32;
            launch_stencil<float>(P.levels[0].geo, M_APPLY, a, s);
            launch_rbmc<float>(q32, W.x64, P.levels[0].d_diag64, W.slot_a, N, b.nblk, ns, W.t64, W.t64 + N, s);
        } else {
            apply64(P, b.nblk, W.x64, W.r64, s);
            launch_rbmc<double>(W.r64, W.x64, P.levels[0].d_diag64, W.slot_a, N, b.nblk, ns, W.t64, W.t64 + N, s);
        }
        copy_out(var, W.t64, (size_t)N, s);
        if (stderr_) copy_out(stderr_, W.t64 + N, (size_t)N, s);
        GCK(cudaStreamSynchronize(s));
        if (stencil_abort_take(s)) throw Error(GMRF_E_CUDA, "stencil kernel: staged input tile did not arrive (bounded wait)");
        rc = finish(ss, info, b.nrhs, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    });
    return st != GMRF_OK ? st : rc;
}

// One instance of the single-thread batch: the whole gmrf_marginal_var
// enqueued on the prior's stream (sample right-hand sides, the device-driven
// solve, the variance estimator, the mean unpacked), nothing waited for.
// Device outputs are copied in stream order; host outputs after collect.
struct BatchItem {
    int i = -1;
    Batch b;
    double* mean = nullptr;
    double* var = nullptr;
    bool mean_host = false, var_host = false;
};

static void enqueue_marginal_var(Posterior& P, BatchItem& it, int ns, uint64_t seed, const gmrf_solve_opts& o) {
    const cudaStream_t s = P.prior->stream;
    it.b = make_batch(ns, it.mean != nullptr);
    const Batch& b = it.b;
    Workspace& W = workspace(P, b.nblk);
    const long long N = P.levels[0].N;
    GCK(cudaMemcpyAsync(W.slot_a, b.sample.data(), sizeof(int32_t) * b.sample.size(), cudaMemcpyHostToDevice, s));
    const long long orows = std::max<long long>(P.nrows, 1);
    if (W.z2_n < (size_t)b.nblk * orows * 4) {
        dev_free(W.z2);
        W.z2_n = (size_t)b.nblk * orows * 4;
        W.z2 = dev_alloc<double>(W.z2_n);
    }
    launch_sample_rhs(P.levels[0].geo, P.levels[0].view<double>(), seed, W.slot_a, P.linearised ? P.d_blin : P.d_bdata,
                      W.b64, W.t64, W.z2, orows, b.nblk, s);
    GCK(cudaMemsetAsync(W.x64, 0, sizeof(double) * b.nblk * N * 4, s));
    solve_graph_launch(P, b.nblk, W.b64, W.x64, o, s);
    // Rao-Blackwellised variances from the FP32 apply of the samples (as gmrf_marginal_var)
    float* x32 = static_cast<float*>(W.v32.pcg[0]);
    float* q32 = static_cast<float*>(W.v32.pcg[3]);
    launch_cast<float>(W.x64, x32, (long long)b.nblk * N * 4, s);
    StencilArgs<float> a{};
    a.L = P.levels[0].view<float>();
    a.nblk = b.nblk;
    a.x = x32;
    a.out = q32;
    launch_stencil<float>(P.levels[0].geo, M_APPLY, a, s);
    launch_rbmc<float>(q32, W.x64, P.levels[0].d_diag64, W.slot_a, N, b.nblk, ns, W.t64, W.t64 + N, s);
    it.var_host = !is_device_ptr(it.var);
    if (!it.var_host) GCK(cudaMemcpyAsync(it.var, W.t64, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    if (it.mean) {
        GCK(cudaMemcpyAsync(W.slot_b, b.mean_row.data(), sizeof(int32_t) * b.mean_row.size(), cudaMemcpyHostToDevice, s));
        launch_unpack(W.x64, W.r64, W.slot_b, N, b.nblk, s);
        it.mean_host = !is_device_ptr(it.mean);
        if (!it.mean_host) GCK(cudaMemcpyAsync(it.mean, W.r64, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    }
}

static SolveStats collect_marginal_var(Posterior& P, BatchItem& it) {
    const cudaStream_t s = P.prior->stream;
    GCK(cudaStreamSynchronize(s));
    const SolveStats st = solve_graph_collect(P, it.b.nblk, s);
    Workspace& W = workspace(P, it.b.nblk);
    const long long N = P.levels[0].N;
    if (it.var_host) GCK(cudaMemcpy(it.var, W.t64, sizeof(double) * N, cudaMemcpyDeviceToHost));
    if (it.mean && it.mean_host) GCK(cudaMemcpy(it.mean, W.r64, sizeof(double) * N, cudaMemcpyDeviceToHost));
    return st;
}

// The batch on one host thread: every instance is enqueued on its prior's
// stream before any is waited for (the device-driven solves need no host
// round trip), then all are collected in list order.  An instance whose
// posterior is still in flight is collected before it is enqueued again.
static gmrf_status marginal_var_batch_async(gmrf_posterior* const* posts, int32_t count, int32_t ns, uint64_t seed,
                                            double* const* means, double* const* vars, const gmrf_solve_opts& o,
                                            gmrf_solve_info* infos) {
    std::vector<BatchItem> items((size_t)count);
    std::vector<gmrf_status> sts((size_t)count, GMRF_OK);
    std::vector<std::string> errs((size_t)count);
    std::map<gmrf_posterior*, int> inflight;
    std::vector<std::chrono::steady_clock::time_point> t0((size_t)count);
    auto collect = [&](int i) {
        gmrf_posterior* p = posts[i];
        inflight.erase(p);
        const gmrf_status st = guard([&] {
            const SolveStats ss = collect_marginal_var(p->impl, items[(size_t)i]);
            gmrf_solve_info inf;
            std::memset(&inf, 0, sizeof(inf));
            const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0[(size_t)i]).count();
            const gmrf_status rc = finish(ss, &inf, items[(size_t)i].b.nrhs, sec);
            if (infos) infos[i] = inf;
            if (rc != GMRF_OK) throw Error(rc, g_err);
        });
        sts[(size_t)i] = st;
        if (st != GMRF_OK) errs[(size_t)i] = g_err;
    };
    for (int i = 0; i < count; ++i) {
        gmrf_posterior* p = posts[i];
        auto f = inflight.find(p);
        if (f != inflight.end()) collect(f->second);
        items[(size_t)i].i = i;
        items[(size_t)i].mean = means ? means[i] : nullptr;
        items[(size_t)i].var = vars[i];
        t0[(size_t)i] = std::chrono::steady_clock::now();
        const gmrf_status st = guard([&] {
            enter(p->prior);
            enqueue_marginal_var(p->impl, items[(size_t)i], ns, seed + (uint64_t)i, o);
        });
        if (st != GMRF_OK) {
            sts[(size_t)i] = st;
            errs[(size_t)i] = g_err;
            cudaStreamSynchronize(p->impl.prior->stream);
            continue;
        }
        inflight[p] = i;
    }
    for (int i = 0; i < count; ++i)
        if (inflight.count(posts[i]) && inflight[posts[i]] == i) collect(i);
    for (int i = 0; i < count; ++i) {       // report the first failing instance in list order
        if (sts[(size_t)i] != GMRF_OK) {
            g_err = "instance " + std::to_string(i) + ": " + errs[(size_t)i];
            return sts[(size_t)i];
        }
    }
    return GMRF_OK;
}

gmrf_status gmrf_marginal_var_batch(gmrf_posterior* const* posts, int32_t count, int32_t ns, uint64_t seed,
                                    double* const* means, double* const* vars, const gmrf_solve_opts* opts,
                                    gmrf_solve_info* infos, int32_t nthreads) {
    if (!posts || count < 0 || !vars) {
        g_err = "gmrf_marginal_var_batch: bad argument";
        return GMRF_E_INVALID;
    }
    for (int i = 0; i < count; ++i) {
        if (!posts[i] || !vars[i]) {
            g_err = "gmrf_marginal_var_batch: null posterior or output at instance " + std::to_string(i);
            return GMRF_E_INVALID;
        }
    }
    if (ns < 1) {
        g_err = "gmrf_marginal_var_batch: ns must be >= 1";
        return GMRF_E_INVALID;
    }
    {
        const gmrf_solve_opts o = resolve_opts(opts);
        bool fp32_inner = true;
        for (int i = 0; i < count; ++i) fp32_inner &= !inner_needs_fp64(posts[i]->impl);
        if (nthreads <= 1 && fp32_inner && device_loop_usable(o))
            return marginal_var_batch_async(posts, count, ns, seed, means, vars, o, infos);
    }
    // Posteriors of one prior share its stream (and a posterior listed twice
    // shares its workspace), so each group of instances with the same prior
    // goes to one worker, in list order; groups run concurrently.
    std::vector<std::vector<int>> groups;
    {
        std::map<const gmrf_prior*, size_t> at;
        for (int i = 0; i < count; ++i) {
            auto it = at.find(posts[i]->prior);
            if (it == at.end()) {
                at.emplace(posts[i]->prior, groups.size());
                groups.push_back({i});
            } else {
                groups[it->second].push_back(i);
            }
        }
    }
    const int ngroups = (int)groups.size();
    const int nt = std::max(1, std::min<int>(nthreads > 0 ? nthreads : 16, std::max(ngroups, 1)));
    std::atomic<int> next{0};
    std::vector<gmrf_status> sts((size_t)std::max(count, 1), GMRF_OK);
    std::vector<std::string> errs((size_t)std::max(count, 1));
    int dev = 0;
    cudaGetDevice(&dev);
    auto worker = [&]() {
        cudaSetDevice(dev);
        for (;;) {
            const int g = next.fetch_add(1);
            if (g >= ngroups) break;
            for (const int i : groups[(size_t)g]) {
                gmrf_solve_info inf;
                std::memset(&inf, 0, sizeof(inf));
                const gmrf_status st = gmrf_marginal_var(posts[i], ns, seed + (uint64_t)i, means ? means[i] : nullptr,
                                                         vars[i], nullptr, opts, &inf);
                if (infos) infos[i] = inf;
                sts[(size_t)i] = st;
                if (st != GMRF_OK) errs[(size_t)i] = g_err;
            }
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    for (int i = 0; i < count; ++i) {       // report the first failing instance in list order
        if (sts[(size_t)i] != GMRF_OK) {
            g_err = "instance " + std::to_string(i) + ": " + errs[(size_t)i];
            return sts[(size_t)i];
        }
    }
    return GMRF_OK;
}

gmrf_status gmrf_apply_posterior(gmrf_posterior* post, int32_t k, const double* x, double* y) {
    return guard([&] {
        require(post && k >= 1 && x && y, "bad argument");
        enter(post->prior);
        Posterior& P = post->impl;
        const cudaStream_t s = P.prior->stream;
        const int nblk = (k + 3) / 4;
        Workspace& W = workspace(P, nblk);
        const long long N = P.levels[0].N;
        std::vector<int32_t> rows((size_t)nblk * 4, -1);
        for (int i = 0; i < k; ++i) rows[(size_t)i] = i;
        copy_in(W.t64, x, (size_t)N * k, s);
        GCK(cudaMemcpyAsync(W.slot_b, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice, s));
        launch_pack(W.t64, W.b64, W.slot_b, N, nblk, s);
        apply64(P, nblk, W.b64, W.r64, s);
        launch_unpack(W.r64, W.t64, W.slot_b, N, nblk, s);
        copy_out(y, W.t64, (size_t)N * k, s);
        GCK(cudaStreamSynchronize(s));
        if (stencil_abort_take(s)) throw Error(GMRF_E_CUDA, "stencil kernel: staged input tile did not arrive (bounded wait)");
    });
}

gmrf_status gmrf_normals(uint64_t seed, int32_t stream, int32_t sample0, int32_t count, int64_t n, double* out) {
    return guard([&] {
        require(out && count >= 0 && n >= 0 && stream >= 0 && sample0 >= 0, "bad argument");
        if (count == 0 || n == 0) return;
        double* d = dev_alloc<double>((size_t)count * n);
        launch_normals(seed, stream, sample0, count, n, d, 0);
        cudaError_t e = cudaMemcpy(out, d, sizeof(double) * count * n, cudaMemcpyDefault);
        cudaFree(d);
        cuda_check(e, "gmrf_normals copy");
    });
}

gmrf_status gmrf_time_stencil(gmrf_posterior* post, int32_t kernel, int32_t k, int32_t iters, double* ms) {
    return guard([&] {
        require(post && k >= 1 && iters >= 1 && ms && kernel >= 0 && kernel <= 3, "bad argument");
        enter(post->prior);
        *ms = time_stencil(post->impl, kernel, (k + 3) / 4, iters, post->prior->impl.stream);
    });
}

gmrf_status gmrf_stencil_step(gmrf_posterior* post, int32_t level, int32_t precision, int32_t mode, int32_t k,
                              const double* x, const double* b, const double* d, double c0, double c1, double c2,
                              double* out, double* out2, double* dots) {
    return guard([&] {
        require(post && k >= 1 && out && dots, "bad argument");
        require(level >= 0 && level < (int32_t)post->impl.levels.size(), "level out of range");
        require(precision == 0 || precision == 1, "precision must be 0 or 1");
        require(mode >= 0 && mode <= 5, "mode must be 0..5");
        require(mode != 5 || level == 0, "mode 5 (preconditioner) is for level 0");
        require(mode == 3 || mode == 5 || x, "x is required");
        require(mode == 0 || b, "b is required");
        require(mode < 2 || mode == 5 || out2, "out2 is required for the Chebyshev and PCG modes");
        require(mode != 4 || d, "d is required for the PCG mode");
        enter(post->prior);
        Posterior& P = post->impl;
        const cudaStream_t s = P.prior->stream;
        const long long N = P.levels[(size_t)level].N;
        const size_t n = (size_t)N * k;
        double* buf = dev_alloc<double>(6 * n);
        const double* src[3] = {x, b, d};
        const double* din[3] = {nullptr, nullptr, nullptr};
        for (int i = 0; i < 3; ++i)
            if (src[i]) {
                copy_in(buf + i * n, src[i], n, s);
                din[i] = buf + i * n;
            }
        try {
            stencil_step(P, level, precision, mode, k, din[0], mode == 0 ? nullptr : din[1],
                         (mode == 2 || mode == 4) ? din[2] : nullptr, c0, c1, c2, buf + 3 * n,
                         (mode >= 2 && mode <= 4) ? buf + 4 * n : nullptr,
                         mode == 4 ? buf + 5 * n : nullptr, dots, s);
            copy_out(out, buf + 3 * n, n, s);
            if (mode >= 2 && mode <= 4) copy_out(out2, buf + 4 * n, n, s);
            if (mode == 4) copy_out(out2 + n, buf + 5 * n, n, s);
            GCK(cudaStreamSynchronize(s));
        } catch (...) {
            cudaStreamSynchronize(s);
            dev_free(buf);
            throw;
        }
        dev_free(buf);
    });
}

gmrf_status gmrf_prior_logdet(const gmrf_prior_desc* desc, double* logdet, double* trace) {
    return guard([&] {
        require(desc && (logdet || trace), "null argument");
        const gmrf_prior_desc& d = *desc;
        require(d.kind >= 0 && d.kind <= 3, "unknown prior kind");
        require(d.nx >= 3 && (d.kind == GMRF_ADVDIFF_ST_1D ? d.ny == 1 : d.ny >= 3), "bad grid");
        require(d.eps2 > 0 && d.tau > 0, "eps2 and tau must be positive");
        require(d.bc == GMRF_BC_DIRICHLET ||
                    (d.bc == GMRF_BC_PERIODIC && d.kind != GMRF_ADVDIFF_ST_1D && d.kind != GMRF_ADVDIFF_ST_2D && d.nx >= 5 && d.ny >= 5),
                "bad boundary");
        std::vector<Level> lv;
        build_hierarchy(d, lv);
        const PriorDet r = prior_logdet(d, lv[0]);
        if (logdet) *logdet = r.logdet;
        if (trace)
            for (int q = 0; q < 4; ++q) trace[q] = r.tr[q];
    });
}

void gmrf_test_set_wait_cap(int32_t cap) { set_wait_cap(cap); }

uint64_t gmrf_launch_count(void) { return launch_count(); }

int32_t gmrf_autotune_mode(int32_t mode) {
    if (mode < 0) return tune_enabled() ? 1 : 0;
    return tune_set_mode(mode);
}

int64_t gmrf_autotune_log(char* buf, int64_t cap) {
    std::string s;
    try {
        s = tune_log();
    } catch (...) {
        return -1;
    }
    if (buf && cap > 0) {
        const size_t n = std::min<size_t>(s.size(), (size_t)cap - 1);
        std::memcpy(buf, s.data(), n);
        buf[n] = '\0';
    }
    return (int64_t)s.size();
}

gmrf_status gmrf_gauss_newton_step(gmrf_posterior* post, double* mu_k, double* delta_prev, double* newton_decrement,
                                   double* alpha, const gmrf_solve_opts* opts, gmrf_solve_info* info) {
    gmrf_status rc = GMRF_OK;
    const gmrf_status st = guard([&] {
        require(post && mu_k && delta_prev && newton_decrement, "null argument");
        enter(post->prior);
        Posterior& P = post->impl;
        const gmrf_solve_opts o = resolve_opts(opts);
        const auto t0 = std::chrono::steady_clock::now();
        const GnResult r = gauss_newton_step(P, mu_k, delta_prev, is_device_ptr(mu_k), is_device_ptr(delta_prev), o,
                                             P.prior->stream);
        *newton_decrement = r.decrement;
        if (alpha) *alpha = r.alpha;
        rc = finish(r.stats, info, 1, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    });
    return st != GMRF_OK ? st : rc;
}

gmrf_status gmrf_loglik_grad_ex(gmrf_posterior* post, int32_t nprobes, uint64_t seed, int32_t max_lanczos,
                                double* loglik, gmrf_loglik_info* li, double* grad, double* grad_stderr,
                                const gmrf_solve_opts* opts, gmrf_solve_info* info) {
    gmrf_status rc = GMRF_OK;
    const gmrf_status st = guard([&] {
        require(post && grad && nprobes >= 1, "bad argument");
        Posterior& P = post->impl;
        require(P.nic == 0 && P.colloc_kind == 0, "gmrf_loglik_grad is defined for point data only");
        require(!P.levels[0].noise, "gmrf_loglik_grad: white transition noise only");
        enter(post->prior);
        const gmrf_solve_opts o = resolve_opts(opts);
        const auto t0 = std::chrono::steady_clock::now();
        double g[5], se[5];
        LoglikOut out;
        const bool value = loglik != nullptr || li != nullptr;
        const SolveStats ss = loglik_grad(P, nprobes, seed, o, max_lanczos > 0 ? max_lanczos : 400, value ? &out : nullptr,
                                          g, se, P.prior->stream);
        for (int i = 0; i < 5; ++i) {
            grad[i] = g[i];
            if (grad_stderr) grad_stderr[i] = se[i];
        }
        if (loglik) *loglik = out.loglik;
        if (li) {
            li->loglik_stderr = out.loglik_se;
            li->logdet_prior = out.logdet_prior;
            li->logdet_post = out.logdet_post;
            li->lanczos_steps = out.lanczos_steps;
            li->lanczos_converged = out.lanczos_converged ? 1 : 0;
        }
        rc = finish(ss, info, nprobes + 1, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    });
    return st != GMRF_OK ? st : rc;
}

gmrf_status gmrf_loglik_grad(gmrf_posterior* post, int32_t nprobes, uint64_t seed, double* loglik, double* grad,
                             double* grad_stderr, const gmrf_solve_opts* opts, gmrf_solve_info* info) {
    return gmrf_loglik_grad_ex(post, nprobes, seed, 0, loglik, nullptr, grad, grad_stderr, opts, info);
}

}  // extern "C"
