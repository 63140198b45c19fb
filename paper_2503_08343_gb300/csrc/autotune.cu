// Launch-shape autotuner: the measurement loop, the process-wide table and
// its optional file (the policy is described in autotune.h).
#include "autotune.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>

#include "host.h"

namespace gmrf {

namespace {

struct Entry {
    TuneChoice choice;
    std::string detail;   // candidate times (ms per launch) as JSON
};

std::mutex g_mu;
std::map<std::string, Entry> g_table;
bool g_loaded = false;
std::atomic<int> g_mode{-1};
thread_local int g_suppress = 0;
thread_local std::vector<std::function<void(cudaStream_t)>> g_pending;

int mode() {
    int m = g_mode.load();
    if (m < 0) {
        const char* e = std::getenv("GMRF_AUTOTUNE");
        m = (e != nullptr && e[0] == '0') ? 0 : 1;
        int expect = -1;
        g_mode.compare_exchange_strong(expect, m);
        m = g_mode.load();
    }
    return m;
}

const char* tune_file() {
    const char* f = std::getenv("GMRF_AUTOTUNE_FILE");
    return (f != nullptr && f[0] != '\0') ? f : nullptr;
}

// device name and SM count: a file may be shared between machines
std::string device_tag() {
    static std::string tag = [] {
        int dev = 0;
        cudaDeviceProp p;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return std::string("?");
        std::string n = p.name;
        for (char& c : n)
            if (c == ' ' || c == '"' || c == '|') c = '_';
        return n + "/" + std::to_string(p.multiProcessorCount) + "sm";
    }();
    return tag;
}

// one line per choice: {"key": "...", "ctas_per_sm": k, "aux": a, "ms": {...}}
std::string line_of(const std::string& key, const Entry& e) {
    std::ostringstream o;
    o << "{\"key\": \"" << key << "\", \"ctas_per_sm\": " << e.choice.ctas_per_sm << ", \"aux\": " << e.choice.aux
      << ", \"ms\": " << (e.detail.empty() ? "null" : e.detail) << "}";
    return o.str();
}

void load_file_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char* f = tune_file();
    if (!f) return;
    FILE* fp = std::fopen(f, "r");
    if (!fp) return;
    char buf[4096];
    while (std::fgets(buf, sizeof(buf), fp)) {
        char key[512];
        int k = 0, a = 0;
        if (std::sscanf(buf, "{\"key\": \"%511[^\"]\", \"ctas_per_sm\": %d, \"aux\": %d", key, &k, &a) == 3 && k > 0)
            g_table[key] = Entry{TuneChoice{k, a}, std::string()};
    }
    std::fclose(fp);
}

}  // namespace

std::string TuneKey::str() const {
    std::ostringstream o;
    o << device_tag() << "|" << kernel << "|nblk" << nblk << "|u" << units_bucket << "|o" << obs_bucket;
    return o.str();
}

int tune_units_bucket(long long units) { return (int)std::lround(2.0 * std::log2((double)std::max(1LL, units))); }

int tune_obs_bucket(int ostride_bytes, bool has_obs) {
    if (!has_obs) return 0;
    return 1 + (int)std::lround(std::log2((double)std::max(1, ostride_bytes)));
}

bool tune_lookup(const TuneKey& key, TuneChoice* out) {
    const std::string k = key.str();
    std::lock_guard<std::mutex> lock(g_mu);
    load_file_locked();
    auto it = g_table.find(k);
    if (it == g_table.end()) return false;
    *out = it->second.choice;
    return true;
}

bool tune_enabled() { return mode() != 0 && g_suppress == 0; }

bool tune_now(cudaStream_t s) {
    if (!tune_enabled()) return false;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st == cudaStreamCaptureStatusNone;
}

TuneChoice tune_measure(const TuneKey& key, const std::vector<TuneChoice>& cands,
                        const std::function<void(const TuneChoice&, cudaStream_t)>& run, cudaStream_t s) {
    if (cands.empty()) throw std::runtime_error("autotune: no candidate shapes");
    cudaEvent_t e0, e1;
    GCK(cudaEventCreate(&e0));
    GCK(cudaEventCreate(&e1));
    std::vector<double> ms(cands.size(), 0.0);
    try {
        for (size_t i = 0; i < cands.size(); ++i) {
            run(cands[i], s);                       // warm: code, TMA descriptors, L2
            GCK(cudaEventRecord(e0, s));
            run(cands[i], s);
            GCK(cudaEventRecord(e1, s));
            GCK(cudaEventSynchronize(e1));
            float one = 0.f;
            GCK(cudaEventElapsedTime(&one, e0, e1));
            const int reps = std::max(3, std::min(50, (int)std::ceil(0.5 / std::max(1e-4, (double)one))));
            GCK(cudaEventRecord(e0, s));
            for (int r = 0; r < reps; ++r) run(cands[i], s);
            GCK(cudaEventRecord(e1, s));
            GCK(cudaEventSynchronize(e1));
            float tot = 0.f;
            GCK(cudaEventElapsedTime(&tot, e0, e1));
            ms[i] = (double)tot / reps;
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    size_t best = 0;
    for (size_t i = 1; i < cands.size(); ++i)
        if (ms[i] < ms[best]) best = i;
    std::ostringstream d;
    d << "{";
    for (size_t i = 0; i < cands.size(); ++i) {
        char t[32];
        std::snprintf(t, sizeof(t), "%.9g", ms[i]);
        d << (i ? ", " : "") << "\"" << cands[i].ctas_per_sm << "x" << cands[i].aux << "\": " << t;
    }
    d << "}";
    Entry e{cands[best], d.str()};
    const std::string k = key.str();
    std::lock_guard<std::mutex> lock(g_mu);
    load_file_locked();
    g_table[k] = e;
    if (const char* f = tune_file()) {
        if (FILE* fp = std::fopen(f, "a")) {
            std::fprintf(fp, "%s\n", line_of(k, e).c_str());
            std::fclose(fp);
        }
    }
    return e.choice;
}

void tune_defer(std::function<void(cudaStream_t)> task) {
    if (tune_enabled()) g_pending.push_back(std::move(task));
}

bool tune_flush(cudaStream_t s) {
    if (g_pending.empty()) return false;
    std::vector<std::function<void(cudaStream_t)>> tasks;
    tasks.swap(g_pending);
    if (!tune_now(s)) return false;
    for (auto& t : tasks) t(s);
    return true;
}

TuneSuppress::TuneSuppress() { ++g_suppress; }
TuneSuppress::~TuneSuppress() { --g_suppress; }

void* TuneScratch::zeros(size_t bytes, cudaStream_t s) {
    stream = s;
    void* p = nullptr;
    GCK(cudaMalloc(&p, std::max<size_t>(bytes, 16)));
    bufs.push_back(p);
    GCK(cudaMemsetAsync(p, 0, std::max<size_t>(bytes, 16), s));
    return p;
}

TuneScratch::~TuneScratch() {
    if (bufs.empty()) return;
    cudaStreamSynchronize(stream);
    for (void* p : bufs) cudaFree(p);
}

int tune_set_mode(int m) {
    const int prev = mode();
    g_mode.store(m != 0 ? 1 : 0);
    return prev;
}

std::string tune_log() {
    std::lock_guard<std::mutex> lock(g_mu);
    load_file_locked();
    std::string out;
    for (const auto& kv : g_table) out += line_of(kv.first, kv.second) + "\n";
    return out;
}

}  // namespace gmrf
