// Launch-shape autotuner of the persistent stencil kernels.
//
// A persistent stencil launch has free shape parameters that the source does
// not fix: how many CTAs it keeps on each SM (its grid, up to the occupancy
// limit) and, for the marching space-time kernel, how many time chunks a
// level is cut into (how many units of work the grid shares).  More CTAs per
// SM hide more latency; fewer give each CTA longer runs of neighbouring tiles
// (whose halos overlap in L2) and fewer dot partials; shorter time chunks
// balance the load but re-read one more plane per chunk.  The best shape
// depends on the kernel, the number of right-hand-side blocks, the size of
// the level and its observation tables, so it is measured.
//
// A key is (instantiation, right-hand-side blocks, units of work to half an
// octave, observation-table stride to an octave).  The first launch of a key
// that has more units than SMs times every candidate shape on zero-filled
// scratch copies of its vectors (CUDA events on the launching stream) and
// keeps the fastest; a choice is stored relative to the launch (CTAs per SM,
// time-chunk multiplier) so that it carries over to every level of the same
// bucket.  A launch recorded into a CUDA graph cannot be measured: it takes
// the default shape and queues its measurement, which the capturing code runs
// after the capture ends (tune_flush) before it captures again.
//
// Choices live in a process-wide table, listed by gmrf_autotune_log().  When
// GMRF_AUTOTUNE_FILE names a file, the table is read from it at first use and
// every new choice is appended to it.  GMRF_AUTOTUNE=0 (or gmrf_autotune_mode)
// turns measuring off: launches then take the default shape (every resident
// CTA; time chunks for about two units per resident CTA).
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <vector>

namespace gmrf {

struct TuneChoice {
    int ctas_per_sm;   // persistent grid = min(units, SMs x ctas_per_sm)
    int aux;           // marching kernel: time-chunk multiplier (units ~ aux x resident CTAs); else 0
};

struct TuneKey {
    std::string kernel;   // instantiation, e.g. "stencil<xy,f32,cheb,col0>"
    int nblk;             // right-hand-side blocks of four
    int units_bucket;     // round(2 log2(units))
    int obs_bucket;       // 0 without observation tables, else 1 + round(log2(stride bytes))
    std::string str() const;
};

int tune_units_bucket(long long units);
int tune_obs_bucket(int ostride_bytes, bool has_obs);

// Cached choice for key (true), or false (not measured yet).
bool tune_lookup(const TuneKey& key, TuneChoice* out);
// Measuring is on (mode and no TuneSuppress on this thread).
bool tune_enabled();
// Measuring is on and s (and this thread) is not capturing a graph.
bool tune_now(cudaStream_t s);
// Times run(c, s) for every candidate (one warm launch, then enough repeats
// for about half a millisecond), records the fastest under key and returns it.
TuneChoice tune_measure(const TuneKey& key, const std::vector<TuneChoice>& cands,
                        const std::function<void(const TuneChoice&, cudaStream_t)>& run, cudaStream_t s);
// Queues a measurement for after the current capture (this thread).
void tune_defer(std::function<void(cudaStream_t)> task);
// Runs the queued measurements on s; true if there were any (the caller then
// captures again so that the graph takes the measured shapes).
bool tune_flush(cudaStream_t s);

// While alive, launches on this thread neither measure nor queue (the
// allocation-free entry point).
struct TuneSuppress {
    TuneSuppress();
    ~TuneSuppress();
};

// Zero-filled device buffers of one measurement, freed on destruction.
struct TuneScratch {
    std::vector<void*> bufs;
    cudaStream_t stream = nullptr;
    void* zeros(size_t bytes, cudaStream_t s);
    ~TuneScratch();
};

// 0 off, 1 on; returns the previous mode.
int tune_set_mode(int mode);
// Every recorded choice, one JSON object per line.
std::string tune_log();

}  // namespace gmrf
