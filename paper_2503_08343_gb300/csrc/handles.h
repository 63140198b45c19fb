// Definitions of the opaque C handles (shared by the C ABI translation units).
#pragma once

#include <atomic>

#include "host.h"

// A prior lives while its handle or any posterior built on it is alive, so
// the handles may be destroyed in any order.
struct gmrf_prior {
    gmrf::Prior impl;
    cudaStream_t user = 0;   // unused: work runs on impl.stream
    bool own = false;        // impl.stream created by the library
    std::atomic<int> refs{1};
};

struct gmrf_posterior {
    gmrf::Posterior impl;
    gmrf_prior* prior = nullptr;
};
