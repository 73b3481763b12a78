// Host-side fault injection: which event of a context (or of an
// allocation-free call) fails on purpose, so that tests can drive every
// error path without making the GPU fault, trap or hang.
//
// A fault comes from gxp_config.fault / fault_at, or from the GXP_FAULT
// environment variable, "kind[:n][,kind[:n]...]" with kind one of
//   alloc    the n-th device allocation fails (as an out-of-memory would)
//   h2d      the n-th host-to-device copy is not enqueued (a failed copy)
//   sync     the n-th exchange between partitions is dropped (a lost message)
//   timeout  every bounded device-side wait gives up at once (then drains)
// and n >= 1 (default 1). The configuration takes precedence over the
// environment for the kinds it names.
#pragma once

#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "gxp.h"

namespace gxp {

struct FaultPlan {
    uint64_t alloc_at = 0;   // 1-based index of the event that fails; 0 = never
    uint64_t h2d_at = 0;
    uint64_t sync_at = 0;
    bool timeout = false;
};

// Parse GXP_FAULT (or `spec`, when given). Unknown kinds are ignored.
inline FaultPlan fault_plan_from_env(const char* spec = nullptr) {
    FaultPlan f;
    const char* s = spec ? spec : std::getenv("GXP_FAULT");
    if (!s) return f;
    while (*s) {
        const char* end = std::strchr(s, ',');
        const size_t len = end ? (size_t)(end - s) : std::strlen(s);
        const char* colon = static_cast<const char*>(std::memchr(s, ':', len));
        const size_t klen = colon ? (size_t)(colon - s) : len;
        uint64_t n = 1;
        if (colon) {
            n = std::strtoull(colon + 1, nullptr, 10);
            if (n == 0) n = 1;
        }
        auto is = [&](const char* k) { return klen == std::strlen(k) && std::strncmp(s, k, klen) == 0; };
        if (is("alloc")) f.alloc_at = n;
        else if (is("h2d")) f.h2d_at = n;
        else if (is("sync")) f.sync_at = n;
        else if (is("timeout")) f.timeout = true;
        if (!end) break;
        s = end + 1;
    }
    return f;
}

// The plan of a context: the environment's, overridden by the configuration.
inline FaultPlan fault_plan(const gxp_config& cfg) {
    FaultPlan f = fault_plan_from_env();
    const uint64_t n = cfg.fault_at ? cfg.fault_at : 1;
    switch (cfg.fault) {
        case GXP_FAULT_ALLOC: f.alloc_at = n; break;
        case GXP_FAULT_H2D: f.h2d_at = n; break;
        case GXP_FAULT_SYNC_DROP: f.sync_at = n; break;
        case GXP_FAULT_TIMEOUT: f.timeout = true; break;
        default: break;
    }
    return f;
}

}  // namespace gxp
