// rs_ctx.hpp -- host-side context behind the rs_ctx handle of rs.h.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rs.h"

namespace rs {

enum KernelClass : int { KC_HIST = 0, KC_PASS = 1, KC_FILL = 2, KC_PACK = 3, KC_SEG = 4, KC_COUNT_ };

inline int kernel_class_of(const char* name) {
    if (!name) return -1;
    if (!std::strcmp(name, "hist")) return KC_HIST;
    if (!std::strcmp(name, "pass")) return KC_PASS;
    if (!std::strcmp(name, "fill")) return KC_FILL;
    if (!std::strcmp(name, "pack")) return KC_PACK;
    if (!std::strcmp(name, "seg")) return KC_SEG;
    return -1;
}

constexpr size_t kMaxTimedLaunches = 65536;

struct TimedLaunch {
    cudaEvent_t begin;
    cudaEvent_t end;
};

}  // namespace rs

struct rs_ctx {
    int device = 0;
    // device area allocated once at creation: [status word | pad | DevInfo]
    void* d_area = nullptr;
    uint32_t* d_status = nullptr;
    void* d_info = nullptr;
    rs_status host_error = RS_OK;  // sticky host-known error
    uint64_t launches = 0;
    uint32_t last_passes_total = 0;
    uint32_t last_tiles = 0;
    // sorts of at most this many keys take the narrow pass tile where one
    // exists (rs_ctx_set_pass_tile_limit; the default is the measured
    // crossover on GB300)
    uint64_t narrow_max_n = (uint64_t)1 << 19;
    bool timing = false;
    std::vector<rs::TimedLaunch> timed[rs::KC_COUNT_];
    std::vector<cudaEvent_t> event_pool;
    std::mutex mu;

    cudaEvent_t take_event() {
        if (!event_pool.empty()) {
            cudaEvent_t e = event_pool.back();
            event_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
};

namespace rs {

// RAII: make ctx->device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Brackets one kernel launch with events when the context is timing.
struct LaunchTimer {
    rs_ctx* ctx;
    int cls;
    cudaStream_t stream;
    cudaEvent_t b = nullptr;
    LaunchTimer(rs_ctx* c, int k, cudaStream_t s) : ctx(c), cls(k), stream(s) {
        ctx->launches++;
        if (ctx->timing && ctx->timed[cls].size() < kMaxTimedLaunches) {
            b = ctx->take_event();
            if (b) cudaEventRecord(b, stream);
        }
    }
    ~LaunchTimer() {
        if (!b) return;
        cudaEvent_t e = ctx->take_event();
        if (!e) return;
        cudaEventRecord(e, stream);
        ctx->timed[cls].push_back({b, e});
    }
};

}  // namespace rs
