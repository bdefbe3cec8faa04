// Host-side state of a context (shared by the runtime and the serving loop).
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/rrs.h"
#include "rrs_internal.h"

namespace rrs {

struct Dataset {
    int64_t n = 0;
    int32_t d = 0;
    int32_t ldx = 0;
    int32_t kp = 0;
    float* X32 = nullptr;
    float* Xt = nullptr;       // d <= 16: the FP32 rows in 32-row tiles, 16-byte chunks interleaved (tile_rows)
    double* X64 = nullptr;
    float* xnorm = nullptr;
    uint16_t* Xbf = nullptr;
    float* center = nullptr;   // d, then (d <= RRS_COV_MAX_D) d*d covariance, then the radius
    float* cov = nullptr;
    float rc = 0.0f;
    size_t bytes = 0;
};

}  // namespace rrs

struct rrs_ctx {
    int device = 0;
    uint64_t budget = 0;
    uint64_t used = 0;
    int64_t next_id = 1;
    std::map<int64_t, rrs::Dataset> datasets;
    uint64_t launches = 0;
    int* d_err = nullptr;
    std::mutex mu;
    // cached captured graphs of batched calls (keyed by the request bytes)
    struct GraphEntry {
        std::vector<char> key;
        cudaGraphExec_t exec = nullptr;
        void* ws = nullptr;
        size_t ws_bytes = 0;
        size_t launches = 0;
    };
    std::vector<GraphEntry> graphs;
    // selection-kernel autotuning: (n, ldx, m) -> directions per CTA
    std::map<std::tuple<int64_t, int, int>, int> pd_tune;
    std::map<std::pair<int64_t, int>, int> tc_tune;   // (n, kp) -> points per tensor-core tile
    // per-stage CUDA-event timing (rrs_profile_*)
    bool profiling = false;
    struct Mark {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> event_pool;
    double stage_ms[RRS_NSTAGES] = {};
    int64_t stage_launches[RRS_NSTAGES] = {};
};

namespace rrs {
// Build (once) the BF16 hi/lo planes the tensor-core halfspace kernel streams;
// UNSUPPORTED for d + 2 > 128, BUDGET when they do not fit the context's budget.
rrs_status ensure_bf16_planes(rrs_ctx* ctx, Dataset& D);
}  // namespace rrs
