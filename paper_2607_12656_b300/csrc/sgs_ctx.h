// The decode context (internal): scratch, status word, streams and events of the decode
// pipeline.  Shared by the single-scene and batched decode entry points.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sgs.h"

constexpr int kMaxStages = 8;

struct sgs_ctx {
    int device;
    uint8_t *scratch;
    size_t scratch_bytes;
    int *status_dev;
    int *status_host;  // pinned
    uint64_t launches; // kernels launched by decode calls on this context
    int profile;       // record stage events in decode calls
    int n_marks;
    cudaEvent_t marks[kMaxStages + 1];  // caller's stream: start, tokens, octree, end
    cudaEvent_t amarks[2];              // attribute stream: start, end
    cudaStream_t aux;                   // attribute decode (lowest priority), forked from the caller
    cudaStream_t geo;                   // geometry chain (highest priority)
    cudaEvent_t fork, join, gjoin;
    uint32_t wait_limit;                // polls of each bounded device wait (sgs_set_wait_limit)
    uint32_t shape[4];                  // attribute decoder launch shape per coding mode (0: built-in)
    uint8_t *rws;                       // sgs_render workspace (grown on demand)
    size_t rws_bytes;
};
