// Launch tracing: CUDA-event timing, algorithmic bytes, launch and transfer
// counters. A ProfScope placed around a kernel launch records an event pair
// on the launching stream when timing is enabled.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/arso.h"

namespace arso {

void prof_begin(int kind, double bytes, cudaStream_t st, cudaEvent_t *ev_out);
void prof_end(int kind, double bytes, cudaStream_t st, cudaEvent_t start, double flops = 0.0, double smem = 0.0);
void prof_count_h2d(uint64_t bytes);
void prof_count_d2h(uint64_t bytes);
// while suspended (stream capture) scopes record nothing
void prof_suspend(bool on);
// a replayed graph: count its kernel launches under `kind` and time it as one scope
void prof_add_launches(int kind, uint64_t n);

struct ProfScope {
    int kind;
    double bytes, flops, smem;
    cudaStream_t st;
    cudaEvent_t start = nullptr;
    ProfScope(int k, double b, cudaStream_t s, double f = 0.0, double sm = 0.0)
        : kind(k), bytes(b), flops(f), smem(sm), st(s) {
        prof_begin(kind, bytes, st, &start);
    }
    ~ProfScope() { prof_end(kind, bytes, st, start, flops, smem); }
};

}  // namespace arso
