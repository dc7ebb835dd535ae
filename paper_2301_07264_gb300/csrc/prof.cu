// Launch tracing (see prof.h and the tracing section of arso.h).
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.h"
#include "prof.h"

namespace arso {

namespace {
struct Pending {
    int kind;
    double bytes, flops, smem;
    cudaEvent_t a, b;
};
struct State {
    std::mutex mu;
    bool timing = false;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> free_events;
    arso_kernel_stats stats[ARSO_K_COUNT] = {};
};
State &state() {
    static State s;
    return s;
}
std::atomic<uint64_t> g_launches{0}, g_h2d{0}, g_d2h{0};
thread_local bool g_suspended = false;

cudaEvent_t take_event(State &s) {
    if (!s.free_events.empty()) {
        cudaEvent_t e = s.free_events.back();
        s.free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void resolve(State &s) {
    for (Pending &p : s.pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            s.stats[p.kind].ms += ms;
            s.stats[p.kind].bytes += p.bytes;
            s.stats[p.kind].flops += p.flops;
            s.stats[p.kind].smem_bytes += p.smem;
        } else {
            cudaGetLastError();
        }
        s.free_events.push_back(p.a);
        s.free_events.push_back(p.b);
    }
    s.pending.clear();
}
}  // namespace

void prof_begin(int kind, double, cudaStream_t st, cudaEvent_t *ev_out) {
    *ev_out = nullptr;
    if (g_suspended) return;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    State &s = state();
    std::lock_guard<std::mutex> lk(s.mu);
    s.stats[kind].launches += 1;
    if (!s.timing) return;
    cudaEvent_t e = take_event(s);
    if (e && cudaEventRecord(e, st) == cudaSuccess) *ev_out = e;
}

void prof_end(int kind, double bytes, cudaStream_t st, cudaEvent_t start, double flops, double smem) {
    if (!start) return;
    State &s = state();
    std::lock_guard<std::mutex> lk(s.mu);
    cudaEvent_t e = take_event(s);
    if (e && cudaEventRecord(e, st) == cudaSuccess) {
        s.pending.push_back(Pending{kind, bytes, flops, smem, start, e});
        if (s.pending.size() > 4096) resolve(s);
    } else {
        s.free_events.push_back(start);
    }
}

void prof_count_h2d(uint64_t b) { g_h2d.fetch_add(b, std::memory_order_relaxed); }
void prof_suspend(bool on) { g_suspended = on; }
void prof_add_launches(int kind, uint64_t n) {
    g_launches.fetch_add(n, std::memory_order_relaxed);
    State &s = state();
    std::lock_guard<std::mutex> lk(s.mu);
    s.stats[kind].launches += n;
}
void prof_count_d2h(uint64_t b) { g_d2h.fetch_add(b, std::memory_order_relaxed); }

}  // namespace arso

using namespace arso;

extern "C" {

arso_status arso_profile_enable(int on) {
    State &s = state();
    std::lock_guard<std::mutex> lk(s.mu);
    s.timing = on != 0;
    return ARSO_OK;
}

arso_status arso_profile_reset(void) {
    State &s = state();
    std::lock_guard<std::mutex> lk(s.mu);
    resolve(s);
    for (auto &x : s.stats) x = arso_kernel_stats{};
    g_launches = 0;
    g_h2d = 0;
    g_d2h = 0;
    return ARSO_OK;
}

arso_status arso_profile_read(uint32_t kernel, arso_kernel_stats *out) {
    if (kernel >= ARSO_K_COUNT || !out) {
        set_last_error("bad kernel id or NULL out");
        return ARSO_EINVAL;
    }
    State &s = state();
    std::lock_guard<std::mutex> lk(s.mu);
    resolve(s);
    *out = s.stats[kernel];
    return ARSO_OK;
}

arso_status arso_profile_counters(uint64_t *launches, uint64_t *h2d, uint64_t *d2h) {
    if (launches) *launches = g_launches.load();
    if (h2d) *h2d = g_h2d.load();
    if (d2h) *d2h = g_d2h.load();
    return ARSO_OK;
}

}  // extern "C"
