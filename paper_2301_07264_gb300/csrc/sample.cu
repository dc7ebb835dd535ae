// Monte Carlo Pauli error sampling on the GPU (Sec. IV-B.2).
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): a round maps the counter
// (c0, c1, c2, c3) under key (k0, k1) to
//   (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// M0 = 0xD2511F53, M1 = 0xCD9E8D57, and the key is advanced by the Weyl
// increments (0x9E3779B9, 0xBB67AE85) before every round after the first.
//
// Trajectory t, location pair j = l >> 1 draws one block with counter
// (j, t mod 2^32, t >> 32, 0x41525345) and key (seed mod 2^32, seed >> 32);
// even l uses words (w0, w1), odd l (w2, w3). Error iff w_a < thr; the type
// compares w_b with the cut points (X below cut_x, Z below cut_xz, else Y).
#include <algorithm>

#include "kernels.h"
#include "prof.h"

namespace arso {

constexpr uint32_t STREAM_ERRORS = 0x41525345u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t pauli_of(uint32_t wb, const SampleArgs &a) {
    const bool below_x = a.cut_x_all || wb < a.cut_x;
    const bool below_xz = a.cut_xz_all || wb < a.cut_xz;
    return below_x ? 1u : (below_xz ? 2u : 3u);
}

// one CTA per trajectory: number of errors
__global__ void sample_count_kernel(SampleArgs a, uint32_t *counts) {
    __shared__ uint32_t red[32];
    const uint32_t pairs = (a.L + 1) / 2;
    for (uint64_t b = blockIdx.x; b < a.n_traj; b += gridDim.x) {
        const uint64_t t = a.traj_begin + b;
        uint32_t cnt = 0;
        for (uint32_t j = threadIdx.x; j < pairs; j += blockDim.x) {
            const uint4 w = philox4x32_10(make_uint4(j, (uint32_t)t, (uint32_t)(t >> 32), STREAM_ERRORS),
                                          (uint32_t)a.seed, (uint32_t)(a.seed >> 32));
            cnt += w.x < a.thr;
            cnt += (2 * j + 1 < a.L) && (w.z < a.thr);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t s = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
            counts[b] = s;
        }
    }
}

// one CTA per trajectory: write the events in location order
__global__ void sample_fill_kernel(SampleArgs a, const uint64_t *__restrict__ offsets,
                                   const uint32_t *__restrict__ loc_key, uint32_t *ev_loc, uint32_t *ev_key) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    const uint32_t pairs = (a.L + 1) / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint64_t b = blockIdx.x; b < a.n_traj; b += gridDim.x) {
        const uint64_t t = a.traj_begin + b;
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        const uint64_t out0 = offsets[b];
        for (uint32_t j0 = 0; j0 < pairs; j0 += blockDim.x) {
            const uint32_t j = j0 + threadIdx.x;
            uint4 w = make_uint4(0xFFFFFFFFu, 0, 0xFFFFFFFFu, 0);
            if (j < pairs)
                w = philox4x32_10(make_uint4(j, (uint32_t)t, (uint32_t)(t >> 32), STREAM_ERRORS), (uint32_t)a.seed,
                                  (uint32_t)(a.seed >> 32));
            const bool h0 = j < pairs && w.x < a.thr;
            const bool h1 = j < pairs && (2 * j + 1 < a.L) && w.z < a.thr;
            const uint32_t c = (uint32_t)h0 + (uint32_t)h1;
            // block exclusive scan of c
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) warp_tot[warp] = incl;
            __syncthreads();
            uint32_t before = carry;
            for (int k = 0; k < warp; ++k) before += warp_tot[k];
            uint64_t pos = out0 + before + incl - c;
            if (h0) {
                const uint32_t l = 2 * j;
                const uint32_t code = pauli_of(w.y, a);
                ev_loc[pos] = (l << 2) | code;
                ev_key[pos] = (loc_key[l] << 2) | code;
                ++pos;
            }
            if (h1) {
                const uint32_t l = 2 * j + 1;
                const uint32_t code = pauli_of(w.w, a);
                ev_loc[pos] = (l << 2) | code;
                ev_key[pos] = (loc_key[l] << 2) | code;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t tot = 0;
                for (int k = 0; k < nw; ++k) tot += warp_tot[k];
                carry += tot;
            }
            __syncthreads();
        }
    }
}

// single-CTA exclusive scan: offsets[0] = 0, offsets[i+1] = offsets[i] + counts[i]
__global__ void exclusive_scan_kernel(const uint32_t *__restrict__ counts, uint64_t n, uint64_t *offsets) {
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        carry = 0;
        offsets[0] = 0;
    }
    __syncthreads();
    for (uint64_t i0 = 0; i0 < n; i0 += blockDim.x) {
        const uint64_t i = i0 + threadIdx.x;
        unsigned long long incl = i < n ? counts[i] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        unsigned long long before = carry;
        for (int k = 0; k < warp; ++k) before += warp_tot[k];
        if (i < n) offsets[i + 1] = before + incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int k = 0; k < nw; ++k) tot += warp_tot[k];
            carry += tot;
        }
        __syncthreads();
    }
}

__global__ void keys_from_loc_kernel(const uint32_t *__restrict__ ev_loc, uint64_t n, const uint32_t *__restrict__ loc_key,
                                     uint32_t *ev_key) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t e = ev_loc[i];
        ev_key[i] = (loc_key[e >> 2] << 2) | (e & 3u);
    }
}

// Engine order differs from circuit order in streaming schedules: sort each
// trajectory's keys (insertion sort; lists are short).
__global__ void sort_keys_kernel(const uint64_t *__restrict__ offsets, uint64_t n_traj, uint32_t *ev_key) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n_traj;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t *k = ev_key + offsets[t];
        const uint64_t m = offsets[t + 1] - offsets[t];
        for (uint64_t i = 1; i < m; ++i) {
            const uint32_t v = k[i];
            uint64_t j = i;
            while (j > 0 && k[j - 1] > v) {
                k[j] = k[j - 1];
                --j;
            }
            k[j] = v;
        }
    }
}

__global__ void first_event_kernel(const uint64_t *__restrict__ offsets, uint64_t n_traj,
                                   const uint32_t *__restrict__ ev_key, uint32_t *first, uint32_t *last) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n_traj;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const bool any = offsets[t + 1] > offsets[t];
        first[t] = any ? (ev_key[offsets[t]] >> 3) : NO_EVENT;
        last[t] = any ? (ev_key[offsets[t + 1] - 1] >> 3) : NO_EVENT;
    }
}

// sums3 = {sum score, sum score^2, sum pass} in FP64 (fixed order per block,
// then block partials summed by one block)
__global__ void sum_scores_kernel(const double *__restrict__ score, const uint8_t *__restrict__ pf, uint64_t n,
                                  double *sums3) {
    __shared__ double r0[32], r1[32], r2[32];
    double a = 0, b = 0, c = 0;
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double s = score[i];
        a += s;
        b += s * s;
        c += pf ? (double)pf[i] : 0.0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r0[threadIdx.x >> 5] = a;
        r1[threadIdx.x >> 5] = b;
        r2[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0, z = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            x += r0[w];
            y += r1[w];
            z += r2[w];
        }
        sums3[0] = x;
        sums3[1] = y;
        sums3[2] = z;
    }
}

static unsigned grid_for(uint64_t work, unsigned per_block, unsigned cap) {
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((work + per_block - 1) / per_block, cap));
}

// ------------------------------------------------------ batched sampling ---
// The lists of many circuits at once: the same draws, counts, scans and event
// words as the per-list kernels above, each kernel launched once for the batch.
// Global trajectory g belongs to the job whose [traj0, traj0 + n_traj) holds it.
__device__ __forceinline__ uint32_t job_of(const SampleJob *__restrict__ jobs, uint32_t n_jobs, uint64_t g) {
    uint32_t lo = 0, hi = n_jobs;  // first job with traj0 > g, minus one
    while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        if (jobs[mid].traj0 <= g) lo = mid + 1;
        else hi = mid;
    }
    return lo - 1;
}

__global__ void sample_count_batch_kernel(const SampleJob *__restrict__ jobs, uint32_t n_jobs, uint64_t n_total,
                                          uint32_t *counts) {
    __shared__ uint32_t red[32];
    for (uint64_t g = blockIdx.x; g < n_total; g += gridDim.x) {
        const SampleJob &J = jobs[job_of(jobs, n_jobs, g)];
        const SampleArgs &a = J.a;
        const uint64_t t = a.traj_begin + (g - J.traj0);
        const uint32_t pairs = a.thr ? (a.L + 1) / 2 : 0;
        uint32_t cnt = 0;
        for (uint32_t j = threadIdx.x; j < pairs; j += blockDim.x) {
            const uint4 w = philox4x32_10(make_uint4(j, (uint32_t)t, (uint32_t)(t >> 32), STREAM_ERRORS),
                                          (uint32_t)a.seed, (uint32_t)(a.seed >> 32));
            cnt += w.x < a.thr;
            cnt += (2 * j + 1 < a.L) && (w.z < a.thr);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t sum = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
            counts[g] = sum;
        }
    }
}

// one CTA per job: exclusive scan of its counts into its offsets; totals[job] = events
__global__ void scan_batch_kernel(const SampleJob *__restrict__ jobs, const uint32_t *__restrict__ counts,
                                  uint64_t *totals) {
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long carry;
    const SampleJob &J = jobs[blockIdx.x];
    const uint64_t n = J.a.n_traj;
    const uint32_t *cnt = counts + J.traj0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        carry = 0;
        J.offsets[0] = 0;
    }
    __syncthreads();
    for (uint64_t i0 = 0; i0 < n; i0 += blockDim.x) {
        const uint64_t i = i0 + threadIdx.x;
        unsigned long long incl = i < n ? cnt[i] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        unsigned long long before = carry;
        for (int k = 0; k < warp; ++k) before += warp_tot[k];
        if (i < n) J.offsets[i + 1] = before + incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int k = 0; k < nw; ++k) tot += warp_tot[k];
            carry += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void sample_fill_batch_kernel(const SampleJob *__restrict__ jobs, uint32_t n_jobs, uint64_t n_total) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint64_t g = blockIdx.x; g < n_total; g += gridDim.x) {
        const SampleJob &J = jobs[job_of(jobs, n_jobs, g)];
        const SampleArgs &a = J.a;
        const uint64_t b = g - J.traj0, t = a.traj_begin + b;
        const uint64_t out0 = J.offsets[b];
        if (J.offsets[b + 1] == out0) continue;  // no event (uniform over the CTA)
        const uint32_t pairs = (a.L + 1) / 2;
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (uint32_t j0 = 0; j0 < pairs; j0 += blockDim.x) {
            const uint32_t j = j0 + threadIdx.x;
            uint4 w = make_uint4(0xFFFFFFFFu, 0, 0xFFFFFFFFu, 0);
            if (j < pairs)
                w = philox4x32_10(make_uint4(j, (uint32_t)t, (uint32_t)(t >> 32), STREAM_ERRORS), (uint32_t)a.seed,
                                  (uint32_t)(a.seed >> 32));
            const bool h0 = j < pairs && w.x < a.thr;
            const bool h1 = j < pairs && (2 * j + 1 < a.L) && w.z < a.thr;
            const uint32_t c = (uint32_t)h0 + (uint32_t)h1;
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) warp_tot[warp] = incl;
            __syncthreads();
            uint32_t before = carry;
            for (int k = 0; k < warp; ++k) before += warp_tot[k];
            uint64_t pos = out0 + before + incl - c;
            if (h0) {
                const uint32_t l = 2 * j, code = pauli_of(w.y, a);
                J.ev_loc[pos] = (l << 2) | code;
                J.ev_key[pos] = (J.loc_key[l] << 2) | code;
                ++pos;
            }
            if (h1) {
                const uint32_t l = 2 * j + 1, code = pauli_of(w.w, a);
                J.ev_loc[pos] = (l << 2) | code;
                J.ev_key[pos] = (J.loc_key[l] << 2) | code;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t tot = 0;
                for (int k = 0; k < nw; ++k) tot += warp_tot[k];
                carry += tot;
            }
            __syncthreads();
        }
    }
}

// per trajectory: keys into engine order (when the schedule reorders gates), then the
// first and last event positions
__global__ void finish_batch_kernel(const SampleJob *__restrict__ jobs, uint32_t n_jobs, uint64_t n_total) {
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < n_total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const SampleJob &J = jobs[job_of(jobs, n_jobs, g)];
        const uint64_t b = g - J.traj0, o0 = J.offsets[b], o1 = J.offsets[b + 1];
        uint32_t *k = J.ev_key + o0;
        const uint64_t m = o1 - o0;
        if (!J.identity)
            for (uint64_t i = 1; i < m; ++i) {
                const uint32_t v = k[i];
                uint64_t j = i;
                while (j > 0 && k[j - 1] > v) {
                    k[j] = k[j - 1];
                    --j;
                }
                k[j] = v;
            }
        J.first[b] = m ? (k[0] >> 3) : NO_EVENT;
        J.last[b] = m ? (k[m - 1] >> 3) : NO_EVENT;
    }
}

void launch_sample_batch_count(const SampleJob *jobs, uint32_t n_jobs, uint64_t n_total, uint32_t *counts,
                               uint64_t *totals, cudaStream_t st) {
    if (!n_jobs) return;
    if (n_total) {
        ProfScope ps_(ARSO_K_SAMPLE, 4.0 * n_total, st);
        sample_count_batch_kernel<<<(unsigned)std::min<uint64_t>(n_total, 152ull * 64), 128, 0, st>>>(jobs, n_jobs,
                                                                                                     n_total, counts);
        ARSO_CUDA(cudaGetLastError());
    }
    ProfScope ps_(ARSO_K_OTHER, 0.0, st);
    scan_batch_kernel<<<n_jobs, 1024, 0, st>>>(jobs, counts, totals);
    ARSO_CUDA(cudaGetLastError());
}

void launch_sample_batch_fill(const SampleJob *jobs, uint32_t n_jobs, uint64_t n_total, bool any_events,
                              cudaStream_t st) {
    if (!n_jobs || !n_total) return;
    if (any_events) {
        ProfScope ps_(ARSO_K_SAMPLE, 0.0, st);
        sample_fill_batch_kernel<<<(unsigned)std::min<uint64_t>(n_total, 152ull * 64), 128, 0, st>>>(jobs, n_jobs,
                                                                                                    n_total);
        ARSO_CUDA(cudaGetLastError());
    }
    ProfScope ps_(ARSO_K_OTHER, 0.0, st);
    finish_batch_kernel<<<grid_for(n_total, 128, 152 * 16), 128, 0, st>>>(jobs, n_jobs, n_total);
    ARSO_CUDA(cudaGetLastError());
}

void launch_sample_count(const SampleArgs &a, uint32_t *counts, cudaStream_t st) {
    if (!a.n_traj) return;
    const unsigned grid = (unsigned)std::min<uint64_t>(a.n_traj, 152ull * 64);
    const int nt = a.L <= 64 ? 32 : (a.L <= 512 ? 128 : 256);
    ProfScope ps_(ARSO_K_SAMPLE, 4.0 * a.n_traj, st);
    sample_count_kernel<<<grid, nt, 0, st>>>(a, counts);
    ARSO_CUDA(cudaGetLastError());
}
void launch_exclusive_scan(const uint32_t *counts, uint64_t n, uint64_t *offsets, cudaStream_t st) {
    ProfScope ps_(ARSO_K_OTHER, 0.0, st);
    exclusive_scan_kernel<<<1, 1024, 0, st>>>(counts, n, offsets);
    ARSO_CUDA(cudaGetLastError());
}
void launch_sample_fill(const SampleArgs &a, const uint64_t *offsets, const uint32_t *loc_key, uint32_t *ev_loc,
                        uint32_t *ev_key, cudaStream_t st) {
    if (!a.n_traj) return;
    const unsigned grid = (unsigned)std::min<uint64_t>(a.n_traj, 152ull * 64);
    const int nt = a.L <= 64 ? 32 : (a.L <= 512 ? 128 : 256);
    ProfScope ps_(ARSO_K_SAMPLE, 0.0, st);
    sample_fill_kernel<<<grid, nt, 0, st>>>(a, offsets, loc_key, ev_loc, ev_key);
    ARSO_CUDA(cudaGetLastError());
}
void launch_keys_from_loc(const uint32_t *ev_loc, uint64_t n_events, const uint32_t *loc_key, uint32_t *ev_key,
                          cudaStream_t st) {
    if (!n_events) return;
    ProfScope ps_(ARSO_K_OTHER, 0.0, st);
    keys_from_loc_kernel<<<grid_for(n_events, 256, 152 * 16), 256, 0, st>>>(ev_loc, n_events, loc_key, ev_key);
    ARSO_CUDA(cudaGetLastError());
}
void launch_sort_keys(const uint64_t *offsets, uint64_t n_traj, uint32_t *ev_key, cudaStream_t st) {
    if (!n_traj) return;
    ProfScope ps_(ARSO_K_OTHER, 0.0, st);
    sort_keys_kernel<<<grid_for(n_traj, 128, 152 * 16), 128, 0, st>>>(offsets, n_traj, ev_key);
    ARSO_CUDA(cudaGetLastError());
}
void launch_first_event(const uint64_t *offsets, uint64_t n_traj, const uint32_t *ev_key, uint32_t *first,
                        uint32_t *last, cudaStream_t st) {
    if (!n_traj) return;
    ProfScope ps_(ARSO_K_OTHER, 0.0, st);
    first_event_kernel<<<grid_for(n_traj, 256, 152 * 16), 256, 0, st>>>(offsets, n_traj, ev_key, first, last);
    ARSO_CUDA(cudaGetLastError());
}
void launch_sum_scores(const double *score, const uint8_t *pass_flags, uint64_t n, double *sums3, cudaStream_t st) {
    ProfScope ps_(ARSO_K_REDUCE, 0.0, st);
    sum_scores_kernel<<<1, 1024, 0, st>>>(score, pass_flags, n, sums3);
    ARSO_CUDA(cudaGetLastError());
}

}  // namespace arso
