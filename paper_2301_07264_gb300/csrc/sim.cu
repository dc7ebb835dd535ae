// Trajectory simulation kernels.
//
// Resident engine: one CTA per trajectory holds the whole 2^n state in shared
// memory, restarts from the cached error-free state at the checkpoint before
// the trajectory's first error, applies the remaining gates with the sampled
// Pauli error gates right after the gates they follow (Sec. IV-B), and
// scores the final state (Sec. II criteria) with an FP64 block reduction.
//
// Streaming engine: one launch per fused pass; CTA (tile, slot) loads a tile
// of 2^t amplitudes from HBM with 16-byte vector loads, applies the pass's
// gates and error gates in shared memory and writes the tile back (or, in the
// last pass, reduces it into a criterion partial instead of writing it).
#include <algorithm>

#include "sim_common.cuh"
#include "prof.h"

namespace arso {

// ------------------------------------------------------------- resident ---

template <typename T>
__device__ void resident_run_gates(T *s, int n, const DGate *__restrict__ gates, const T *__restrict__ mats,
                                   uint32_t g0, uint32_t G, const uint32_t *ev, const uint32_t *ev_end) {
    uint32_t next = ev < ev_end ? *ev : NO_EVENT;
    for (uint32_t g = g0; g < G; ++g) {
        const DGate gate = gates[g];
        if (gate.cls != GC_NOP) {
            tile_gate(s, n, gate, mats + gate.mat);
            __syncthreads();
        }
        while (next != NO_EVENT && ev_pos(next) == g) {
            tile_pauli(s, n, ev_slot(next) ? gate.q1 : gate.q0, ev_code(next));
            __syncthreads();
            ++ev;
            next = ev < ev_end ? *ev : NO_EVENT;
        }
    }
}

template <typename T>
__global__ void resident_kernel(ResidentArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    __shared__ Partial red[32];
    const int n = a.n;
    const uint32_t N = 1u << n;
    const T *cache = static_cast<const T *>(a.cache);
    const T *ref = cache + (size_t)(a.n_ckpt - 1) * N;
    const DCrit crit = a.crit;
    for (uint64_t b = blockIdx.x; b < a.count; b += gridDim.x) {
        const uint64_t tr = a.first_traj + b;
        const uint32_t first = a.first[tr];
        if (first == NO_EVENT && !a.states_out) {
            if (threadIdx.x == 0) {
                a.score[tr] = *a.ref_score;
                if (a.pass_flags) a.pass_flags[tr] = *a.ref_score >= crit.threshold;
            }
            continue;
        }
        const uint32_t ck = first == NO_EVENT ? a.n_ckpt - 1 : (uint32_t)(first / a.ckpt_every);
        const uint32_t g0 = first == NO_EVENT ? a.G : (uint32_t)(ck * a.ckpt_every);
        const T *src = cache + (size_t)ck * N;
        for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) s[i] = src[i];
        __syncthreads();
        const uint32_t *ev = a.keys + a.offsets[tr];
        const uint32_t *ev_end = a.keys + a.offsets[tr + 1];
        resident_run_gates(s, n, a.gates, static_cast<const T *>(a.mats), g0, a.G, ev, ev_end);
        if (a.states_out) {
            T *dst = static_cast<T *>(a.states_out) + (size_t)b * N;
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) dst[i] = s[i];
        } else {
            Partial acc = empty_partial();
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) accumulate(acc, crit, s[i], ref, i);
            acc = block_reduce_partial(acc, red);
            if (threadIdx.x == 0) {
                const double sc = finish_score(crit, acc);
                a.score[tr] = sc;
                if (a.pass_flags) a.pass_flags[tr] = sc >= crit.threshold;
            }
        }
        __syncthreads();
    }
}

// Error-free run that fills the checkpoint cache: entry c holds the state
// after gates [0, c * every); the last entry holds psi_R.
template <typename T>
__global__ void resident_ideal_kernel(ResidentArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    const int n = a.n;
    const uint32_t N = 1u << n;
    T *cache = static_cast<T *>(const_cast<void *>(a.cache));
    const T *mats = static_cast<const T *>(a.mats);
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
        T z;
        z.x = i == 0 ? 1 : 0;
        z.y = 0;
        s[i] = z;
    }
    __syncthreads();
    for (uint32_t g = 0; g <= a.G; ++g) {
        if (g % a.ckpt_every == 0 || g == a.G) {
            const uint32_t c = g == a.G ? a.n_ckpt - 1 : (uint32_t)(g / a.ckpt_every);
            T *dst = cache + (size_t)c * N;
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) dst[i] = s[i];
        }
        if (g == a.G) break;
        const DGate gate = a.gates[g];
        tile_gate(s, n, gate, mats + gate.mat);
        __syncthreads();
    }
}

// ------------------------------------------------------------ streaming ---

__device__ __forceinline__ uint64_t tile_base(uint64_t tile, uint64_t rest_mask) {
    // deposit the bits of `tile` into the set bits of rest_mask
    uint64_t base = 0;
    for (uint64_t m = rest_mask; m; m &= m - 1) {
        const uint64_t low = m & (~m + 1);
        if (tile & 1) base |= low;
        tile >>= 1;
    }
    return base;
}

template <typename T>
__device__ __forceinline__ uint64_t tile_index(uint32_t j, uint64_t base, const uint32_t *__restrict__ offs, int c) {
    return base + offs[j >> c] + (j & ((1u << c) - 1));
}

template <typename T, bool LAST>
__global__ void pass_kernel(PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    __shared__ Partial red[32];
    const int t = a.t, c = a.c;
    const uint32_t slot = blockIdx.y;
    const uint64_t N = 1ull << a.n;
    int start, end = 0;
    uint64_t tr = 0;
    const T *src;
    T *dst;
    if (a.ideal) {
        start = 0;
        src = static_cast<const T *>(a.ideal_src);
        dst = static_cast<T *>(a.ideal_dst);
    } else {
        start = a.start_pass[slot];
        end = a.end_pass[slot];
        if (a.pass < start || a.pass > end) return;
        tr = a.slot_traj[slot];
        T *mine = static_cast<T *>(a.work) + (size_t)slot * N;
        src = a.pass == start ? static_cast<const T *>(a.cache) + (size_t)a.cache_slot[start] * N : mine;
        dst = mine;
    }
    const uint64_t base = tile_base(blockIdx.x, a.rest_mask);
    const uint32_t *offs = a.offs;
    const uint32_t tile_n = 1u << t;
    // load: two amplitudes (16 bytes for complex64) per step; bit 0 is a tile bit
    for (uint32_t v = threadIdx.x; v < tile_n / 2; v += blockDim.x) {
        const uint32_t j = 2 * v;
        const uint64_t gi = tile_index<T>(j, base, offs, c);
        if (sizeof(T) == 8) {
            const float4 w = __ldg(reinterpret_cast<const float4 *>(src + gi));
            reinterpret_cast<float4 *>(s)[v] = w;
        } else {
            s[j] = src[gi];
            s[j + 1] = src[gi + 1];
        }
    }
    __syncthreads();
    const uint32_t *ev = nullptr, *ev_end = nullptr;
    if (!a.ideal) {
        // events of this trajectory with engine position in [gb, ge)
        const uint32_t *lo = a.keys + a.offsets[tr];
        const uint32_t *hi = a.keys + a.offsets[tr + 1];
        const uint32_t key_lo = a.gb << 3;
        while (lo < hi) {
            const uint32_t *mid = lo + (hi - lo) / 2;
            if (*mid < key_lo) lo = mid + 1; else hi = mid;
        }
        ev = lo;
        ev_end = a.keys + a.offsets[tr + 1];
    }
    {
        uint32_t next = ev && ev < ev_end ? *ev : NO_EVENT;
        const T *mats = static_cast<const T *>(a.mats);
        for (uint32_t g = a.gb; g < a.ge; ++g) {
            const DGate gate = a.gates[g];
            if (gate.cls != GC_NOP) {
                tile_gate(s, t, gate, mats + gate.mat);
                __syncthreads();
            }
            while (next != NO_EVENT && ev_pos(next) == g) {
                tile_pauli(s, t, ev_slot(next) ? gate.q1 : gate.q0, ev_code(next));
                __syncthreads();
                ++ev;
                next = ev < ev_end ? *ev : NO_EVENT;
            }
        }
    }
    if (!a.ideal && !a.store_last && a.pass == end) {
        const T *ref = static_cast<const T *>(a.ref_cache ? a.ref_cache : a.cache) + (size_t)a.cache_slot[end + 1] * N;
        Partial acc = empty_partial();
        for (uint32_t j = threadIdx.x; j < tile_n; j += blockDim.x) {
            const uint64_t gi = tile_index<T>(j, base, offs, c);
            accumulate(acc, a.crit, s[j], ref, gi);
        }
        acc = block_reduce_partial(acc, red);
        if (threadIdx.x == 0) a.partials[(size_t)slot * gridDim.x + blockIdx.x] = acc;
    } else {
        for (uint32_t v = threadIdx.x; v < tile_n / 2; v += blockDim.x) {
            const uint32_t j = 2 * v;
            const uint64_t gi = tile_index<T>(j, base, offs, c);
            if (sizeof(T) == 8) {
                reinterpret_cast<float4 *>(dst + gi)[0] = reinterpret_cast<const float4 *>(s)[v];
            } else {
                dst[gi] = s[j];
                dst[gi + 1] = s[j + 1];
            }
        }
    }
}

// Combine per-tile partials of each slot (fixed order) into its score.
__global__ void finish_partials_kernel(const Partial *__restrict__ partials, uint32_t tiles, uint32_t slots,
                                       const uint64_t *__restrict__ slot_traj, DCrit crit, double *score,
                                       uint8_t *pass_flags) {
    __shared__ Partial red[32];
    for (uint32_t slot = blockIdx.x; slot < slots; slot += gridDim.x) {
        Partial acc = empty_partial();
        for (uint32_t i = threadIdx.x; i < tiles; i += blockDim.x) {
            const Partial p = partials[(size_t)slot * tiles + i];
            acc.a += p.a;
            acc.b += p.b;
            argmax_merge(acc.maxp, acc.idx, p.maxp, p.idx);
        }
        acc = block_reduce_partial(acc, red);
        if (threadIdx.x == 0) {
            const double sc = finish_score(crit, acc);
            const uint64_t tr = slot_traj ? slot_traj[slot] : slot;
            score[tr] = sc;
            if (pass_flags) pass_flags[tr] = sc >= crit.threshold;
        }
        __syncthreads();
    }
}

// Trajectories without errors take the error-free score.
__global__ void fill_error_free_kernel(const uint32_t *__restrict__ first, uint64_t n_traj,
                                       const double *__restrict__ ref_score, double threshold, double *score,
                                       uint8_t *pass_flags) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_traj;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (first[i] == NO_EVENT) {
            score[i] = *ref_score;
            if (pass_flags) pass_flags[i] = *ref_score >= threshold;
        }
    }
}

// ------------------------------------------------- single-step HBM kernels --

// One gate on a device state: coalesced strided pair (or quad) updates; each
// thread owns one pair (i, i | 2^q) whose low index bits follow the thread id.
__global__ void gate_pairs_kernel(float2 *psi, int n, DGate g, M16 mm) {
    const float2 *m16 = mm.m;
    const float2 m0 = m16[0], m1 = m16[1], m2 = m16[2], m3 = m16[3];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (g.arity == 1) {
        const uint64_t bit = 1ull << g.q0, lo = bit - 1;
        for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < (1ull << (n - 1)); p += stride) {
            const uint64_t i0 = ((p & ~lo) << 1) | (p & lo), i1 = i0 | bit;
            const float2 a0 = psi[i0], a1 = psi[i1];
            if (g.cls == GC_X) {
                psi[i0] = a1;
                psi[i1] = a0;
            } else if (g.cls == GC_DIAG1) {
                psi[i0] = cmul(m0, a0);
                psi[i1] = cmul(m1, a1);
            } else if (g.cls == GC_DENSE1) {
                psi[i0] = cmac2(m0, a0, m1, a1);
                psi[i1] = cmac2(m2, a0, m3, a1);
            }
        }
    } else {
        const uint32_t lo = g.q0 < g.q1 ? g.q0 : g.q1, hi = g.q0 < g.q1 ? g.q1 : g.q0;
        const uint64_t b0 = 1ull << g.q0, b1 = 1ull << g.q1;
        for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < (1ull << (n - 2)); p += stride) {
            uint64_t i = p;
            i = ((i & ~((1ull << lo) - 1)) << 1) | (i & ((1ull << lo) - 1));
            i = ((i & ~((1ull << hi) - 1)) << 1) | (i & ((1ull << hi) - 1));
            const uint64_t idx[4] = {i, i | b0, i | b1, i | b0 | b1};
            float2 a[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) a[k] = psi[idx[k]];
            if (g.cls == GC_CX) {
                psi[idx[1]] = a[3];
                psi[idx[3]] = a[1];
            } else if (g.cls == GC_SWAP) {
                psi[idx[1]] = a[2];
                psi[idx[2]] = a[1];
            } else if (g.cls == GC_DIAG2) {
#pragma unroll
                for (int k = 0; k < 4; ++k) psi[idx[k]] = cmul(m16[5 * k], a[k]);
            } else if (g.cls == GC_DENSE2) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float2 acc = cmac2(m16[4 * k], a[0], m16[4 * k + 1], a[1]);
                    const float2 acc2 = cmac2(m16[4 * k + 2], a[2], m16[4 * k + 3], a[3]);
                    acc.x += acc2.x;
                    acc.y += acc2.y;
                    psi[idx[k]] = acc;
                }
            }
        }
    }
}

// Pauli error gate on a device state (Eq. (2)): X/Y permute the pair
// (i, i | 2^q), Z/Y apply the phase.
__global__ void pauli_kernel(float2 *psi, int n, uint32_t q, uint32_t code) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t bit = 1ull << q, lo = bit - 1;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < (1ull << (n - 1)); p += stride) {
        const uint64_t i0 = ((p & ~lo) << 1) | (p & lo), i1 = i0 | bit;
        const float2 a0 = psi[i0], a1 = psi[i1];
        if (code == 1) {
            psi[i0] = a1;
            psi[i1] = a0;
        } else if (code == 2) {
            psi[i1] = cneg(a1);
        } else if (code == 3) {
            psi[i0] = make_float2(a1.y, -a1.x);
            psi[i1] = make_float2(-a0.y, a0.x);
        }
    }
}

// Criterion partials of one state, one per block (grid-stride over amplitudes).
template <typename T>
__global__ void score_partials_kernel(const T *__restrict__ psi, const T *__restrict__ ref, int n, DCrit crit,
                                      Partial *partials) {
    __shared__ Partial red[32];
    Partial acc = empty_partial();
    const uint64_t N = 1ull << n;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x)
        accumulate(acc, crit, psi[i], ref, i);
    acc = block_reduce_partial(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void init_zero_state_kernel(void *psi, uint64_t N, int is_double) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        if (is_double)
            static_cast<double2 *>(psi)[i] = make_double2(i == 0 ? 1.0 : 0.0, 0.0);
        else
            static_cast<float2 *>(psi)[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
    }
}

// ------------------------------------------------------------- launchers ---

template <typename T> static void set_smem(const void *fn, size_t bytes) {
    if (bytes > 48 * 1024) ARSO_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

void launch_resident(const ResidentArgs &a, bool ideal, int precision, double bytes, cudaStream_t st) {
    ProfScope ps_(ARSO_K_RESIDENT, bytes, st);
    const uint32_t N = 1u << a.n;
    const int nt = (int)std::min<uint32_t>(256, std::max<uint32_t>(32, N / 2));
    if (precision == ARSO_C64) {
        const size_t smem = N * sizeof(float2);
        const void *fn = ideal ? (const void *)resident_ideal_kernel<float2> : (const void *)resident_kernel<float2>;
        set_smem<float2>(fn, smem);
        const unsigned grid = ideal ? 1u : (unsigned)std::min<uint64_t>(a.count, 152ull * 32);
        if (ideal) resident_ideal_kernel<float2><<<grid, nt, smem, st>>>(a);
        else resident_kernel<float2><<<grid, nt, smem, st>>>(a);
    } else {
        const size_t smem = N * sizeof(double2);
        const void *fn = ideal ? (const void *)resident_ideal_kernel<double2> : (const void *)resident_kernel<double2>;
        set_smem<double2>(fn, smem);
        const unsigned grid = ideal ? 1u : (unsigned)std::min<uint64_t>(a.count, 152ull * 32);
        if (ideal) resident_ideal_kernel<double2><<<grid, nt, smem, st>>>(a);
        else resident_kernel<double2><<<grid, nt, smem, st>>>(a);
    }
    ARSO_CUDA(cudaGetLastError());
}

void launch_pass(const PassArgs &a, bool last, int precision, uint32_t slots, double bytes, cudaStream_t st) {
    ProfScope ps_(last && !a.store_last ? ARSO_K_PASS_LAST : ARSO_K_PASS, bytes, st);
    const uint32_t tiles = 1u << (a.n - a.t);
    const int nt = 256;
    dim3 grid(tiles, slots);
    if (precision == ARSO_C64) {
        const size_t smem = (size_t(1) << a.t) * sizeof(float2);
        if (last) {
            set_smem<float2>((const void *)pass_kernel<float2, true>, smem);
            pass_kernel<float2, true><<<grid, nt, smem, st>>>(a);
        } else {
            set_smem<float2>((const void *)pass_kernel<float2, false>, smem);
            pass_kernel<float2, false><<<grid, nt, smem, st>>>(a);
        }
    } else {
        const size_t smem = (size_t(1) << a.t) * sizeof(double2);
        if (last) {
            set_smem<double2>((const void *)pass_kernel<double2, true>, smem);
            pass_kernel<double2, true><<<grid, nt, smem, st>>>(a);
        } else {
            set_smem<double2>((const void *)pass_kernel<double2, false>, smem);
            pass_kernel<double2, false><<<grid, nt, smem, st>>>(a);
        }
    }
    ARSO_CUDA(cudaGetLastError());
}

void launch_finish_partials(const Partial *partials, uint32_t tiles, uint32_t slots, const uint64_t *slot_traj,
                            const DCrit &crit, double *score, uint8_t *pass_flags, cudaStream_t st) {
    const unsigned grid = std::min<uint32_t>(slots, 152u * 8);
    ProfScope ps_(ARSO_K_REDUCE, 0.0, st);
    finish_partials_kernel<<<grid, 256, 0, st>>>(partials, tiles, slots, slot_traj, crit, score, pass_flags);
    ARSO_CUDA(cudaGetLastError());
}

void launch_fill_error_free(const uint32_t *first, uint64_t n_traj, const double *ref_score, double threshold,
                            double *score, uint8_t *pass_flags, cudaStream_t st) {
    if (!n_traj) return;
    const unsigned grid = (unsigned)std::min<uint64_t>((n_traj + 255) / 256, 152ull * 16);
    ProfScope ps_(ARSO_K_OTHER, 0.0, st);
    fill_error_free_kernel<<<grid, 256, 0, st>>>(first, n_traj, ref_score, threshold, score, pass_flags);
    ARSO_CUDA(cudaGetLastError());
}

void launch_gate_pairs(float2 *psi, int n, const DGate &g, const M16 &m, cudaStream_t st) {
    const uint64_t work = 1ull << (n - g.arity);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((work + 255) / 256, 152ull * 16));
    ProfScope ps_(ARSO_K_OTHER, 16.0 * (double)(1ull << n), st);
    gate_pairs_kernel<<<grid, 256, 0, st>>>(psi, n, g, m);
    ARSO_CUDA(cudaGetLastError());
}

void launch_pauli(float2 *psi, int n, uint32_t q, uint32_t code, cudaStream_t st) {
    const uint64_t work = 1ull << (n - 1);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((work + 255) / 256, 152ull * 16));
    ProfScope ps_(ARSO_K_OTHER, 16.0 * (double)(1ull << n), st);
    pauli_kernel<<<grid, 256, 0, st>>>(psi, n, q, code);
    ARSO_CUDA(cudaGetLastError());
}

uint32_t launch_score_partials(const void *psi, const void *ref, int n, int precision, const DCrit &crit,
                               Partial *partials, uint32_t max_blocks, cudaStream_t st) {
    const uint64_t N = 1ull << n;
    const uint32_t blocks = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((N + 255) / 256, max_blocks));
    ProfScope ps_(ARSO_K_REDUCE, (double)N * (precision == ARSO_C64 ? 8 : 16), st);
    if (precision == ARSO_C64)
        score_partials_kernel<float2><<<blocks, 256, 0, st>>>(static_cast<const float2 *>(psi),
                                                              static_cast<const float2 *>(ref), n, crit, partials);
    else
        score_partials_kernel<double2><<<blocks, 256, 0, st>>>(static_cast<const double2 *>(psi),
                                                               static_cast<const double2 *>(ref), n, crit, partials);
    ARSO_CUDA(cudaGetLastError());
    return blocks;
}

void launch_init_zero_state(void *psi, int n, int precision, cudaStream_t st) {
    const uint64_t N = 1ull << n;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((N + 255) / 256, 152ull * 16));
    ProfScope ps_(ARSO_K_OTHER, 0.0, st);
    init_zero_state_kernel<<<grid, 256, 0, st>>>(psi, N, precision == ARSO_C128);
    ARSO_CUDA(cudaGetLastError());
}


// ------------------------------------------- single-error fidelity values ---
// For the fidelity criterion the final state with one Pauli error P on qubit q
// after gate g scores |<psi_g|P|psi_g>|^2 (the rest of the circuit is unitary
// and maps psi_g to psi_R), so the exhaustive analysis needs only the Pauli
// expectations <X_q>, <Z_q>, <Y_q> of the error-free state after every gate.
// Per pair (a0, a1) along bit q: Z contributes |a0|^2 - |a1|^2, X
// 2 Re(conj(a0) a1), Y 2 Im(conj(a0) a1). FP64 accumulation.
template <typename T>
__device__ __forceinline__ void pauli_terms(T a0, T a1, double &x, double &z, double &y) {
    const double r0 = a0.x, i0 = a0.y, r1 = a1.x, i1 = a1.y;
    z += r0 * r0 + i0 * i0 - r1 * r1 - i1 * i1;
    x += 2.0 * (r0 * r1 + i0 * i1);
    y += 2.0 * (r0 * i1 - i0 * r1);
}

// block-wide sum of three doubles; every thread gets the result
__device__ __forceinline__ void block_sum3(double &x, double &z, double &y, double (*red)[32]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        z += __shfl_down_sync(0xffffffffu, z, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[0][warp] = x, red[1][warp] = z, red[2][warp] = y;
    __syncthreads();
    x = z = y = 0.0;
    for (int w = 0; w < nw; ++w) x += red[0][w], z += red[1][w], y += red[2][w];
}

// Whole state in one CTA's shared memory: CTA b starts from cached error-free
// checkpoint b (engine position seg_pos[b]), applies the gates up to
// seg_pos[b + 1] in engine order and writes (<X>, <Z>, <Y>) of each gate's
// qubits after it to out[3 * location]; the segments run in parallel.
template <typename T>
__global__ void expect_resident_kernel(const DGate *__restrict__ gates, const T *__restrict__ mats, int n,
                                       const T *__restrict__ ckpt, const uint32_t *__restrict__ seg_pos,
                                       const uint32_t *__restrict__ first_loc, double *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3][32];
    T *s = reinterpret_cast<T *>(smem_raw);
    const uint32_t N = 1u << n;
    const T *src = ckpt + (size_t)blockIdx.x * N;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) s[i] = src[i];
    __syncthreads();
    const uint32_t pe = seg_pos[blockIdx.x + 1];
    for (uint32_t pos = seg_pos[blockIdx.x]; pos < pe; ++pos) {
        const DGate g = gates[pos];
        tile_gate(s, n, g, mats + g.mat);
        __syncthreads();
        for (int j = 0; j < g.arity; ++j) {
            const uint32_t q = j ? g.q1 : g.q0, bit = 1u << q;
            double x = 0.0, z = 0.0, y = 0.0;
            for (uint32_t p = threadIdx.x; p < N / 2; p += blockDim.x) {
                const uint32_t i0 = insert_zero(p, q);
                pauli_terms(s[i0], s[i0 | bit], x, z, y);
            }
            block_sum3(x, z, y, red);
            if (threadIdx.x == 0) {
                double *o = out + 3 * (size_t)(first_loc[pos] + j);
                o[0] = x;
                o[1] = z;
                o[2] = y;
            }
        }
    }
}

void launch_expect_resident(const DGate *gates, const void *mats, int n, int precision, const void *ckpt,
                            const uint32_t *seg_pos, uint32_t n_seg, const uint32_t *first_loc, double *out,
                            cudaStream_t st) {
    if (!n_seg) return;
    const size_t smem = (size_t(1) << n) * (precision == ARSO_C64 ? 8 : 16);
    ProfScope ps_(ARSO_K_OTHER, (double)n_seg * smem, st);
    if (precision == ARSO_C64) {
        if (smem > 48 * 1024)
            ARSO_CUDA(cudaFuncSetAttribute(expect_resident_kernel<float2>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        expect_resident_kernel<float2><<<n_seg, 512, smem, st>>>(gates, static_cast<const float2 *>(mats), n,
                                                                 static_cast<const float2 *>(ckpt), seg_pos,
                                                                 first_loc, out);
    } else {
        if (smem > 48 * 1024)
            ARSO_CUDA(cudaFuncSetAttribute(expect_resident_kernel<double2>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        expect_resident_kernel<double2><<<n_seg, 512, smem, st>>>(gates, static_cast<const double2 *>(mats), n,
                                                                  static_cast<const double2 *>(ckpt), seg_pos,
                                                                  first_loc, out);
    }
    ARSO_CUDA(cudaGetLastError());
}

// One gate on a complex64 state in HBM fused with the Pauli expectations of its
// qubits on the amplitudes it just wrote (the pairs along each of the gate's
// qubits lie inside the pair or quad a thread updates). Per-thread FP32 sums,
// FP64 block sums; block b of position `pos` writes partials[(pos * blocks + b) * 6
// + 3 j + {0, 1, 2}] = (X, Z, Y) terms of the gate's j-th qubit.
__device__ __forceinline__ void pauli_terms_f(float2 a0, float2 a1, float &x, float &z, float &y) {
    z += a0.x * a0.x + a0.y * a0.y - a1.x * a1.x - a1.y * a1.y;
    x += 2.f * (a0.x * a1.x + a0.y * a1.y);
    y += 2.f * (a0.x * a1.y - a0.y * a1.x);
}

// apply the one-qubit class to a pair
__device__ __forceinline__ void gate1(const DGate &g, float2 m0, float2 m1, float2 m2, float2 m3, float2 &a0,
                                      float2 &a1) {
    if (g.cls == GC_X) {
        const float2 t = a0;
        a0 = a1;
        a1 = t;
    } else if (g.cls == GC_DIAG1) {
        a0 = cmul(m0, a0);
        a1 = cmul(m1, a1);
    } else if (g.cls == GC_DENSE1) {
        const float2 b0 = cmac2(m0, a0, m1, a1), b1 = cmac2(m2, a0, m3, a1);
        a0 = b0;
        a1 = b1;
    }
}

// apply the two-qubit class to a quad (local index bit(q0) + 2 bit(q1))
__device__ __forceinline__ void gate2(const DGate &g, const float2 *m16, float2 (&a)[4]) {
    float2 b[4];
    if (g.cls == GC_CX) {
        b[0] = a[0], b[1] = a[3], b[2] = a[2], b[3] = a[1];
    } else if (g.cls == GC_SWAP) {
        b[0] = a[0], b[1] = a[2], b[2] = a[1], b[3] = a[3];
    } else if (g.cls == GC_DIAG2) {
#pragma unroll
        for (int k = 0; k < 4; ++k) b[k] = cmul(m16[5 * k], a[k]);
    } else {  // GC_DENSE2
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 acc = cmac2(m16[4 * k], a[0], m16[4 * k + 1], a[1]);
            const float2 acc2 = cmac2(m16[4 * k + 2], a[2], m16[4 * k + 3], a[3]);
            acc.x += acc2.x;
            acc.y += acc2.y;
            b[k] = acc;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = b[k];
}

// UNROLL pairs (quads) per thread and round: every load of a round is issued before
// the first store, so that more of them are in flight (the pairs are disjoint)
constexpr int GE_UNROLL = 4;

__global__ void gate_expect_kernel(float2 *psi, int n, DGate g, M16 mm, double *partials) {
    __shared__ double red[3][32];
    const float2 *m16 = mm.m;
    const float2 m0 = m16[0], m1 = m16[1], m2 = m16[2], m3 = m16[3];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const bool write = g.cls != GC_NOP;
    float x0 = 0.f, z0 = 0.f, y0 = 0.f, x1 = 0.f, z1 = 0.f, y1 = 0.f;
    if (g.arity == 1) {
        const uint64_t bit = 1ull << g.q0, lo = bit - 1, half = 1ull << (n - 1);
        for (uint64_t p0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p0 < half; p0 += GE_UNROLL * stride) {
            float2 a0[GE_UNROLL], a1[GE_UNROLL];
            uint64_t i0[GE_UNROLL];
#pragma unroll
            for (int u = 0; u < GE_UNROLL; ++u) {
                const uint64_t p = p0 + u * stride;
                i0[u] = ((p & ~lo) << 1) | (p & lo);
                if (p < half) a0[u] = psi[i0[u]], a1[u] = psi[i0[u] | bit];
            }
#pragma unroll
            for (int u = 0; u < GE_UNROLL; ++u) {
                if (p0 + u * stride >= half) break;
                gate1(g, m0, m1, m2, m3, a0[u], a1[u]);
                if (write) psi[i0[u]] = a0[u], psi[i0[u] | bit] = a1[u];
                pauli_terms_f(a0[u], a1[u], x0, z0, y0);
            }
        }
    } else {
        const uint32_t lo = g.q0 < g.q1 ? g.q0 : g.q1, hi = g.q0 < g.q1 ? g.q1 : g.q0;
        const uint64_t b0 = 1ull << g.q0, b1 = 1ull << g.q1, quarter = 1ull << (n - 2);
        for (uint64_t p0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p0 < quarter; p0 += 2 * stride) {
            float2 a[2][4];
            uint64_t base[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                uint64_t i = p0 + u * stride;
                if (i >= quarter) continue;
                i = ((i & ~((1ull << lo) - 1)) << 1) | (i & ((1ull << lo) - 1));
                i = ((i & ~((1ull << hi) - 1)) << 1) | (i & ((1ull << hi) - 1));
                base[u] = i;
                a[u][0] = psi[i], a[u][1] = psi[i | b0], a[u][2] = psi[i | b1], a[u][3] = psi[i | b0 | b1];
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (p0 + u * stride >= quarter) break;
                if (write) {
                    gate2(g, m16, a[u]);
                    const uint64_t i = base[u];
                    psi[i] = a[u][0], psi[i | b0] = a[u][1], psi[i | b1] = a[u][2], psi[i | b0 | b1] = a[u][3];
                }
                pauli_terms_f(a[u][0], a[u][1], x0, z0, y0);  // along q0
                pauli_terms_f(a[u][2], a[u][3], x0, z0, y0);
                pauli_terms_f(a[u][0], a[u][2], x1, z1, y1);  // along q1
                pauli_terms_f(a[u][1], a[u][3], x1, z1, y1);
            }
        }
    }
    double *out = partials + (size_t)blockIdx.x * 6;
    double x = x0, z = z0, y = y0;
    block_sum3(x, z, y, red);
    if (threadIdx.x == 0) out[0] = x, out[1] = z, out[2] = y;
    if (g.arity == 2) {
        x = x1, z = z1, y = y1;
        block_sum3(x, z, y, red);
        if (threadIdx.x == 0) out[3] = x, out[4] = z, out[5] = y;
    }
}

// Adds the block partials of `count` gate positions in a fixed order: block k
// reduces position k and writes (X, Z, Y) of its qubits to out3[3 * (loc[k] + j)].
__global__ void gate_expect_reduce_kernel(const double *__restrict__ partials, uint32_t blocks,
                                          const uint32_t *__restrict__ loc, const uint8_t *__restrict__ arity,
                                          double *out3) {
    __shared__ double red[6][256];
    const double *p = partials + (size_t)blockIdx.x * blocks * 6;
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (uint32_t b = threadIdx.x; b < blocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] += p[(size_t)b * 6 + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) red[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
#pragma unroll
            for (int k = 0; k < 6; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3u * arity[blockIdx.x]) out3[3 * (size_t)loc[blockIdx.x] + threadIdx.x] = red[threadIdx.x][0];
}

void launch_gate_expect(float2 *psi, int n, const DGate &g, const M16 &m, double *partials, cudaStream_t st) {
    const uint32_t blocks = expect_hbm_blocks(n);
    ProfScope ps_(ARSO_K_OTHER, 16.0 * (double)(1ull << n), st);
    gate_expect_kernel<<<blocks, 256, 0, st>>>(psi, n, g, m, partials);
    ARSO_CUDA(cudaGetLastError());
}

void launch_gate_expect_reduce(const double *partials, uint32_t count, uint32_t blocks, const uint32_t *loc,
                               const uint8_t *arity, double *out3, cudaStream_t st) {
    if (!count) return;
    ProfScope ps_(ARSO_K_REDUCE, 48.0 * count * blocks, st);
    gate_expect_reduce_kernel<<<count, 256, 0, st>>>(partials, blocks, loc, arity, out3);
    ARSO_CUDA(cudaGetLastError());
}

// ------------------------------------------- single-error outcome values ---
// For a rank-1 criterion |<tau|psi>|^2 (outcome probability: tau = |t>) the final
// state with one Pauli error P on qubit q after gate g scores |<phi_g|P|psi_g>|^2,
// where psi_g is the error-free state after gate g and phi_g = W^dagger tau for the
// error-free rest W of the circuit (the backward state). Both are carried backward
// from (psi_R, tau) with the adjoint gates: at each engine position the cross terms
// of the gate's qubits are taken, then the gate is undone on both states.
// Per pair (a0, a1) of psi and (b0, b1) of phi along bit q (Eq. (2) for P):
//   <phi|X|psi> += conj(b0) a1 + conj(b1) a0
//   <phi|Z|psi> += conj(b0) a0 - conj(b1) a1
//   <phi|Y|psi> += -i conj(b0) a1 + i conj(b1) a0
// stored as (Re X, Im X, Re Z, Im Z, Re Y, Im Y).
template <typename T, typename A>
__device__ __forceinline__ void cross_terms(T a0, T a1, T b0, T b1, A (&c)[6]) {
    const A ar0 = a0.x, ai0 = a0.y, ar1 = a1.x, ai1 = a1.y, br0 = b0.x, bi0 = b0.y, br1 = b1.x, bi1 = b1.y;
    // conj(b) a = (br ar + bi ai) + i (br ai - bi ar)
    const A r01 = br0 * ar1 + bi0 * ai1, i01 = br0 * ai1 - bi0 * ar1;
    const A r10 = br1 * ar0 + bi1 * ai0, i10 = br1 * ai0 - bi1 * ar0;
    const A r00 = br0 * ar0 + bi0 * ai0, i00 = br0 * ai0 - bi0 * ar0;
    const A r11 = br1 * ar1 + bi1 * ai1, i11 = br1 * ai1 - bi1 * ar1;
    c[0] += r01 + r10;
    c[1] += i01 + i10;
    c[2] += r00 - r11;
    c[3] += i00 - i11;
    c[4] += i01 - i10;  // -i (r01 + i i01) + i (r10 + i i10)
    c[5] += r10 - r01;
}

// block-wide sum of six doubles; every thread gets the result
__device__ __forceinline__ void block_sum6(double (&v)[6], double (*red)[32]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) red[k][warp] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        v[k] = 0.0;
        for (int w = 0; w < nw; ++w) v[k] += red[k][w];
    }
}

// Whole circuit in one CTA: psi and phi in shared memory; adj[pos] is the adjoint
// of the gate at engine position pos (global qubits, matrices in mats).
template <typename T>
__global__ void dual_expect_resident_kernel(const DGate *__restrict__ adj, const T *__restrict__ mats, uint32_t G,
                                            int n, const T *__restrict__ psi_R, uint64_t target,
                                            const uint32_t *__restrict__ first_loc, double *__restrict__ out6) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[6][32];
    const uint32_t N = 1u << n;
    T *s = reinterpret_cast<T *>(smem_raw);
    T *f = s + N;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
        s[i] = psi_R[i];
        T z;
        z.x = i == target ? 1 : 0;
        z.y = 0;
        f[i] = z;
    }
    __syncthreads();
    for (uint32_t pos = G; pos-- > 0;) {
        const DGate g = adj[pos];
        for (int j = 0; j < g.arity; ++j) {
            const uint32_t q = j ? g.q1 : g.q0, bit = 1u << q;
            double c[6] = {0, 0, 0, 0, 0, 0};
            for (uint32_t p = threadIdx.x; p < N / 2; p += blockDim.x) {
                const uint32_t i0 = insert_zero(p, q);
                cross_terms(s[i0], s[i0 | bit], f[i0], f[i0 | bit], c);
            }
            block_sum6(c, red);  // its barriers also end this round's reads of s and f
            if (threadIdx.x == 0) {
                double *o = out6 + 6 * (size_t)(first_loc[pos] + j);
#pragma unroll
                for (int k = 0; k < 6; ++k) o[k] = c[k];
            }
        }
        if (g.cls != GC_NOP) {
            __syncthreads();
            tile_gate(s, n, g, mats + g.mat);
            tile_gate(f, n, g, mats + g.mat);
            __syncthreads();
        }
    }
}

void launch_dual_expect_resident(const DGate *adj, const void *mats, uint32_t G, int n, int precision,
                                 const void *psi_R, uint64_t target, const uint32_t *first_loc, double *out6,
                                 cudaStream_t st) {
    const size_t smem = (size_t(2) << n) * (precision == ARSO_C64 ? 8 : 16);
    ProfScope ps_(ARSO_K_OTHER, (double)smem, st);
    if (precision == ARSO_C64) {
        if (smem > 48 * 1024)
            ARSO_CUDA(cudaFuncSetAttribute(dual_expect_resident_kernel<float2>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        dual_expect_resident_kernel<float2><<<1, 512, smem, st>>>(adj, static_cast<const float2 *>(mats), G, n,
                                                                  static_cast<const float2 *>(psi_R), target,
                                                                  first_loc, out6);
    } else {
        if (smem > 48 * 1024)
            ARSO_CUDA(cudaFuncSetAttribute(dual_expect_resident_kernel<double2>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        dual_expect_resident_kernel<double2><<<1, 512, smem, st>>>(adj, static_cast<const double2 *>(mats), G, n,
                                                                   static_cast<const double2 *>(psi_R), target,
                                                                   first_loc, out6);
    }
    ARSO_CUDA(cudaGetLastError());
}

// The same backward step on complex64 states in HBM, one launch per gate: each
// thread takes the cross terms of its pairs (quads) before undoing the gate on
// them. Per-thread FP32 sums, FP64 block partials: block b of a position writes
// partials[b * 12 + 6 j + k] for the gate's j-th qubit.
__global__ void dual_gate_expect_kernel(float2 *psi, float2 *phi, int n, DGate g, M16 mm, double *partials) {
    __shared__ double red[6][32];
    const float2 *m16 = mm.m;
    const float2 m0 = m16[0], m1 = m16[1], m2 = m16[2], m3 = m16[3];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const bool write = g.cls != GC_NOP;
    float c0[6] = {0, 0, 0, 0, 0, 0}, c1[6] = {0, 0, 0, 0, 0, 0};
    if (g.arity == 1) {
        const uint64_t bit = 1ull << g.q0, lo = bit - 1, half = 1ull << (n - 1);
        for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < half; p += stride) {
            const uint64_t i0 = ((p & ~lo) << 1) | (p & lo), i1 = i0 | bit;
            float2 a0 = psi[i0], a1 = psi[i1], b0 = phi[i0], b1 = phi[i1];
            cross_terms(a0, a1, b0, b1, c0);
            if (write) {
                gate1(g, m0, m1, m2, m3, a0, a1);
                gate1(g, m0, m1, m2, m3, b0, b1);
                psi[i0] = a0, psi[i1] = a1, phi[i0] = b0, phi[i1] = b1;
            }
        }
    } else {
        const uint32_t lo = g.q0 < g.q1 ? g.q0 : g.q1, hi = g.q0 < g.q1 ? g.q1 : g.q0;
        const uint64_t b0 = 1ull << g.q0, b1 = 1ull << g.q1, quarter = 1ull << (n - 2);
        for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < quarter; p += stride) {
            uint64_t i = p;
            i = ((i & ~((1ull << lo) - 1)) << 1) | (i & ((1ull << lo) - 1));
            i = ((i & ~((1ull << hi) - 1)) << 1) | (i & ((1ull << hi) - 1));
            const uint64_t idx[4] = {i, i | b0, i | b1, i | b0 | b1};
            float2 a[4], b[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) a[k] = psi[idx[k]], b[k] = phi[idx[k]];
            cross_terms(a[0], a[1], b[0], b[1], c0);  // along q0
            cross_terms(a[2], a[3], b[2], b[3], c0);
            cross_terms(a[0], a[2], b[0], b[2], c1);  // along q1
            cross_terms(a[1], a[3], b[1], b[3], c1);
            if (write) {
                gate2(g, m16, a);
                gate2(g, m16, b);
#pragma unroll
                for (int k = 0; k < 4; ++k) psi[idx[k]] = a[k], phi[idx[k]] = b[k];
            }
        }
    }
    double v[6];
    double *out = partials + (size_t)blockIdx.x * 12;
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = c0[k];
    block_sum6(v, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) out[k] = v[k];
    if (g.arity == 2) {
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = c1[k];
        block_sum6(v, red);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < 6; ++k) out[6 + k] = v[k];
    }
}

// Adds the block partials of `count` positions in a fixed order: block k reduces
// position k and writes its qubits' six sums to out6[6 * (loc[k] + j)].
__global__ void dual_expect_reduce_kernel(const double *__restrict__ partials, uint32_t blocks,
                                          const uint32_t *__restrict__ loc, const uint8_t *__restrict__ arity,
                                          double *out6) {
    __shared__ double red[12][128];
    const double *p = partials + (size_t)blockIdx.x * blocks * 12;
    double v[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t b = threadIdx.x; b < blocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] += p[(size_t)b * 12 + k];
#pragma unroll
    for (int k = 0; k < 12; ++k) red[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
#pragma unroll
            for (int k = 0; k < 12; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 6u * arity[blockIdx.x]) out6[6 * (size_t)loc[blockIdx.x] + threadIdx.x] = red[threadIdx.x][0];
}

void launch_dual_gate_expect(float2 *psi, float2 *phi, int n, const DGate &g, const M16 &m, double *partials,
                             cudaStream_t st) {
    const uint32_t blocks = expect_hbm_blocks(n);
    ProfScope ps_(ARSO_K_OTHER, 32.0 * (double)(1ull << n), st);
    dual_gate_expect_kernel<<<blocks, 256, 0, st>>>(psi, phi, n, g, m, partials);
    ARSO_CUDA(cudaGetLastError());
}

void launch_dual_expect_reduce(const double *partials, uint32_t count, uint32_t blocks, const uint32_t *loc,
                               const uint8_t *arity, double *out6, cudaStream_t st) {
    if (!count) return;
    ProfScope ps_(ARSO_K_REDUCE, 96.0 * count * blocks, st);
    dual_expect_reduce_kernel<<<count, 128, 0, st>>>(partials, blocks, loc, arity, out6);
    ARSO_CUDA(cudaGetLastError());
}

uint32_t expect_hbm_blocks(int n) {
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(((1ull << (n - 1)) + 255) / 256, 152ull * 8));
}

}  // namespace arso
