// Learned surrogate of the success probability: a 33 -> 256 -> 256 -> 1 MLP
// trained on the GPU on pass flags produced by the trajectory simulator, and
// the surrogate-bracketed tolerable-rate search (Sec. IV-D, Monte Carlo
// branch: the surrogate proposes the bracket, plain trajectories verify it).
//
// Weights are bfloat16 (with FP32 masters for Adam); every product
// accumulates in FP32. The MLP costs ~1.5e5 FMA per row, negligible next to
// the trajectories that label it, so the kernels are plain tiled SIMT GEMMs.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <random>

#include "kernels.h"
#include "prof.h"
#include "umma.cuh"

namespace arso {

constexpr int IN = ARSO_SURROGATE_INPUTS, HID = 256;
constexpr size_t OFF_W1 = 0, OFF_B1 = OFF_W1 + IN * HID, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
                 OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID, N_PARAMS = OFF_B3 + 1;
static_assert(N_PARAMS == ARSO_SURROGATE_PARAMS, "parameter layout");

// ------------------------------------------------------------------ GEMM ---
// C[m, n] = epi( sum_k A(m, k) B(n, k) ) on the tensor cores (tcgen05, kind::f16):
// one CTA per 128 x 128 output tile, FP32 accumulator in tensor memory, K in
// blocks of 64 staged through two shared-memory buffers. A bfloat16 B operand with
// a tensor map comes by TMA; otherwise the CTA's threads read an operand with
// element strides, A(m, k) = A[m * sr + k * sk], and convert it on the way into
// shared memory: a bfloat16 operand goes in as it is; an FP32 operand is split
// into bfloat16 terms x = x0 + x1 + x2 + r, x0 = bf16(x), x1 = bf16(x - x0),
// x2 = bf16(x - x0 - x1), |r| <= 2^-27 |x|. Products of bfloat16 are exact in
// FP32 and the tile accumulates the terms A_i B_j with i + j <= 2 (three against
// bfloat16 weights, six for two FP32 operands); each dropped term is below about
// 2^-24 of its product, so the result is an FP32 product up to the accumulation.
// With gridDim.z > 1 each z takes one K chunk and writes its partial tile to
// C + z * M * ldc.
enum { EPI_NONE = 0, EPI_BIAS_RELU = 1, EPI_RELU_MASK = 3 };

constexpr int GM_BM = 128, GM_BN = 128, GM_BK = 64, GM_THREADS = 512;
constexpr int GM_WG = GM_THREADS / 128;  // warps sharing each 32-row lane quarter (column groups)
static_assert(GM_BN == GM_WG * 32, "one 32-column chunk per warp in the epilogue");
constexpr int GM_NT = HID / GM_BN;  // output tiles across a hidden layer (partial logits)
constexpr int GM_A_BYTES = GM_BM * GM_BK * 2, GM_B_BYTES = GM_BN * GM_BK * 2;
constexpr int GM_STAGE_BYTES = 2 * GM_A_BYTES + 2 * GM_B_BYTES;  // two planes of A and two of B
constexpr int GM_TILE_BYTES = 2 * GM_STAGE_BYTES;
constexpr int GM_SMEM = GM_TILE_BYTES + 64 + GM_WG * GM_BM * 4;  // + barriers, tmem slot, logit parts
constexpr uint32_t GM_IDESC = idesc_bf16_f32(GM_BM, GM_BN);

struct GemmOperand {
    const void *p;
    long sr, sk;                // element strides along the row (m or n) and along k
    int bf16;                   // 1: bfloat16 elements, 0: FP32 (split into bfloat16 terms)
    const CUtensorMap *tmap;    // B only, optional: the same bfloat16 matrix, K-major, for TMA
};

struct GemmArgs {
    CUtensorMap tmb;  // B by TMA (b_tma): 2-D map over (k, n), box of 8 k x 128 rows
    int b_tma;
    int M, N, K, k_chunk;
    GemmOperand a, b;
    float *C;  // NULL: no store (the fused logit is the only output)
    long ldc;
    int epi;
    const __nv_bfloat16 *bias;
    const float *mask;
    long ldm;
    const __nv_bfloat16 *w3;  // EPI_BIAS_RELU: z[blockIdx.x * M + m] = sum over this tile's n of relu(...)[m, n] w3[n]
    float *z;
    float *colsum;  // EPI_RELU_MASK: colsum[blockIdx.y * N + n] = sum of the tile's rows of column n
    unsigned *err;
    uint32_t wait_limit;  // polls per bounded wait
    uint32_t stall;       // failure-path test: arm the TMA barrier for B's bytes but issue no copy
};

__device__ unsigned g_gemm_err;

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

// Stage rows [r0, r0 + R) x k [k0, k0 + 64) of an operand (zero outside
// rows < r_end, k < k_end) as `terms` bfloat16 planes (1 for a bfloat16 operand).
// Shared layout of a plane: 16-byte unit (r, kc) holds k = 8 kc .. 8 kc + 7 of row r
// at unit ((r / 8) * 8 + kc) * 8 + r % 8, so each 8 x 8 core matrix is 128
// contiguous bytes, K-adjacent core matrices are 128 bytes apart and row groups 1024.
__device__ __forceinline__ float bf16_bits_to_float(uint32_t packed, int half) {
    return __uint_as_float(((packed >> (16 * half)) & 0xFFFFu) << 16);
}

constexpr int GM_UNITS = GM_BM * 8 / GM_THREADS;  // 16-byte shared-memory units per thread and operand
static_assert(GM_BM == GM_BN, "both operand tiles stage the same number of units");

// unit j of this thread: row r and k chunk kc of the tile
__device__ __forceinline__ void unit_of(bool rows_contiguous, int j, int &r, int &kc) {
    const int u = threadIdx.x + j * GM_THREADS;
    if (rows_contiguous) {  // a warp reads 32 consecutive rows at each k
        r = u % GM_BM;
        kc = u / GM_BM;
    } else {  // eight consecutive rows per quarter warp, k chunks across the warp
        r = (u & 7) | ((u >> 6) << 3);
        kc = (u >> 3) & 7;
    }
}

__device__ __forceinline__ bool rows_contiguous(const GemmOperand &o) { return o.sr == 1 && o.sk != 1; }

// Read this thread's units of rows [r0, r0 + 128) x k [k0, k0 + 64) into registers
// (zero outside rows < r_end, k < k_end); every load is issued before any is used.
__device__ __forceinline__ void load_operand(const GemmOperand &o, int r0, int r_end, int k0, int k_end,
                                             float (&v)[GM_UNITS][8]) {
    const bool rc = rows_contiguous(o);
    // vector path: rows contiguous in k and 16-byte aligned, whole 8-element chunks
    const bool vec = o.sk == 1 && (o.sr & (o.bf16 ? 7 : 3)) == 0 && ((uintptr_t)o.p & 15) == 0;
#pragma unroll
    for (int j = 0; j < GM_UNITS; ++j) {
        int r, kc;
        unit_of(rc, j, r, kc);
        const int gr = r0 + r, gk = k0 + kc * 8;
#pragma unroll
        for (int i = 0; i < 8; ++i) v[j][i] = 0.f;
        if (gr >= r_end) continue;
        const long base = (long)gr * o.sr;
        if (vec && o.bf16 && gk + 8 <= k_end) {
            const uint4 x = __ldg(reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(o.p) + base + gk));
            const uint32_t xw[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) v[j][i] = bf16_bits_to_float(xw[i >> 1], i & 1);
        } else if (vec && gk + 8 <= k_end) {
            const float4 *q = reinterpret_cast<const float4 *>(static_cast<const float *>(o.p) + base + gk);
            const float4 x0 = __ldg(q), x1 = __ldg(q + 1);
            v[j][0] = x0.x, v[j][1] = x0.y, v[j][2] = x0.z, v[j][3] = x0.w;
            v[j][4] = x1.x, v[j][5] = x1.y, v[j][6] = x1.z, v[j][7] = x1.w;
        } else if (o.bf16) {
            const __nv_bfloat16 *p = static_cast<const __nv_bfloat16 *>(o.p);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (gk + i < k_end) v[j][i] = __bfloat162float(p[base + (long)(gk + i) * o.sk]);
        } else {
            const float *p = static_cast<const float *>(o.p);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (gk + i < k_end) v[j][i] = __ldg(p + base + (long)(gk + i) * o.sk);
        }
    }
}

// Write the registers of load_operand as `terms` bfloat16 planes (1 for a bfloat16
// operand). Shared layout of a plane: 16-byte unit (r, kc) holds k = 8 kc .. 8 kc + 7
// of row r at unit ((r / 8) * 8 + kc) * 8 + r % 8, so each 8 x 8 core matrix is 128
// contiguous bytes, K-adjacent core matrices are 128 bytes apart and row groups 1024.
__device__ __forceinline__ void store_operand(const GemmOperand &o, float (&v)[GM_UNITS][8], int terms, uint4 *p0,
                                              uint4 *p1, uint4 *p2) {
    const bool rc = rows_contiguous(o);
    uint4 *planes[3] = {p0, p1, p2};
#pragma unroll
    for (int j = 0; j < GM_UNITS; ++j) {
        int r, kc;
        unit_of(rc, j, r, kc);
        const int idx = ((r >> 3) * 8 + kc) * 8 + (r & 7);
        float x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = v[j][i];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (t >= terms) break;
            uint4 q;
            q.x = pack_bf16(x[0], x[1]);
            q.y = pack_bf16(x[2], x[3]);
            q.z = pack_bf16(x[4], x[5]);
            q.w = pack_bf16(x[6], x[7]);
            planes[t][idx] = q;
            const uint32_t qw[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] -= bf16_bits_to_float(qw[i >> 1], i & 1);  // exact in FP32
        }
    }
}

// One instantiation per operand route, so that each holds only its own staging code:
// B_MODE 0: bfloat16 B by TMA; 1: bfloat16 B through the threads; 2: FP32 B through
// the threads (six term products, one buffer). A is FP32 through the threads.
template <int B_MODE>
__global__ void __launch_bounds__(GM_THREADS, 1) umma_gemm_kernel(const __grid_constant__ GemmArgs a) {
    constexpr bool B_TMA = B_MODE == 0;
    extern __shared__ __align__(1024) uint8_t gm_smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(gm_smem + GM_TILE_BYTES);        // buffer free again (MMAs done)
    uint64_t *full = reinterpret_cast<uint64_t *>(gm_smem + GM_TILE_BYTES + 16);  // B tile landed (TMA)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gm_smem + GM_TILE_BYTES + 32);
    float *s_z = reinterpret_cast<float *>(gm_smem + GM_TILE_BYTES + 64);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * GM_BM, n0 = blockIdx.x * GM_BN;
    const int kz0 = blockIdx.z * a.k_chunk, kz1 = min(a.K, kz0 + a.k_chunk);
    const int nkb = (kz1 - kz0 + GM_BK - 1) / GM_BK;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        mbar_init(full, 1);
        mbar_init(full + 1, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, GM_BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // bfloat16 terms per operand (1: a bfloat16 operand, 3: FP32); two FP32 operands
    // take six planes and a single buffer, the other cases two buffers
    constexpr int ta = 3, tb = B_MODE == 2 ? 3 : 1;
    constexpr int nst = tb == 3 ? 1 : 2;
    uint32_t parity[2] = {0u, 0u}, fparity[2] = {0u, 0u};
    bool pending[2] = {false, false};
    bool bad = false;
    // thread 0 only: a stage whose TMA copies were issued and not yet seen to land,
    // and the barrier phase they complete (drained before the CTA returns)
    bool tma_inflight[2] = {false, false};
    uint32_t tma_phase[2] = {0u, 0u};
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % nst;
        if (pending[s]) {  // the MMAs of block kb - nst read this buffer
            bad |= !mbar_wait_bounded(bar + s, parity[s], a.wait_limit);
            parity[s] ^= 1u;
            pending[s] = false;
        }
        if (__syncthreads_or(bad)) {
            bad = true;
            break;
        }
        uint8_t *st = gm_smem + s * GM_STAGE_BYTES;
        uint4 *pa[3], *pb[3];
        if (nst == 2) {  // per buffer: A0 | A1 | B0 | B1, with A2 in B1's place when B is bfloat16
            pa[0] = reinterpret_cast<uint4 *>(st);
            pa[1] = reinterpret_cast<uint4 *>(st + GM_A_BYTES);
            pb[0] = reinterpret_cast<uint4 *>(st + 2 * GM_A_BYTES);
            pb[1] = pa[2] = reinterpret_cast<uint4 *>(st + 2 * GM_A_BYTES + GM_B_BYTES);
            pb[2] = pb[1];
        } else {  // one buffer: A0 | A1 | A2 | B0 | B1 | B2
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                pa[t] = reinterpret_cast<uint4 *>(st + t * GM_A_BYTES);
                pb[t] = reinterpret_cast<uint4 *>(st + 3 * GM_A_BYTES + t * GM_B_BYTES);
            }
        }
        const int k0 = kz0 + kb * GM_BK;
        if (B_TMA && threadIdx.x == 0) {
            // B by TMA: one 8 k x 128 row box per k chunk, 2 KB apart, so that row
            // groups are 128 bytes apart and k chunks 2048 (the descriptor below)
            mbar_arrive_expect_tx(full + s, GM_B_BYTES);
            if (!a.stall) {
#pragma unroll
                for (int c = 0; c < GM_BK / 8; ++c)
                    tma_load_2d(reinterpret_cast<uint8_t *>(pb[0]) + c * (GM_BN * 16), &a.tmb, k0 + 8 * c, n0,
                                full + s);
                tma_inflight[s] = true;
                tma_phase[s] = fparity[s];
            }
        }
        {
            float va[GM_UNITS][8];
            load_operand(a.a, m0, a.M, k0, kz1, va);
            if (!B_TMA) {
                float vb[GM_UNITS][8];
                load_operand(a.b, n0, a.N, k0, kz1, vb);
                store_operand(a.b, vb, tb, pb[0], pb[1], pb[2]);
            }
            store_operand(a.a, va, ta, pa[0], pa[1], pa[2]);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            bool landed = true;
            if (B_TMA) {
                landed = mbar_wait_bounded(full + s, fparity[s], a.wait_limit);
                if (landed) tma_inflight[s] = false;
                bad |= !landed;
            }
            tc_fence_after();
            uint32_t sa[3], sb[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) sa[t] = smem_u32(pa[t]), sb[t] = smem_u32(pb[t]);
            // thread-staged planes: k chunks 128 bytes apart, row groups 1024
            constexpr uint32_t b_lbo = B_TMA ? GM_BN * 16 : 128, b_sbo = B_TMA ? 128 : 1024;
#pragma unroll 1
            for (int k = 0; k < GM_BK / 16 && landed; ++k) {  // 16 k per MMA: two core matrices along K
                // the terms A_i B_j with i + j <= 2, largest first
                for (int i = 0; i < ta; ++i)
                    for (int j = 0; j < tb && i + j <= 2; ++j)
                        umma_bf16(tmem, smem_desc_kmajor(sa[i] + k * 256, 128, 1024),
                                  smem_desc_kmajor(sb[j] + k * 2 * b_lbo, b_lbo, b_sbo), GM_IDESC,
                                  (kb > 0 || k > 0 || i > 0 || j > 0) ? 1u : 0u);
            }
            umma_commit(bar + s);  // with no MMA issued it arrives at once
        }
        if (B_TMA) fparity[s] ^= 1u;
        pending[s] = true;
    }
    for (int s = 0; s < 2; ++s)
        if (pending[s]) {
            bad |= !mbar_wait_bounded(bar + s, parity[s], a.wait_limit);
            parity[s] ^= 1u;
        }
    bad = __syncthreads_or(bad) || nkb == 0;
    if (bad && B_TMA && threadIdx.x == 0) {
        // a wait gave up: let copies still in flight into this CTA's shared memory
        // land (again a bounded wait) before the memory is reused or released
        for (int s = 0; s < 2; ++s)
            if (tma_inflight[s]) (void)mbar_wait_bounded(full + s, tma_phase[s], a.wait_limit);
    }
    __syncthreads();
    tc_fence_after();

    if (!bad) {
        // warp w reads lanes (rows) 32 (w mod 4) .. +31 and the 32 columns of group w / 4;
        // the 32 x 32 chunk turns through a padded tile in the (now idle) operand buffers
        // so that each store, and each mask read, is one row segment of the warp
        const int q = warp & 3, h = warp >> 2;
        const int mw = m0 + q * 32, nb = n0 + h * 32, n = nb + lane;
        float mk[32];
        if (a.epi == EPI_RELU_MASK) {  // all 32 mask loads in flight before the first use
#pragma unroll
            for (int r = 0; r < 32; ++r)
                mk[r] = (n < a.N && mw + r < a.M) ? __ldg(a.mask + (size_t)(mw + r) * a.ldm + n) : 0.f;
        }
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 32), v);
        float zacc = 0.f;
        if (a.epi == EPI_BIAS_RELU) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (nb + j >= a.N) break;
                v[j] = fmaxf(v[j] + __bfloat162float(a.bias[nb + j]), 0.f);
                if (a.z) zacc = fmaf(v[j], __bfloat162float(a.w3[nb + j]), zacc);
            }
        }
        float *C = a.C ? a.C + (size_t)blockIdx.z * a.M * a.ldc : nullptr;
        if (C) {
            float(*T)[33] = reinterpret_cast<float(*)[33]>(gm_smem + warp * (32 * 33 * 4));
#pragma unroll
            for (int j = 0; j < 32; ++j) T[lane][j] = v[j];
            __syncwarp();
            float cs = 0.f;
            if (n < a.N) {
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    if (mw + r < a.M) {
                        float x = T[r][lane];
                        if (a.epi == EPI_RELU_MASK) x = mk[r] > 0.f ? x : 0.f;
                        C[(size_t)(mw + r) * a.ldc + n] = x;
                        cs += x;
                    }
                }
            }
            if (a.colsum) {  // the four row quarters of each column, added in order
                s_z[h * GM_BM + q * 32 + lane] = cs;
                __syncthreads();
                if (q == 0 && n < a.N) {
                    const float *c4 = s_z + h * GM_BM + lane;
                    a.colsum[(size_t)blockIdx.y * a.N + n] = ((c4[0] + c4[32]) + c4[64]) + c4[96];
                }
            }
        }
        if (a.z) {
            s_z[h * GM_BM + q * 32 + lane] = zacc;
            __syncthreads();
            if (threadIdx.x < GM_BM && m0 + (int)threadIdx.x < a.M) {
                float zs = s_z[threadIdx.x];
#pragma unroll
                for (int g = 1; g < GM_WG; ++g) zs += s_z[g * GM_BM + threadIdx.x];
                a.z[(size_t)blockIdx.x * a.M + m0 + threadIdx.x] = zs;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_free(tmem, GM_BN);
    }
    if (bad && nkb > 0 && threadIdx.x == 0) atomicOr(a.err ? a.err : &g_gemm_err, 1u);
}

// set by arso_debug_stall_next_gemm: the next GEMM with a TMA operand is made to give up
static std::atomic<bool> g_stall_next_gemm{false};

// C = epi(A B^T) for the operands above. With `part` set (weight gradients, K =
// batch rows) the K range is cut into chunks of at least 256 rows, at most about 64
// of them, and chunk z writes its M x N partial to part + z * M * N; the caller adds
// the chunks in order (grad_finish_kernel). Returns the number of chunks.
static int umma_gemm(int M, int N, int K, GemmOperand A, GemmOperand B, float *C, long ldc, int epi,
                     const __nv_bfloat16 *bias, const float *mask, long ldm, const __nv_bfloat16 *w3, float *z,
                     float *colsum, DeviceBuffer *part, cudaStream_t st) {
    static uint64_t attr_set = 0;  // one bit per device
    int dev = 0;
    ARSO_CUDA(cudaGetDevice(&dev));
    if (dev >= 64 || !(attr_set >> dev & 1)) {
        ARSO_CUDA(cudaFuncSetAttribute(umma_gemm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, GM_SMEM));
        ARSO_CUDA(cudaFuncSetAttribute(umma_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, GM_SMEM));
        ARSO_CUDA(cudaFuncSetAttribute(umma_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, GM_SMEM));
        if (dev < 64) attr_set |= 1ull << dev;
    }
    if (A.bf16) throw Error(ARSO_EINVAL, "tensor-core GEMM: A is an FP32 operand");
    GemmArgs g{};
    g.wait_limit = UMMA_WAIT_LIMIT;
    if (B.tmap && g_stall_next_gemm.exchange(false)) {  // failure-path test (arso_debug_stall_next_gemm)
        g.stall = 1;  // the TMA barrier waits for bytes that no copy delivers; nothing is in flight
        g.wait_limit = 1u << 12;
    }
    if (B.tmap) {
        if (!B.bf16) throw Error(ARSO_EINVAL, "tensor-core GEMM: TMA operands are bfloat16");
        g.tmb = *B.tmap;
        g.b_tma = 1;
    }
    g.M = M, g.N = N, g.K = K, g.a = A, g.b = B, g.ldc = ldc, g.epi = epi, g.bias = bias, g.mask = mask, g.ldm = ldm;
    g.w3 = w3, g.z = z, g.colsum = colsum, g.err = nullptr;
    int splits = 1;
    g.k_chunk = K;
    g.C = C;
    if (part) {
        g.k_chunk = std::max(256, ((K + 63) / 64 + 63) / 64 * 64);
        splits = (K + g.k_chunk - 1) / g.k_chunk;
        part->ensure((size_t)splits * M * N * sizeof(float));
        g.C = part->as<float>();
        g.ldc = N;
    }
    dim3 grid((N + GM_BN - 1) / GM_BN, (M + GM_BM - 1) / GM_BM, splits);
    const double bytes = (double)M * K * (A.bf16 ? 2 : 4) + (double)N * K * (B.bf16 ? 2 : 4) +
                         (double)M * N * 4 * splits * (g.C ? 1 : 0) + (mask ? (double)M * N * 4 : 0.0);
    ProfScope ps_(ARSO_K_GEMM, bytes, st, 2.0 * M * N * K);
    if (g.b_tma) umma_gemm_kernel<0><<<grid, GM_THREADS, GM_SMEM, st>>>(g);
    else if (B.bf16) umma_gemm_kernel<1><<<grid, GM_THREADS, GM_SMEM, st>>>(g);
    else umma_gemm_kernel<2><<<grid, GM_THREADS, GM_SMEM, st>>>(g);
    ARSO_CUDA(cudaGetLastError());
    return splits;
}

// raise ARSO_ETIMEOUT if a GEMM gave up waiting on its tensor-core work (call after a sync)
static void check_gemm_err() {
    unsigned e = 0;
    ARSO_CUDA(cudaMemcpyFromSymbol(&e, g_gemm_err, sizeof(e)));
    if (e) {
        const unsigned zero = 0;
        ARSO_CUDA(cudaMemcpyToSymbol(g_gemm_err, &zero, sizeof(zero)));
        throw Error(ARSO_ETIMEOUT, "tensor-core GEMM: a bounded wait on its MMAs gave up");
    }
}

// Output-layer backward over a chunk of DH2_ROWS rows per block, one thread per
// hidden unit k: dh2[i, k] = dz[i] w3[k] where h2[i, k] > 0 (else 0), and the chunk's
// partial sums of db2[k] = sum_i dh2[i, k], dW3[k] = sum_i h2[i, k] dz[i] and
// db3 = sum_i dz[i].
constexpr int DH2_ROWS = 64;
__global__ void __launch_bounds__(HID) dh2_kernel(const float *__restrict__ dz, const __nv_bfloat16 *__restrict__ w3,
                                                  const float *__restrict__ h2, int rows, float *dh2, float *p_b2,
                                                  float *p_w3, float *p_b3) {
    const int k = threadIdx.x, c = blockIdx.x;
    const int r0 = c * DH2_ROWS, r1 = min(rows, r0 + DH2_ROWS);
    const float w = __bfloat162float(w3[k]);
    float sb = 0.f, sw = 0.f, sz = 0.f;
#pragma unroll 8
    for (int r = r0; r < r1; ++r) {
        const float d = dz[r], h = h2[(size_t)r * HID + k];
        const float g = h > 0.f ? d * w : 0.f;
        dh2[(size_t)r * HID + k] = g;
        sb += g;
        sw = fmaf(h, d, sw);
        sz += d;
    }
    p_b2[(size_t)c * HID + k] = sb;
    p_w3[(size_t)c * HID + k] = sw;
    if (k == 0) p_b3[c] = sz;
}

// Where each parameter block's gradient partials are: count partial arrays of the
// block's size, `stride` floats apart, summed in order into g.
struct GradParts {
    const float *src[6];
    int count[6];
};

__global__ void grad_finish_kernel(GradParts p, float *__restrict__ g) {
    const size_t off[7] = {OFF_W1, OFF_B1, OFF_W2, OFF_B2, OFF_W3, OFF_B3, N_PARAMS};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N_PARAMS; i += (size_t)gridDim.x * blockDim.x) {
        int b = 0;
        while (i >= off[b + 1]) ++b;
        const size_t j = i - off[b], stride = off[b + 1] - off[b];
        const float *src = p.src[b];
        float s = 0.f;
#pragma unroll 8
        for (int c = 0; c < p.count[b]; ++c) s += src[c * stride + j];
        g[i] = s;
    }
}

// gather and standardise a batch: xb[i, c] = (x[idx[i], c] - mean[c]) / sd[c]
__global__ void gather_norm_kernel(const float *__restrict__ x, const uint32_t *__restrict__ idx, uint64_t base,
                                   int rows, const float *__restrict__ norm, float *xb) {
    const int i = blockIdx.x, c = threadIdx.x;
    if (i >= rows || c >= IN) return;
    const uint64_t r = idx ? idx[base + i] : base + i;
    xb[(long)i * IN + c] = (x[r * IN + c] - norm[c]) / norm[IN + c];
}

// logit of row i: the output tiles' partial sums, in order, plus the output bias
__device__ __forceinline__ float logit(const float *__restrict__ zp, int rows, const __nv_bfloat16 *b3, int i) {
    float z = zp[i];
#pragma unroll
    for (int t = 1; t < GM_NT; ++t) z += zp[(size_t)t * rows + i];
    return z + __bfloat162float(*b3);
}

// logit gradient of the mean BCE: dz = (sigmoid(z) - y) / B; loss += softplus(z) - y z
__global__ void bce_kernel(const float *__restrict__ zp, const __nv_bfloat16 *b3, const float *__restrict__ y,
                           const uint32_t *__restrict__ idx, uint64_t base, int rows, float inv_b, float *dz,
                           double *loss_sum) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < rows) {
        const uint64_t r = idx ? idx[base + i] : base + i;
        const float zi = logit(zp, rows, b3, i), yi = y[r];
        const float s = 1.f / (1.f + __expf(-zi));
        dz[i] = (s - yi) * inv_b;
        l = (double)(fmaxf(zi, 0.f) + log1pf(__expf(-fabsf(zi))) - yi * zi);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss_sum, l);
}

__global__ void sigmoid_kernel(const float *__restrict__ zp, const __nv_bfloat16 *b3, int n, float *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = 1.f / (1.f + __expf(-logit(zp, n, b3, i)));
}

// K-major bfloat16 copies of the weight matrices for the forward GEMMs' TMA loads:
// W1^T as 256 rows of T1_LD (>= 33) and W2^T as 256 rows of 256, both (n, k) row-major
constexpr int T1_LD = 64;
constexpr size_t T_W1 = 0, T_W2 = (size_t)HID * T1_LD, T_SIZE = T_W2 + (size_t)HID * HID;

__device__ __forceinline__ void store_bf16(__nv_bfloat16 *w16, __nv_bfloat16 *w16t, size_t i, float x) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    w16[i] = h;
    static_assert(OFF_W1 == 0, "W1 leads the parameter vector");
    if (i < OFF_B1) {
        const size_t j = i - OFF_W1;  // W1[k][n], k = j / HID
        w16t[T_W1 + (j % HID) * T1_LD + j / HID] = h;
    } else if (i >= OFF_W2 && i < OFF_B2) {
        const size_t j = i - OFF_W2;
        w16t[T_W2 + (j % HID) * HID + j / HID] = h;
    }
}

// Adam (Kingma & Ba 2015) on the FP32 masters; refresh the bfloat16 copies
__global__ void adam_kernel(float *w, __nv_bfloat16 *w16, __nv_bfloat16 *w16t, const float *__restrict__ g, float *m,
                            float *v, size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        store_bf16(w16, w16t, i, wi);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ w, __nv_bfloat16 *w16, __nv_bfloat16 *w16t, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        store_bf16(w16, w16t, i, w[i]);
}

// per-column sum and sum of squares (FP64) for the standardisation
__global__ void moments_kernel(const float *__restrict__ x, uint64_t n, double *out) {
    const int c = blockIdx.x;
    double s = 0, q = 0;
    for (uint64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double v = x[r * IN + c];
        s += v;
        q += v * v;
    }
    __shared__ double rs[256], rq[256];
    rs[threadIdx.x] = s;
    rq[threadIdx.x] = q;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            rs[threadIdx.x] += rs[threadIdx.x + o];
            rq[threadIdx.x] += rq[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * c] = rs[0];
        out[2 * c + 1] = rq[0];
    }
}

}  // namespace arso

struct arso_surrogate {
    CUtensorMap tm_w1t, tm_w2t, tm_w2;  // TMA maps of W1^T, W2^T (forward) and W2 (dh1)
    arso::DeviceBuffer w, w16, w16t, m, v, g, norm;
    float mean[arso::IN], sd[arso::IN];
    bool norm_set = false;
    uint64_t t = 0;
};

namespace arso {

struct Activations {
    DeviceBuffer xb, h1, h2, z, dz, dh1, dh2, lsum;
    DeviceBuffer pw1, pb1, pw2, pb2, pw3, pb3;  // gradient partials, summed by grad_finish_kernel
    int cap = 0;
    void ensure(int rows) {
        if (rows <= cap) return;
        xb.ensure((size_t)rows * IN * 4);
        h1.ensure((size_t)rows * HID * 4);
        h2.ensure((size_t)rows * HID * 4);
        z.ensure((size_t)rows * GM_NT * 4);  // partial logits, one row of them per output tile
        dz.ensure((size_t)rows * 4);
        dh1.ensure((size_t)rows * HID * 4);
        dh2.ensure((size_t)rows * HID * 4);
        const size_t chunks = (rows + DH2_ROWS - 1) / DH2_ROWS, tiles = (size_t)(rows + GM_BM - 1) / GM_BM;
        pb1.ensure(tiles * HID * 4);
        pb2.ensure(chunks * HID * 4);
        pw3.ensure(chunks * HID * 4);
        pb3.ensure(chunks * 4);
        lsum.ensure(8);
        cap = rows;
    }
};

static void upload_norm(arso_surrogate *s) {
    float h[2 * IN];
    std::memcpy(h, s->mean, sizeof(s->mean));
    std::memcpy(h + IN, s->sd, sizeof(s->sd));
    s->norm.ensure(sizeof(h));
    ARSO_CUDA(cudaMemcpy(s->norm.ptr, h, sizeof(h), cudaMemcpyHostToDevice));
}

// forward of `rows` gathered rows: xb -> h1 -> h2 -> z (logits); the output layer
// is fused into the second GEMM's epilogue (keep_h2 = false: h2 is not stored)
static void mlp_forward(const arso_surrogate *s, Activations &a, int rows, bool keep_h2, cudaStream_t st) {
    const __nv_bfloat16 *w = s->w16.as<__nv_bfloat16>();
    umma_gemm(rows, HID, IN, {a.xb.ptr, IN, 1, 0}, {w + OFF_W1, 1, HID, 1, &s->tm_w1t}, a.h1.as<float>(), HID,
              EPI_BIAS_RELU,
              w + OFF_B1, nullptr, 0, nullptr, nullptr, nullptr, nullptr, st);
    umma_gemm(rows, HID, HID, {a.h1.ptr, HID, 1, 0}, {w + OFF_W2, 1, HID, 1, &s->tm_w2t},
              keep_h2 ? a.h2.as<float>() : nullptr,
              HID, EPI_BIAS_RELU, w + OFF_B2, nullptr, 0, w + OFF_W3, a.z.as<float>(), nullptr, nullptr, st);
}

// gradients of the mean BCE into g (FP32) given a.dz: every parameter block is
// accumulated as partial sums (over batch chunks) that one kernel adds in order
static void mlp_backward(const arso_surrogate *s, Activations &a, int rows, float *g, cudaStream_t st) {
    const __nv_bfloat16 *w = s->w16.as<__nv_bfloat16>();
    const int chunks = (rows + DH2_ROWS - 1) / DH2_ROWS, tiles = (rows + GM_BM - 1) / GM_BM;
    {   // dh2 = dz W3^T (h2 > 0); partials of db2, dW3, db3
        ProfScope ps_(ARSO_K_OTHER, (double)rows * HID * 8 + (double)rows * 4, st);
        dh2_kernel<<<chunks, HID, 0, st>>>(a.dz.as<float>(), w + OFF_W3, a.h2.as<float>(), rows, a.dh2.as<float>(),
                                           a.pb2.as<float>(), a.pw3.as<float>(), a.pb3.as<float>());
        ARSO_CUDA(cudaGetLastError());
    }
    // dW2[i, j] = sum_b h1[b, i] dh2[b, j]
    const int s2 = umma_gemm(HID, HID, rows, {a.h1.ptr, 1, HID, 0}, {a.dh2.ptr, 1, HID, 0}, nullptr, HID, EPI_NONE,
                             nullptr, nullptr, 0, nullptr, nullptr, nullptr, &a.pw2, st);
    // dh1 = dh2 W2^T (h1 > 0), with the partials of db1 = sum_b dh1[b, :]
    umma_gemm(rows, HID, HID, {a.dh2.ptr, HID, 1, 0}, {w + OFF_W2, HID, 1, 1, &s->tm_w2}, a.dh1.as<float>(), HID,
              EPI_RELU_MASK,
              nullptr, a.h1.as<float>(), HID, nullptr, nullptr, a.pb1.as<float>(), nullptr, st);
    // dW1[i, j] = sum_b xb[b, i] dh1[b, j]
    const int s1 = umma_gemm(IN, HID, rows, {a.xb.ptr, 1, IN, 0}, {a.dh1.ptr, 1, HID, 0}, nullptr, HID, EPI_NONE,
                             nullptr, nullptr, 0, nullptr, nullptr, nullptr, &a.pw1, st);
    GradParts p{{a.pw1.as<float>(), a.pb1.as<float>(), a.pw2.as<float>(), a.pb2.as<float>(), a.pw3.as<float>(),
                 a.pb3.as<float>()},
                {s1, tiles, s2, chunks, chunks, chunks}};
    const double parts = (double)s1 * IN * HID + (double)tiles * HID + (double)s2 * HID * HID +
                         (double)chunks * (2 * HID + 1);
    ProfScope ps_(ARSO_K_REDUCE, (parts + N_PARAMS) * 4, st);
    grad_finish_kernel<<<(N_PARAMS + 255) / 256, 256, 0, st>>>(p, g);
    ARSO_CUDA(cudaGetLastError());
}

static void gather(const float *x, const uint32_t *idx, uint64_t base, int rows, const arso_surrogate *s,
                   Activations &a, cudaStream_t st) {
    ProfScope ps_(ARSO_K_OTHER, (double)rows * IN * 8, st);
    gather_norm_kernel<<<rows, 64, 0, st>>>(x, idx, base, rows, s->norm.as<float>(), a.xb.as<float>());
    ARSO_CUDA(cudaGetLastError());
}

static void bce(const arso_surrogate *s, Activations &a, const float *y, const uint32_t *idx, uint64_t base, int rows,
                cudaStream_t st) {
    ProfScope ps_(ARSO_K_REDUCE, (double)rows * (GM_NT * 4 + 12), st);
    bce_kernel<<<(rows + 255) / 256, 256, 0, st>>>(a.z.as<float>(), s->w16.as<__nv_bfloat16>() + OFF_B3, y, idx, base,
                                                  rows, 1.f / (float)rows, a.dz.as<float>(), a.lsum.as<double>());
    ARSO_CUDA(cudaGetLastError());
}

// 2-D TMA map over a row-major bfloat16 matrix of `rows` x `cols` (row stride `ld`
// elements), box of 8 columns x 128 rows; out-of-range elements read as zero
static void encode_map(CUtensorMap *m, const void *base, uint64_t cols, uint64_t rows, uint64_t ld) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        ARSO_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn) throw Error(ARSO_ECUDA, "cuTensorMapEncodeTiled is unavailable");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {cols, rows}, strides[1] = {ld * 2};
    const cuuint32_t box[2] = {8, GM_BN}, estr[2] = {1, 1};
    const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(ARSO_ECUDA, "cuTensorMapEncodeTiled failed");
}

static void make_weight_maps(arso_surrogate *s) {
    const __nv_bfloat16 *t = s->w16t.as<__nv_bfloat16>();
    encode_map(&s->tm_w1t, t + T_W1, IN, HID, T1_LD);
    encode_map(&s->tm_w2t, t + T_W2, HID, HID, HID);
    encode_map(&s->tm_w2, s->w16.as<__nv_bfloat16>() + OFF_W2, HID, HID, HID);
}

static void refresh_bf16(arso_surrogate *s, cudaStream_t st) {
    ProfScope ps_(ARSO_K_OTHER, N_PARAMS * 6.0, st);
    to_bf16_kernel<<<64, 256, 0, st>>>(s->w.as<float>(), s->w16.as<__nv_bfloat16>(), s->w16t.as<__nv_bfloat16>(),
                                       N_PARAMS);
    ARSO_CUDA(cudaGetLastError());
}

static void ensure_norm(arso_surrogate *s, const float *x, uint64_t n, cudaStream_t st) {
    if (s->norm_set) return;
    DeviceBuffer mom;
    mom.ensure(2 * IN * sizeof(double));
    {
        ProfScope ps_(ARSO_K_REDUCE, (double)n * IN * 4, st);
        moments_kernel<<<IN, 256, 0, st>>>(x, n, mom.as<double>());
        ARSO_CUDA(cudaGetLastError());
    }
    double h[2 * IN];
    ARSO_CUDA(cudaMemcpyAsync(h, mom.ptr, sizeof(h), cudaMemcpyDeviceToHost, st));
    ARSO_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c < IN; ++c) {
        const double mu = h[2 * c] / (double)n;
        const double var = std::max(0.0, h[2 * c + 1] / (double)n - mu * mu);
        s->mean[c] = (float)mu;
        s->sd[c] = var > 1e-12 ? (float)std::sqrt(var) : 1.f;
    }
    s->norm_set = true;
    upload_norm(s);
}

}  // namespace arso

using namespace arso;

extern "C" {

arso_status arso_surrogate_create(uint64_t seed, arso_surrogate **out) {
    try {
        ARSO_REQUIRE(out != nullptr, "out is NULL");
        std::unique_ptr<arso_surrogate> s(new arso_surrogate());
        std::vector<float> h(N_PARAMS, 0.f);
        std::mt19937_64 rng(seed);
        auto fill = [&](size_t off, int fan_in, size_t cnt) {
            const double lim = std::sqrt(6.0 / fan_in);  // He-uniform
            std::uniform_real_distribution<double> U(-lim, lim);
            for (size_t i = 0; i < cnt; ++i) h[off + i] = (float)U(rng);
        };
        fill(OFF_W1, IN, (size_t)IN * HID);
        fill(OFF_W2, HID, (size_t)HID * HID);
        fill(OFF_W3, HID, HID);
        s->w.ensure(N_PARAMS * 4);
        s->w16.ensure(N_PARAMS * 2);
        s->w16t.ensure(T_SIZE * 2);
        ARSO_CUDA(cudaMemset(s->w16t.ptr, 0, T_SIZE * 2));
        make_weight_maps(s.get());
        s->m.ensure(N_PARAMS * 4);
        s->v.ensure(N_PARAMS * 4);
        s->g.ensure(N_PARAMS * 4);
        ARSO_CUDA(cudaMemcpy(s->w.ptr, h.data(), N_PARAMS * 4, cudaMemcpyHostToDevice));
        ARSO_CUDA(cudaMemset(s->m.ptr, 0, N_PARAMS * 4));
        ARSO_CUDA(cudaMemset(s->v.ptr, 0, N_PARAMS * 4));
        for (int c = 0; c < IN; ++c) s->mean[c] = 0.f, s->sd[c] = 1.f;
        upload_norm(s.get());
        refresh_bf16(s.get(), 0);
        ARSO_CUDA(cudaDeviceSynchronize());
        *out = s.release();
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

void arso_surrogate_free(arso_surrogate *s) { delete s; }

arso_status arso_surrogate_set_norm(arso_surrogate *s, const float *mean, const float *stdev) {
    try {
        ARSO_REQUIRE(s && mean && stdev, "NULL argument");
        for (int c = 0; c < IN; ++c) {
            ARSO_REQUIRE(stdev[c] > 0.f, "standard deviations must be positive");
            s->mean[c] = mean[c];
            s->sd[c] = stdev[c];
        }
        s->norm_set = true;
        upload_norm(s);
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

arso_status arso_surrogate_get_params(const arso_surrogate *s, float *out) {
    try {
        ARSO_REQUIRE(s && out, "NULL argument");
        ARSO_CUDA(cudaMemcpy(out, s->w.ptr, N_PARAMS * 4, cudaMemcpyDeviceToHost));
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

arso_status arso_surrogate_set_params(arso_surrogate *s, const float *in) {
    try {
        ARSO_REQUIRE(s && in, "NULL argument");
        ARSO_CUDA(cudaMemcpy(s->w.ptr, in, N_PARAMS * 4, cudaMemcpyHostToDevice));
        refresh_bf16(s, 0);
        ARSO_CUDA(cudaDeviceSynchronize());
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

arso_status arso_surrogate_grads(const arso_surrogate *s, const float *x, const float *y, uint64_t n, void *stream,
                                 float *grads_out, double *loss_out) {
    try {
        ARSO_REQUIRE(s && x && y && grads_out, "NULL argument");
        ARSO_REQUIRE(n > 0 && n <= (1u << 20), "n must be in [1, 2^20]");
        cudaStream_t st = (cudaStream_t)stream;
        Activations a;
        a.ensure((int)n);
        gather(x, nullptr, 0, (int)n, s, a, st);
        mlp_forward(s, a, (int)n, true, st);
        ARSO_CUDA(cudaMemsetAsync(a.lsum.ptr, 0, 8, st));
        bce(s, a, y, nullptr, 0, (int)n, st);
        DeviceBuffer g;
        g.ensure(N_PARAMS * 4);
        mlp_backward(s, a, (int)n, g.as<float>(), st);
        ARSO_CUDA(cudaMemcpyAsync(grads_out, g.ptr, N_PARAMS * 4, cudaMemcpyDeviceToHost, st));
        double l = 0;
        ARSO_CUDA(cudaMemcpyAsync(&l, a.lsum.ptr, 8, cudaMemcpyDeviceToHost, st));
        ARSO_CUDA(cudaStreamSynchronize(st));
        check_gemm_err();
        if (loss_out) *loss_out = l / (double)n;
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

arso_status arso_surrogate_train(arso_surrogate *s, const float *x, const float *y, uint64_t n, uint32_t epochs,
                                 uint32_t batch, double lr, uint64_t seed, void *stream, double *loss_out) {
    try {
        ARSO_REQUIRE(s && x && y, "NULL argument");
        ARSO_REQUIRE(n > 0 && n < (1ull << 32), "n must be in [1, 2^32)");
        ARSO_REQUIRE(batch > 0 && batch <= 65536, "batch must be in [1, 65536]");
        ARSO_REQUIRE(lr > 0, "lr must be > 0");
        cudaStream_t st = (cudaStream_t)stream;
        ensure_norm(s, x, n, st);
        Activations a;
        a.ensure((int)std::min<uint64_t>(batch, n));
        DeviceBuffer d_idx;
        d_idx.ensure(n * 4);
        std::vector<uint32_t> idx(n);
        std::mt19937_64 rng(seed);
        double last = 0;
        for (uint32_t ep = 0; ep < epochs; ++ep) {
            for (uint64_t i = 0; i < n; ++i) idx[i] = (uint32_t)i;
            std::shuffle(idx.begin(), idx.end(), rng);
            ARSO_CUDA(cudaMemcpyAsync(d_idx.ptr, idx.data(), n * 4, cudaMemcpyHostToDevice, st));
            ARSO_CUDA(cudaMemsetAsync(a.lsum.ptr, 0, 8, st));
            for (uint64_t b0 = 0; b0 < n; b0 += batch) {
                const int rows = (int)std::min<uint64_t>(batch, n - b0);
                gather(x, d_idx.as<uint32_t>(), b0, rows, s, a, st);
                mlp_forward(s, a, rows, true, st);
                bce(s, a, y, d_idx.as<uint32_t>(), b0, rows, st);
                mlp_backward(s, a, rows, s->g.as<float>(), st);
                s->t += 1;
                const float c1 = 1.f - (float)std::pow(0.9, (double)s->t), c2 = 1.f - (float)std::pow(0.999, (double)s->t);
                ProfScope ps_(ARSO_K_OTHER, N_PARAMS * 22.0, st);
                adam_kernel<<<152, 256, 0, st>>>(s->w.as<float>(), s->w16.as<__nv_bfloat16>(),
                                                 s->w16t.as<__nv_bfloat16>(), s->g.as<float>(), s->m.as<float>(),
                                                 s->v.as<float>(), N_PARAMS, (float)lr, 0.9f, 0.999f, 1e-8f, c1, c2);
                ARSO_CUDA(cudaGetLastError());
            }
            ARSO_CUDA(cudaMemcpyAsync(&last, a.lsum.ptr, 8, cudaMemcpyDeviceToHost, st));
            ARSO_CUDA(cudaStreamSynchronize(st));
            check_gemm_err();
        }
        if (loss_out) *loss_out = last / (double)n;
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

arso_status arso_surrogate_predict(const arso_surrogate *s, const float *x, uint64_t n, float *out, void *stream) {
    try {
        ARSO_REQUIRE(s && x && out, "NULL argument");
        cudaStream_t st = (cudaStream_t)stream;
        Activations a;
        const uint64_t chunk = 65536;
        a.ensure((int)std::min<uint64_t>(n, chunk));
        for (uint64_t b0 = 0; b0 < n; b0 += chunk) {
            const int rows = (int)std::min<uint64_t>(chunk, n - b0);
            gather(x, nullptr, b0, rows, s, a, st);
            mlp_forward(s, a, rows, false, st);
            ProfScope ps_(ARSO_K_OTHER, (double)rows * (GM_NT * 4 + 4), st);
            sigmoid_kernel<<<(rows + 255) / 256, 256, 0, st>>>(a.z.as<float>(), s->w16.as<__nv_bfloat16>() + OFF_B3, rows,
                                                              out + b0);
            ARSO_CUDA(cudaGetLastError());
        }
        ARSO_CUDA(cudaStreamSynchronize(st));
        check_gemm_err();
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

arso_status arso_debug_stall_next_gemm(void) {
    g_stall_next_gemm.store(true);
    return ARSO_OK;
}

arso_status arso_circuit_features(const arso_circuit *c, const arso_criterion *crit, float *out) {
    try {
        ARSO_REQUIRE(c && crit && out, "NULL argument");
        const std::vector<float> f = circuit_features(c, crit);
        std::copy(f.begin(), f.end(), out);
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    }
}

}  // extern "C"
