// Register-blocked fused tile pass (complex64, tiles of 2^t >= 2^10 amplitudes).
//
// A CTA of 2^(t-5) threads owns one tile of one trajectory; every thread
// keeps 32 amplitudes in registers. The tile-local index of register ri of
// thread tid is deposit(ri, R) | deposit(tid, complement of R), where R, the 5
// "register bits", changes only between phases (a swizzled shared-memory
// transpose). Within a phase:
//  * dense one-/two-qubit gates and CX targets act on register bits, entirely
//    in registers;
//  * diagonal gates (T, S, Z, RZ, P, CZ, CP) act on any bit in place;
//  * X gates and the X part of Pauli errors never move data: the tile keeps
//    an index mask m with state[j] = stored[j ^ m] (Eq. (2): X swaps the pair
//    (a0, a1), i.e. flips bit q of the index), later gates act on the stored
//    data conjugated by the mask, and the final store writes stored[k] to
//    index k ^ m;
//  * the Z part of a Pauli error is a phase on bit q; Y = i X Z adds a factor
//    i tracked as a power gp and applied at the store.
// Global loads and stores are 16-byte vector accesses in the mapping
// R = {0, t-4, t-3, t-2, t-1}, whose thread bits 1..t-5 are contiguous.
#include <algorithm>

#include "prof.h"
#include "sim_common.cuh"

namespace arso {

__device__ __forceinline__ uint32_t swz(uint32_t j) { return j ^ (((j >> 4) ^ (j >> 8) ^ (j >> 12)) & 15u); }

__device__ __forceinline__ void unpack_r(uint32_t packed, uint32_t (&r)[REG_BITS]) {
#pragma unroll
    for (int b = 0; b < REG_BITS; ++b) r[b] = (packed >> (5 * b)) & 31u;
}

// tid's bits deposited into the tile bits that are not register bits, ascending
__device__ __forceinline__ uint32_t thread_part(uint32_t tid, uint32_t rmask, int t) {
    uint32_t out = 0;
    int k = 0;
    for (int b = 0; b < t; ++b)
        if (!((rmask >> b) & 1u)) {
            out |= ((tid >> k) & 1u) << b;
            ++k;
        }
    return out;
}

// register part of the local index of register ri (ri is a constant after unrolling)
__device__ __forceinline__ uint32_t reg_part(int ri, const uint32_t (&r)[REG_BITS]) {
    uint32_t o = 0;
#pragma unroll
    for (int b = 0; b < REG_BITS; ++b)
        if ((ri >> b) & 1) o |= 1u << r[b];
    return o;
}

// ------------------------------------------------------- register gates ---
template <int P>
__device__ __forceinline__ void rg_dense1(float2 (&v)[32], float2 u00, float2 u01, float2 u10, float2 u11) {
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        if (ri & (1 << P)) continue;
        const float2 a0 = v[ri], a1 = v[ri | (1 << P)];
        v[ri] = cmac2(u00, a0, u01, a1);
        v[ri | (1 << P)] = cmac2(u10, a0, u11, a1);
    }
}

// X H X on the pair: (a0, a1) -> ((a1 - a0)/sqrt2, (a0 + a1)/sqrt2)
template <int P> __device__ __forceinline__ void rg_hflip(float2 (&v)[32]) {
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        if (ri & (1 << P)) continue;
        const float2 a0 = v[ri], a1 = v[ri | (1 << P)];
        v[ri] = make_float2(mul_rsqrt2(a1.x - a0.x), mul_rsqrt2(a1.y - a0.y));
        v[ri | (1 << P)] = make_float2(mul_rsqrt2(a0.x + a1.x), mul_rsqrt2(a0.y + a1.y));
    }
}

template <int P> __device__ __forceinline__ void rg_h(float2 (&v)[32]) {
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        if (ri & (1 << P)) continue;
        const float2 a0 = v[ri], a1 = v[ri | (1 << P)];
        v[ri] = make_float2(mul_rsqrt2(a0.x + a1.x), mul_rsqrt2(a0.y + a1.y));
        v[ri | (1 << P)] = make_float2(mul_rsqrt2(a0.x - a1.x), mul_rsqrt2(a0.y - a1.y));
    }
}

// CX on stored data, target register bit P; control is register bit cpos
// (0..4) or, when cpos == 15, the thread-level bit value cth.
template <int P> __device__ __forceinline__ void rg_cx(float2 (&v)[32], uint32_t cpos, uint32_t cth) {
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        if (ri & (1 << P)) continue;
        const uint32_t ctl = cpos < REG_BITS ? (((uint32_t)ri >> cpos) & 1u) : cth;
        const float2 a0 = v[ri], a1 = v[ri | (1 << P)];
        v[ri] = ctl ? a1 : a0;
        v[ri | (1 << P)] = ctl ? a0 : a1;
    }
}

template <int P0, int P1> __device__ __forceinline__ void rg_dense2(float2 (&v)[32], const float2 (&M)[16]) {
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        if (ri & ((1 << P0) | (1 << P1))) continue;
        const int ix[4] = {ri, ri | (1 << P0), ri | (1 << P1), ri | (1 << P0) | (1 << P1)};
        float2 a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = v[ix[k]];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 acc = cmac2(M[4 * k], a[0], M[4 * k + 1], a[1]);
            const float2 acc2 = cmac2(M[4 * k + 2], a[2], M[4 * k + 3], a[3]);
            acc.x += acc2.x;
            acc.y += acc2.y;
            v[ix[k]] = acc;
        }
    }
}

// Value of tile bit q of the true index (stored index ^ m) for register ri:
// register bit pos < 5 -> (ri >> pos) ^ mq; else the thread-level value th.
__device__ __forceinline__ uint32_t bit_of(int ri, uint32_t pos, uint32_t mq, uint32_t th) {
    return pos < REG_BITS ? ((((uint32_t)ri >> pos) & 1u) ^ mq) : th;
}

struct TileCtx {
    uint32_t r[REG_BITS];  // register bits of the current phase
    uint32_t rmask;        // same as a mask
    uint32_t tpart;        // thread part of the local index
    uint32_t m;            // X mask (stored[j] = state[j ^ m])
    uint32_t gp;           // global phase i^gp
};

__device__ __forceinline__ uint32_t reg_pos(const TileCtx &c, uint32_t q) {
    uint32_t p = 15;
#pragma unroll
    for (int b = 0; b < REG_BITS; ++b)
        if (c.r[b] == q) p = (uint32_t)b;
    return p;
}

// diag(d0, d1) on tile bit q (true index), any bit
__device__ __forceinline__ void rg_diag1(float2 (&v)[32], const TileCtx &c, uint32_t q, float2 d0, float2 d1) {
    const uint32_t pos = reg_pos(c, q), mq = (c.m >> q) & 1u, th = ((c.tpart ^ c.m) >> q) & 1u;
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) v[ri] = cmul(bit_of(ri, pos, mq, th) ? d1 : d0, v[ri]);
}

__device__ __forceinline__ void rg_omega(float2 (&v)[32], const TileCtx &c, uint32_t q, uint32_t k) {
    const uint32_t pos = reg_pos(c, q), mq = (c.m >> q) & 1u, th = ((c.tpart ^ c.m) >> q) & 1u;
    if (pos >= REG_BITS) {
        if (th) {
#pragma unroll
            for (int ri = 0; ri < 32; ++ri) v[ri] = omega_mul(v[ri], k);
        }
        return;
    }
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        const float2 w = omega_mul(v[ri], k);
        v[ri] = bit_of(ri, pos, mq, th) ? w : v[ri];
    }
}

__device__ __forceinline__ void rg_cz(float2 (&v)[32], const TileCtx &c, uint32_t qa, uint32_t qb) {
    const uint32_t pa = reg_pos(c, qa), ma = (c.m >> qa) & 1u, ta = ((c.tpart ^ c.m) >> qa) & 1u;
    const uint32_t pb = reg_pos(c, qb), mb = (c.m >> qb) & 1u, tb = ((c.tpart ^ c.m) >> qb) & 1u;
    if (pa >= REG_BITS && pb >= REG_BITS && !(ta & tb)) return;
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        const uint32_t s = bit_of(ri, pa, ma, ta) & bit_of(ri, pb, mb, tb);
        v[ri] = s ? cneg(v[ri]) : v[ri];
    }
}

__device__ __forceinline__ void rg_diag2(float2 (&v)[32], const TileCtx &c, uint32_t qa, uint32_t qb,
                                         const float2 *__restrict__ d) {
    const uint32_t pa = reg_pos(c, qa), ma = (c.m >> qa) & 1u, ta = ((c.tpart ^ c.m) >> qa) & 1u;
    const uint32_t pb = reg_pos(c, qb), mb = (c.m >> qb) & 1u, tb = ((c.tpart ^ c.m) >> qb) & 1u;
    const float2 d0 = d[0], d1 = d[1], d2 = d[2], d3 = d[3];
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        const uint32_t k = bit_of(ri, pa, ma, ta) | (bit_of(ri, pb, mb, tb) << 1);
        const float2 f = k == 0 ? d0 : (k == 1 ? d1 : (k == 2 ? d2 : d3));
        v[ri] = cmul(f, v[ri]);
    }
}

// Pauli error on tile bit q of the true state (Eq. (2)): Z -> phase -1 on
// bit q; X -> index mask; Y = i X Z.
__device__ __forceinline__ void rg_pauli(float2 (&v)[32], TileCtx &c, uint32_t q, uint32_t code) {
    if (code & 2u) {  // Z part (Z or Y): negate where bit q of the true index is 1
        const uint32_t pos = reg_pos(c, q), mq = (c.m >> q) & 1u, th = ((c.tpart ^ c.m) >> q) & 1u;
#pragma unroll
        for (int ri = 0; ri < 32; ++ri) v[ri] = bit_of(ri, pos, mq, th) ? cneg(v[ri]) : v[ri];
    }
    if (code & 1u) c.m ^= 1u << q;          // X part (X or Y)
    if (code == 3u) c.gp = (c.gp + 1u) & 3u;  // Y = i X Z
}

template <int P>
__device__ __forceinline__ void dispatch_dense1(float2 (&v)[32], const DGate &g, const float2 *__restrict__ M,
                                                uint32_t flip) {
    if (g.cls == GC_H) {
        if (flip) rg_hflip<P>(v);
        else rg_h<P>(v);
        return;
    }
    if (!flip) rg_dense1<P>(v, M[0], M[1], M[2], M[3]);
    else rg_dense1<P>(v, M[3], M[2], M[1], M[0]);
}

template <int P0, int P1>
__device__ __forceinline__ void dispatch_dense2_pp(float2 (&v)[32], const float2 (&M)[16]) {
    rg_dense2<P0, P1>(v, M);
}

__device__ __forceinline__ void apply_dense2(float2 (&v)[32], uint32_t p0, uint32_t p1, const float2 (&M)[16]) {
#define ARSO_D2(a, b) \
    case a * 5 + b: dispatch_dense2_pp<a, b>(v, M); break;
    switch (p0 * 5 + p1) {
        ARSO_D2(0, 1) ARSO_D2(0, 2) ARSO_D2(0, 3) ARSO_D2(0, 4) ARSO_D2(1, 0) ARSO_D2(1, 2) ARSO_D2(1, 3)
        ARSO_D2(1, 4) ARSO_D2(2, 0) ARSO_D2(2, 1) ARSO_D2(2, 3) ARSO_D2(2, 4) ARSO_D2(3, 0) ARSO_D2(3, 1)
        ARSO_D2(3, 2) ARSO_D2(3, 4) ARSO_D2(4, 0) ARSO_D2(4, 1) ARSO_D2(4, 2) ARSO_D2(4, 3)
        default: break;
    }
#undef ARSO_D2
}

__device__ __forceinline__ void apply_gate_rb(float2 (&v)[32], TileCtx &c, const DGate &g, uint8_t rp,
                                              const float2 *__restrict__ mats) {
    const uint32_t p0 = rp & 15u, p1 = rp >> 4;
    const float2 *M = mats + g.mat;
    switch (g.cls) {
        case GC_DENSE1:
        case GC_H: {
            const uint32_t flip = (c.m >> g.q0) & 1u;
            switch (p0) {
                case 0: dispatch_dense1<0>(v, g, M, flip); break;
                case 1: dispatch_dense1<1>(v, g, M, flip); break;
                case 2: dispatch_dense1<2>(v, g, M, flip); break;
                case 3: dispatch_dense1<3>(v, g, M, flip); break;
                default: dispatch_dense1<4>(v, g, M, flip); break;
            }
            break;
        }
        case GC_DIAG1: rg_diag1(v, c, g.q0, M[0], M[1]); break;
        case GC_OMEGA: rg_omega(v, c, g.q0, g.mat); break;
        case GC_X: c.m ^= 1u << g.q0; break;
        case GC_CZ: rg_cz(v, c, g.q0, g.q1); break;
        case GC_DIAG2: rg_diag2(v, c, g.q0, g.q1, M); break;
        case GC_CX: {
            // CX X^m = X^{m'} CX with m' = m ^ (target bit if the control bit is in m)
            const uint32_t cth = (c.tpart >> g.q0) & 1u;
            switch (p1) {
                case 0: rg_cx<0>(v, p0, cth); break;
                case 1: rg_cx<1>(v, p0, cth); break;
                case 2: rg_cx<2>(v, p0, cth); break;
                case 3: rg_cx<3>(v, p0, cth); break;
                default: rg_cx<4>(v, p0, cth); break;
            }
            if ((c.m >> g.q0) & 1u) c.m ^= 1u << g.q1;
            break;
        }
        case GC_DENSE2:
        case GC_SWAP: {
            float2 U[16];
            const uint32_t mab = ((c.m >> g.q0) & 1u) | (((c.m >> g.q1) & 1u) << 1);
            if (g.cls == GC_SWAP) {
#pragma unroll
                for (int k = 0; k < 16; ++k) U[k] = make_float2(0.f, 0.f);
                U[0] = U[15] = U[1 * 4 + 2] = U[2 * 4 + 1] = make_float2(1.f, 0.f);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int l = 0; l < 4; ++l) U[4 * k + l] = M[4 * (k ^ mab) + (l ^ mab)];
            }
            apply_dense2(v, p0, p1, U);
            // SWAP X^m = X^{m with bits q0, q1 exchanged} SWAP
            if (g.cls == GC_SWAP && (((c.m >> g.q0) ^ (c.m >> g.q1)) & 1u)) c.m ^= (1u << g.q0) | (1u << g.q1);
            break;
        }
        default: break;
    }
}

// stored index -> tile-local index bits for the load/store mapping
__device__ __forceinline__ void set_phase(TileCtx &c, uint32_t packed, int t) {
    unpack_r(packed, c.r);
    c.rmask = 0;
#pragma unroll
    for (int b = 0; b < REG_BITS; ++b) c.rmask |= 1u << c.r[b];
    c.tpart = thread_part(threadIdx.x, c.rmask, t);
}

__device__ __forceinline__ void remap(float2 (&v)[32], float2 *sm, TileCtx &c, uint32_t packed, int t) {
    __syncthreads();
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) sm[swz(c.tpart | reg_part(ri, c.r))] = v[ri];
    set_phase(c, packed, t);
    __syncthreads();
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) v[ri] = sm[swz(c.tpart | reg_part(ri, c.r))];
}

template <bool LAST>
__global__ void __launch_bounds__(512, 1) pass_rb_kernel(PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    __shared__ Partial red[32];
    const int t = a.t, cl = a.c;
    const uint32_t slot = blockIdx.y;
    const uint64_t N = 1ull << a.n;
    int start;
    uint64_t tr = 0;
    const float2 *src;
    float2 *dst;
    if (a.ideal) {
        start = 0;
        src = static_cast<const float2 *>(a.ideal_src);
        dst = static_cast<float2 *>(a.ideal_dst);
    } else {
        start = a.start_pass[slot];
        if (a.pass < start) return;
        tr = a.slot_traj[slot];
        float2 *mine = static_cast<float2 *>(a.work) + (size_t)slot * N;
        src = a.pass == start ? static_cast<const float2 *>(a.cache) + (size_t)a.cache_slot[start] * N : mine;
        dst = mine;
    }
    // tile base: deposit the tile index into the non-tile global bits
    uint64_t base = 0;
    {
        uint64_t tile = blockIdx.x;
        for (uint64_t mm = a.rest_mask; mm; mm &= mm - 1) {
            if (tile & 1) base |= mm & (~mm + 1);
            tile >>= 1;
        }
    }
    const uint32_t *offs = a.offs;
    const uint32_t cmask = (1u << cl) - 1u;
    auto gidx = [&](uint32_t j) -> uint64_t { return base + offs[j >> cl] + (j & cmask); };

    // load mapping R = {0, t-4, ..., t-1}: register ri = b0 | hi << 1 holds j = hi << (t-4) | tid << 1 | b0
    const uint32_t load_packed = 0u | ((uint32_t)(t - 4) << 5) | ((uint32_t)(t - 3) << 10) |
                                 ((uint32_t)(t - 2) << 15) | ((uint32_t)(t - 1) << 20);
    float2 v[32];
#pragma unroll
    for (int hi = 0; hi < 16; ++hi) {
        const uint32_t j = ((uint32_t)hi << (t - 4)) | (threadIdx.x << 1);
        const float4 w = __ldg(reinterpret_cast<const float4 *>(src + gidx(j)));
        v[2 * hi] = make_float2(w.x, w.y);
        v[2 * hi + 1] = make_float2(w.z, w.w);
    }
    TileCtx c;
    c.m = 0;
    c.gp = 0;
    set_phase(c, load_packed, t);

    const uint32_t *ev = nullptr, *ev_end = nullptr;
    if (!a.ideal) {
        const uint32_t *lo = a.keys + a.offsets[tr];
        const uint32_t *hi = a.keys + a.offsets[tr + 1];
        const uint32_t key_lo = a.gb << 3;
        while (lo < hi) {
            const uint32_t *mid = lo + (hi - lo) / 2;
            if (*mid < key_lo) lo = mid + 1;
            else hi = mid;
        }
        ev = lo;
        ev_end = a.keys + a.offsets[tr + 1];
    }
    uint32_t next = ev && ev < ev_end ? *ev : NO_EVENT;
    const float2 *mats = static_cast<const float2 *>(a.mats);
    uint32_t cur_packed = load_packed;
    for (uint32_t ph = a.pb; ph < a.pe; ++ph) {
        const uint32_t R = a.ph_R[ph];
        if (R != cur_packed) {
            remap(v, sm, c, R, t);
            cur_packed = R;
        }
        const uint32_t ge = a.ph_gb[ph + 1];
        for (uint32_t g = a.ph_gb[ph]; g < ge; ++g) {
            const DGate gate = a.gates[g];
            apply_gate_rb(v, c, gate, a.rpos[g], mats);
            while (next != NO_EVENT && ev_pos(next) == g) {
                rg_pauli(v, c, ev_slot(next) ? gate.q1 : gate.q0, ev_code(next));
                ++ev;
                next = ev < ev_end ? *ev : NO_EVENT;
            }
        }
    }
    // global phase i^gp
    if (c.gp) {
#pragma unroll
        for (int ri = 0; ri < 32; ++ri) v[ri] = omega_mul(v[ri], 2u * c.gp);
    }
    if (LAST && !a.ideal && !a.store_last) {
        const float2 *ref = static_cast<const float2 *>(a.cache) + (size_t)a.ref_slot * N;
        Partial acc = empty_partial();
#pragma unroll
        for (int ri = 0; ri < 32; ++ri) {
            const uint32_t jj = (c.tpart | reg_part(ri, c.r)) ^ c.m;
            accumulate(acc, a.crit, v[ri], ref, gidx(jj));
        }
        acc = block_reduce_partial(acc, red);
        if (threadIdx.x == 0) a.partials[(size_t)slot * gridDim.x + blockIdx.x] = acc;
        return;
    }
    if (cur_packed != load_packed) remap(v, sm, c, load_packed, t);
    const uint32_t flip0 = c.m & 1u;
#pragma unroll
    for (int hi = 0; hi < 16; ++hi) {
        const uint32_t j = (((uint32_t)hi << (t - 4)) | (threadIdx.x << 1)) ^ (c.m & ~1u);
        const float2 e = flip0 ? v[2 * hi + 1] : v[2 * hi];
        const float2 o = flip0 ? v[2 * hi] : v[2 * hi + 1];
        reinterpret_cast<float4 *>(dst + gidx(j))[0] = make_float4(e.x, e.y, o.x, o.y);
    }
}

void launch_pass_rb(const PassArgs &a, bool last, uint32_t slots, double bytes, cudaStream_t st) {
    ProfScope ps_(last && !a.store_last ? ARSO_K_PASS_LAST : ARSO_K_PASS, bytes, st);
    const uint32_t tiles = 1u << (a.n - a.t);
    const int nt = 1 << (a.t - REG_BITS);
    const size_t smem = (size_t(1) << a.t) * sizeof(float2);
    dim3 grid(tiles, slots);
    if (last) {
        if (smem > 48 * 1024)
            ARSO_CUDA(cudaFuncSetAttribute(pass_rb_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        pass_rb_kernel<true><<<grid, nt, smem, st>>>(a);
    } else {
        if (smem > 48 * 1024)
            ARSO_CUDA(cudaFuncSetAttribute(pass_rb_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        pass_rb_kernel<false><<<grid, nt, smem, st>>>(a);
    }
    ARSO_CUDA(cudaGetLastError());
}

}  // namespace arso
