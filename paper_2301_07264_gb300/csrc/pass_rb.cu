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
// Code size matters: the whole phase loop must stay resident in the
// instruction cache, so only dense one-qubit gates, H and CX are specialised
// per register position (5 copies each); everything else is position-free.

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

// H on register bit P: (a0, a1) -> ((a0 + a1), (a0 - a1)) / sqrt2; with the
// qubit's mask bit set the stored data sees X H X: ((a1 - a0), (a0 + a1)) / sqrt2.
template <int P> __device__ __forceinline__ void rg_h(float2 (&v)[32], uint32_t flip) {
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        if (ri & (1 << P)) continue;
        const float2 a0 = v[ri], a1 = v[ri | (1 << P)];
        const float2 s = make_float2(mul_rsqrt2(a0.x + a1.x), mul_rsqrt2(a0.y + a1.y));
        const float2 d = make_float2(mul_rsqrt2(a0.x - a1.x), mul_rsqrt2(a0.y - a1.y));
        v[ri] = flip ? cneg(d) : s;
        v[ri | (1 << P)] = flip ? s : d;
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
    uint32_t tid, nthr;    // thread index within the tile's thread group, group size
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

// diag(1, e^{i k pi/4}) on tile bit q. On a register bit only the 16 registers
// whose true bit is 1 are touched (two unrolled variants per position); on a
// thread bit all 32 registers of the threads whose bit is 1.
struct OmegaOp {
    bool odd, sw, nx, ny;  // rotate by pi/4, then multiply by i^qq: swap and negate
    __device__ __forceinline__ explicit OmegaOp(uint32_t k) {
        odd = k & 1u;
        const uint32_t qq = (k >> 1) & 3u;
        sw = qq & 1u;
        nx = qq == 1u || qq == 2u;
        ny = qq >= 2u;
    }
    __device__ __forceinline__ float2 operator()(float2 a) const {
        const float2 r = odd ? make_float2(mul_rsqrt2(a.x - a.y), mul_rsqrt2(a.x + a.y)) : a;
        float2 o = sw ? make_float2(r.y, r.x) : r;
        o.x = nx ? -o.x : o.x;
        o.y = ny ? -o.y : o.y;
        return o;
    }
};
template <int P> __device__ __forceinline__ void rg_omega_half(float2 (&v)[32], const OmegaOp &op, uint32_t want) {
    if (want) {
#pragma unroll
        for (int ri = 0; ri < 32; ++ri)
            if (ri & (1 << P)) v[ri] = op(v[ri]);
    } else {
#pragma unroll
        for (int ri = 0; ri < 32; ++ri)
            if (!(ri & (1 << P))) v[ri] = op(v[ri]);
    }
}
__device__ __forceinline__ void rg_omega(float2 (&v)[32], const TileCtx &c, uint32_t q, uint32_t k) {
    const uint32_t pos = reg_pos(c, q), mq = (c.m >> q) & 1u, th = ((c.tpart ^ c.m) >> q) & 1u;
    const OmegaOp op(k);
    if (pos >= REG_BITS) {
        if (th) {
#pragma unroll
            for (int ri = 0; ri < 32; ++ri) v[ri] = op(v[ri]);
        }
        return;
    }
    const uint32_t want = mq ^ 1u;  // stored bit value whose true bit is 1
    switch (pos) {
        case 0: rg_omega_half<0>(v, op, want); break;
        case 1: rg_omega_half<1>(v, op, want); break;
        case 2: rg_omega_half<2>(v, op, want); break;
        case 3: rg_omega_half<3>(v, op, want); break;
        default: rg_omega_half<4>(v, op, want); break;
    }
}

// Registers whose tile bit q (of the true index) is 1, as a 32-bit mask.
__device__ __forceinline__ uint32_t reg_pattern(uint32_t pos) {
    return pos == 0 ? 0xAAAAAAAAu : pos == 1 ? 0xCCCCCCCCu : pos == 2 ? 0xF0F0F0F0u : pos == 3 ? 0xFF00FF00u : 0xFFFF0000u;
}
__device__ __forceinline__ uint32_t bit_mask(const TileCtx &c, uint32_t q) {
    const uint32_t pos = reg_pos(c, q);
    if (pos < REG_BITS) return ((c.m >> q) & 1u) ? ~reg_pattern(pos) : reg_pattern(pos);
    return (((c.tpart ^ c.m) >> q) & 1u) ? 0xFFFFFFFFu : 0u;
}
// negate the registers selected by mask: flip the sign bits
__device__ __forceinline__ void negate_masked(float2 (&v)[32], uint32_t mask) {
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        const uint32_t sgn = (mask << (31 - ri)) & 0x80000000u;
        v[ri].x = __uint_as_float(__float_as_uint(v[ri].x) ^ sgn);
        v[ri].y = __uint_as_float(__float_as_uint(v[ri].y) ^ sgn);
    }
}

__device__ __forceinline__ void rg_cz(float2 (&v)[32], const TileCtx &c, uint32_t qa, uint32_t qb) {
    const uint32_t mask = bit_mask(c, qa) & bit_mask(c, qb);
    if (mask) negate_masked(v, mask);
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
        const uint32_t mask = bit_mask(c, q);
        if (mask) negate_masked(v, mask);
    }
    if (code & 1u) c.m ^= 1u << q;          // X part (X or Y)
    if (code == 3u) c.gp = (c.gp + 1u) & 3u;  // Y = i X Z
}

// stored index -> tile-local index bits for the load/store mapping
__device__ __forceinline__ void set_phase(TileCtx &c, uint32_t packed, int t) {
    unpack_r(packed, c.r);
    c.rmask = 0;
#pragma unroll
    for (int b = 0; b < REG_BITS; ++b) c.rmask |= 1u << c.r[b];
    c.tpart = thread_part(c.tid, c.rmask, t);
}

// The swizzle is linear over XOR, so the shared-memory slot of register ri is
// swz(tpart) ^ (XOR of swz(1 << r[b]) over the set bits b of ri); walking the
// registers in Gray-code order costs one XOR per register.
__host__ __device__ constexpr int ctz5(int x) { return x & 1 ? 0 : x & 2 ? 1 : x & 4 ? 2 : x & 8 ? 3 : 4; }

__device__ __forceinline__ void smem_basis(const TileCtx &c, uint32_t &base, uint32_t (&sw)[REG_BITS]) {
    base = swz(c.tpart);
#pragma unroll
    for (int b = 0; b < REG_BITS; ++b) sw[b] = swz(1u << c.r[b]);
}
__device__ __forceinline__ void to_smem(const float2 (&v)[32], float2 *sm, const TileCtx &c) {
    uint32_t idx, sw[REG_BITS];
    smem_basis(c, idx, sw);
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        sm[idx] = v[k ^ (k >> 1)];
        if (k < 31) idx ^= sw[ctz5(k + 1)];
    }
}
__device__ __forceinline__ void from_smem(float2 (&v)[32], const float2 *sm, const TileCtx &c) {
    uint32_t idx, sw[REG_BITS];
    smem_basis(c, idx, sw);
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        v[k ^ (k >> 1)] = sm[idx];
        if (k < 31) idx ^= sw[ctz5(k + 1)];
    }
}

__device__ __forceinline__ void remap(float2 (&v)[32], float2 *sm, TileCtx &c, uint32_t packed, int t) {
    __syncthreads();
    to_smem(v, sm, c);
    set_phase(c, packed, t);
    __syncthreads();
    from_smem(v, sm, c);
}

// Dense two-qubit gates and SWAP are rare: they run through shared memory on
// the stored data (U already conjugated by the mask) with runtime indices.
__device__ __forceinline__ void smem_dense2(float2 *sm, int t, uint32_t q0, uint32_t q1, const float2 *__restrict__ U,
                                            uint32_t tid, uint32_t nthr) {
    const uint32_t lo = q0 < q1 ? q0 : q1, hi = q0 < q1 ? q1 : q0;
    const uint32_t m0 = 1u << q0, m1 = 1u << q1;
    float2 M[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) M[k] = U[k];
    for (uint32_t p = tid; p < (1u << (t - 2)); p += nthr) {
        const uint32_t i = insert_zero2(p, lo, hi);
        const uint32_t ix[4] = {swz(i), swz(i | m0), swz(i | m1), swz(i | m0 | m1)};
        float2 a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = sm[ix[k]];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 acc = cmac2(M[4 * k], a[0], M[4 * k + 1], a[1]);
            const float2 acc2 = cmac2(M[4 * k + 2], a[2], M[4 * k + 3], a[3]);
            acc.x += acc2.x;
            acc.y += acc2.y;
            sm[ix[k]] = acc;
        }
    }
}

__device__ __forceinline__ void apply_gate_rb(float2 (&v)[32], TileCtx &c, const DGate &g, uint8_t rp,
                                              const float2 *__restrict__ mats, float2 *sm, float2 *ubuf, int t) {
    const uint32_t p0 = rp & 15u, p1 = rp >> 4;
    const float2 *M = mats + g.mat;
    switch (g.cls) {
        case GC_H: {
            const uint32_t flip = (c.m >> g.q0) & 1u;
            switch (p0) {
                case 0: rg_h<0>(v, flip); break;
                case 1: rg_h<1>(v, flip); break;
                case 2: rg_h<2>(v, flip); break;
                case 3: rg_h<3>(v, flip); break;
                default: rg_h<4>(v, flip); break;
            }
            break;
        }
        case GC_DENSE1: {
            // with the qubit's mask bit set the stored data sees X U X = [[u11, u10], [u01, u00]]
            const uint32_t flip = (c.m >> g.q0) & 1u;
            const float2 u00 = flip ? M[3] : M[0], u01 = flip ? M[2] : M[1];
            const float2 u10 = flip ? M[1] : M[2], u11 = flip ? M[0] : M[3];
            switch (p0) {
                case 0: rg_dense1<0>(v, u00, u01, u10, u11); break;
                case 1: rg_dense1<1>(v, u00, u01, u10, u11); break;
                case 2: rg_dense1<2>(v, u00, u01, u10, u11); break;
                case 3: rg_dense1<3>(v, u00, u01, u10, u11); break;
                default: rg_dense1<4>(v, u00, u01, u10, u11); break;
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
            const uint32_t mab = ((c.m >> g.q0) & 1u) | (((c.m >> g.q1) & 1u) << 1);
            if (c.tid < 16) {
                const uint32_t k = c.tid >> 2, l = c.tid & 3u;
                float2 u;
                if (g.cls == GC_SWAP) {
                    const uint32_t perm[4] = {0, 2, 1, 3};
                    u = make_float2(perm[k] == l ? 1.f : 0.f, 0.f);
                } else {
                    u = M[4 * (k ^ mab) + (l ^ mab)];
                }
                ubuf[c.tid] = u;
            }
            __syncthreads();
            to_smem(v, sm, c);
            __syncthreads();
            smem_dense2(sm, t, g.q0, g.q1, ubuf, c.tid, c.nthr);
            __syncthreads();
            from_smem(v, sm, c);
            __syncthreads();
            // SWAP X^m = X^{m with bits q0, q1 exchanged} SWAP
            if (g.cls == GC_SWAP && (((c.m >> g.q0) ^ (c.m >> g.q1)) & 1u)) c.m ^= (1u << g.q0) | (1u << g.q1);
            break;
        }
        default: break;
    }
}

template <bool LAST>
__global__ void __launch_bounds__(512, 1) pass_rb_kernel(PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    __shared__ Partial red[32];
    __shared__ float2 ubuf[16];
    const int t = a.t, cl = a.c;
    const uint32_t slot = blockIdx.y;
    const uint64_t N = 1ull << a.n;
    int start, end = 0;
    uint64_t tr = 0;
    const float2 *src;
    float2 *dst;
    if (a.ideal) {
        start = 0;
        src = static_cast<const float2 *>(a.ideal_src);
        dst = static_cast<float2 *>(a.ideal_dst);
    } else {
        start = a.start_pass[slot];
        end = a.end_pass[slot];
        if (a.pass < start || a.pass > end) return;
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
    c.tid = threadIdx.x;
    c.nthr = blockDim.x;
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
            apply_gate_rb(v, c, gate, a.rpos[g], mats, sm, ubuf, t);
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
    if (!a.ideal && !a.store_last && a.pass == end) {
        const float2 *ref = static_cast<const float2 *>(a.cache) + (size_t)a.cache_slot[end + 1] * N;
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

// ------------------------------------------------------------- resident ---
// Whole state (2^n, 10 <= n <= 13) in one CTA: each trajectory restarts from
// the cached error-free state at the checkpoint (phase boundary) at or before
// its first error and runs the remaining phases; ckpt_every counts phases.

__device__ __forceinline__ void rb_load_linear(float2 (&v)[32], const float2 *src, int t, uint32_t tid) {
#pragma unroll
    for (int hi = 0; hi < 16; ++hi) {
        const uint32_t j = ((uint32_t)hi << (t - 4)) | (tid << 1);
        const float4 w = __ldg(reinterpret_cast<const float4 *>(src + j));
        v[2 * hi] = make_float2(w.x, w.y);
        v[2 * hi + 1] = make_float2(w.z, w.w);
    }
}

// store the true state (mask and global phase applied); leaves v in the load mapping
__device__ __forceinline__ void rb_store_linear(float2 (&v)[32], float2 *sm, TileCtx &c, uint32_t &cur_packed,
                                                uint32_t load_packed, float2 *dst, int t) {
    if (cur_packed != load_packed) {
        remap(v, sm, c, load_packed, t);
        cur_packed = load_packed;
    }
    const uint32_t flip0 = c.m & 1u;
    const uint32_t k2 = 2u * c.gp;
#pragma unroll
    for (int hi = 0; hi < 16; ++hi) {
        const uint32_t j = (((uint32_t)hi << (t - 4)) | (c.tid << 1)) ^ (c.m & ~1u);
        float2 e = flip0 ? v[2 * hi + 1] : v[2 * hi];
        float2 o = flip0 ? v[2 * hi] : v[2 * hi + 1];
        if (k2) {
            e = omega_mul(e, k2);
            o = omega_mul(o, k2);
        }
        reinterpret_cast<float4 *>(dst + j)[0] = make_float4(e.x, e.y, o.x, o.y);
    }
}

template <int MODE>
__global__ void __launch_bounds__(512, 1) resident_rb_kernel(ResidentArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    __shared__ Partial red[32];
    __shared__ float2 ubuf[16];
    const int t = a.n;
    const uint32_t N = 1u << t;
    const float2 *cache = static_cast<const float2 *>(a.cache);
    const float2 *mats = static_cast<const float2 *>(a.mats);
    const uint32_t load_packed = 0u | ((uint32_t)(t - 4) << 5) | ((uint32_t)(t - 3) << 10) |
                                 ((uint32_t)(t - 2) << 15) | ((uint32_t)(t - 1) << 20);
    const uint64_t count = MODE == 2 ? 1 : a.count;
    for (uint64_t b = blockIdx.x; b < count; b += gridDim.x) {
        float2 v[32];
        TileCtx c;
        c.m = 0;
        c.gp = 0;
        c.tid = threadIdx.x;
        c.nthr = blockDim.x;
        set_phase(c, load_packed, t);
        uint32_t cur_packed = load_packed;
        uint32_t ph0 = 0;
        const uint32_t *ev = nullptr, *ev_end = nullptr;
        uint64_t tr = 0;
        if (MODE == 2) {
#pragma unroll
            for (int ri = 0; ri < 32; ++ri) v[ri] = make_float2(0.f, 0.f);
            if (threadIdx.x == 0) v[0] = make_float2(1.f, 0.f);
        } else {
            tr = a.first_traj + b;
            const uint32_t first = a.first[tr];
            if (MODE == 0 && first == NO_EVENT) {
                if (threadIdx.x == 0) {
                    a.score[tr] = *a.ref_score;
                    if (a.pass_flags) a.pass_flags[tr] = *a.ref_score >= a.crit.threshold;
                }
                continue;
            }
            uint32_t ck;
            if (first == NO_EVENT) {
                ck = a.n_ckpt - 1;
                ph0 = a.n_phases;
            } else {
                ck = a.phase_of_pos[first] / (uint32_t)a.ckpt_every;
                ph0 = ck * (uint32_t)a.ckpt_every;
            }
            rb_load_linear(v, cache + (size_t)ck * N, t, c.tid);
            ev = a.keys + a.offsets[tr];
            ev_end = a.keys + a.offsets[tr + 1];
        }
        uint32_t next = ev && ev < ev_end ? *ev : NO_EVENT;
        for (uint32_t ph = ph0; ph < a.n_phases; ++ph) {
            if (MODE == 2 && ph % (uint32_t)a.ckpt_every == 0) {
                float2 *dst = const_cast<float2 *>(cache) + (size_t)(ph / (uint32_t)a.ckpt_every) * N;
                rb_store_linear(v, sm, c, cur_packed, load_packed, dst, t);
            }
            const uint32_t R = a.ph_R[ph];
            if (R != cur_packed) {
                remap(v, sm, c, R, t);
                cur_packed = R;
            }
            const uint32_t ge = a.ph_gb[ph + 1];
            for (uint32_t g = a.ph_gb[ph]; g < ge; ++g) {
                const DGate gate = a.gates[g];
                apply_gate_rb(v, c, gate, a.rpos[g], mats, sm, ubuf, t);
                while (next != NO_EVENT && ev_pos(next) == g) {
                    rg_pauli(v, c, ev_slot(next) ? gate.q1 : gate.q0, ev_code(next));
                    ++ev;
                    next = ev < ev_end ? *ev : NO_EVENT;
                }
            }
        }
        if (MODE == 2) {
            rb_store_linear(v, sm, c, cur_packed, load_packed, const_cast<float2 *>(cache) + (size_t)(a.n_ckpt - 1) * N,
                            t);
        } else if (MODE == 1) {
            rb_store_linear(v, sm, c, cur_packed, load_packed, static_cast<float2 *>(a.states_out) + (size_t)b * N, t);
        } else {
            if (c.gp) {
#pragma unroll
                for (int ri = 0; ri < 32; ++ri) v[ri] = omega_mul(v[ri], 2u * c.gp);
            }
            const float2 *ref = cache + (size_t)(a.n_ckpt - 1) * N;
            Partial acc = empty_partial();
#pragma unroll
            for (int ri = 0; ri < 32; ++ri) {
                const uint32_t jj = (c.tpart | reg_part(ri, c.r)) ^ c.m;
                accumulate(acc, a.crit, v[ri], ref, jj);
            }
            acc = block_reduce_partial(acc, red);
            if (threadIdx.x == 0) {
                const double sc = finish_score(a.crit, acc);
                a.score[tr] = sc;
                if (a.pass_flags) a.pass_flags[tr] = sc >= a.crit.threshold;
            }
        }
        __syncthreads();  // shared memory and red[] are reused by the next trajectory
    }
}

void launch_resident_rb(const ResidentArgs &a, int mode, double bytes, cudaStream_t st) {
    ProfScope ps_(ARSO_K_RESIDENT, bytes, st);
    const int nt = 1 << (a.n - REG_BITS);
    const size_t smem = (size_t(1) << a.n) * sizeof(float2);
    const void *fn = mode == 0 ? (const void *)resident_rb_kernel<0>
                   : mode == 1 ? (const void *)resident_rb_kernel<1> : (const void *)resident_rb_kernel<2>;
    if (smem > 48 * 1024) ARSO_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 1;
    ARSO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem));
    int dev = 0, sms = 152;
    ARSO_CUDA(cudaGetDevice(&dev));
    ARSO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint64_t want = mode == 2 ? 1 : a.count;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::max(per_sm, 1) * sms));
    if (mode == 0) resident_rb_kernel<0><<<grid, nt, smem, st>>>(a);
    else if (mode == 1) resident_rb_kernel<1><<<grid, nt, smem, st>>>(a);
    else resident_rb_kernel<2><<<grid, nt, smem, st>>>(a);
    ARSO_CUDA(cudaGetLastError());
}

// --------------------------------------------------------- batched resident ---
// Persistent CTAs of 256 threads pull (circuit, trajectory block) items from a
// device counter. A circuit of n qubits needs 2^(n-5) threads per trajectory,
// so one CTA runs 2^(13-n) trajectories of the same circuit side by side: the
// sub-groups share the circuit's phase program (uniform barriers) and keep
// their own registers, shared-memory tile, index mask and error events.
constexpr int BATCH_THREADS = 256;

__global__ void __launch_bounds__(BATCH_THREADS, 2)
    batch_resident_kernel(const BatchCircuit *__restrict__ circs, const BatchItem *__restrict__ items, uint32_t n_items,
                          uint32_t *counter, const uint64_t *__restrict__ ids) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_item;
    __shared__ Partial red[BATCH_THREADS / 32];
    __shared__ float2 ubuf[8][16];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_items) return;
        const BatchItem it = items[item];
        const BatchCircuit &C = circs[it.circuit];
        const int t = C.n;
        const uint32_t N = 1u << t, gsize = 1u << (t - REG_BITS), sg = threadIdx.x / gsize;
        float2 *sm = reinterpret_cast<float2 *>(smem_raw) + (size_t)sg * N;
        const bool active = sg < it.count;
        const uint64_t tr = ids[it.off + (active ? sg : 0)];
        const uint32_t load_packed = 0u | ((uint32_t)(t - 4) << 5) | ((uint32_t)(t - 3) << 10) |
                                     ((uint32_t)(t - 2) << 15) | ((uint32_t)(t - 1) << 20);
        TileCtx c;
        c.m = 0;
        c.gp = 0;
        c.tid = threadIdx.x % gsize;
        c.nthr = gsize;
        set_phase(c, load_packed, t);
        float2 v[32];
        rb_load_linear(v, C.cache + (size_t)it.ck * N, t, c.tid);
        const uint32_t *ev = C.keys + C.offsets[tr];
        const uint32_t *ev_end = C.keys + C.offsets[tr + 1];
        uint32_t next = ev < ev_end ? *ev : NO_EVENT;
        uint32_t cur_packed = load_packed;
        for (uint32_t ph = it.ck * C.ckpt_every; ph < C.n_phases; ++ph) {
            const uint32_t R = C.ph_R[ph];
            if (R != cur_packed) {
                remap(v, sm, c, R, t);
                cur_packed = R;
            }
            const uint32_t ge = C.ph_gb[ph + 1];
            for (uint32_t g = C.ph_gb[ph]; g < ge; ++g) {
                const DGate gate = C.gates[g];
                apply_gate_rb(v, c, gate, C.rpos[g], C.mats, sm, ubuf[sg], t);
                while (next != NO_EVENT && ev_pos(next) == g) {
                    rg_pauli(v, c, ev_slot(next) ? gate.q1 : gate.q0, ev_code(next));
                    ++ev;
                    next = ev < ev_end ? *ev : NO_EVENT;
                }
            }
        }
        if (c.gp) {
#pragma unroll
            for (int ri = 0; ri < 32; ++ri) v[ri] = omega_mul(v[ri], 2u * c.gp);
        }
        const float2 *ref = C.cache + (size_t)(C.n_ckpt - 1) * N;
        Partial acc = empty_partial();
#pragma unroll
        for (int ri = 0; ri < 32; ++ri) {
            const uint32_t jj = (c.tpart | reg_part(ri, c.r)) ^ c.m;
            accumulate(acc, C.crit, v[ri], ref, jj);
        }
        // per sub-group reduction: warps reduce by shuffles, the sub-group leader combines its warps
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double a2 = __shfl_down_sync(0xffffffffu, acc.a, o);
            const double b2 = __shfl_down_sync(0xffffffffu, acc.b, o);
            const double mp = __shfl_down_sync(0xffffffffu, acc.maxp, o);
            const unsigned long long mi = __shfl_down_sync(0xffffffffu, acc.idx, o);
            acc.a += a2;
            acc.b += b2;
            argmax_merge(acc.maxp, acc.idx, mp, mi);
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (c.tid == 0 && active) {
            Partial s = empty_partial();
            const uint32_t w0 = (sg * gsize) >> 5, nw = gsize >> 5;
            for (uint32_t w = w0; w < w0 + nw; ++w) {
                s.a += red[w].a;
                s.b += red[w].b;
                argmax_merge(s.maxp, s.idx, red[w].maxp, red[w].idx);
            }
            const double sc = finish_score(C.crit, s);
            C.score[tr] = sc;
            if (C.pass_flags) C.pass_flags[tr] = sc >= C.crit.threshold;
        }
    }
}

void launch_batch_resident(const BatchCircuit *circs, const BatchItem *items, uint32_t n_items, uint32_t *counter,
                           const uint64_t *ids, double bytes, cudaStream_t st) {
    if (!n_items) return;
    ProfScope ps_(ARSO_K_RESIDENT, bytes, st);
    const size_t smem = (size_t(1) << 13) * sizeof(float2);
    ARSO_CUDA(cudaFuncSetAttribute(batch_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 1, dev = 0, sms = 152;
    ARSO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_resident_kernel, BATCH_THREADS, smem));
    ARSO_CUDA(cudaGetDevice(&dev));
    ARSO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)std::min<uint64_t>(n_items, (uint64_t)std::max(per_sm, 1) * sms);
    batch_resident_kernel<<<grid, BATCH_THREADS, smem, st>>>(circs, items, n_items, counter, ids);
    ARSO_CUDA(cudaGetLastError());
}

// Raise the dynamic shared-memory limit of both pass variants once, before any
// launch (and outside stream capture).
void prepare_pass_rb() {
    static bool done = false;
    if (done) return;
    const int smem = (1 << MAX_TILE_QUBITS) * (int)sizeof(float2);
    ARSO_CUDA(cudaFuncSetAttribute(pass_rb_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ARSO_CUDA(cudaFuncSetAttribute(pass_rb_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    done = true;
}

void launch_pass_rb(const PassArgs &a, bool last, uint32_t slots, double bytes, cudaStream_t st) {
    ProfScope ps_(last && !a.store_last ? ARSO_K_PASS_LAST : ARSO_K_PASS, bytes, st);
    prepare_pass_rb();
    const uint32_t tiles = 1u << (a.n - a.t);
    const int nt = 1 << (a.t - REG_BITS);
    const size_t smem = (size_t(1) << a.t) * sizeof(float2);
    dim3 grid(tiles, slots);
    if (last) pass_rb_kernel<true><<<grid, nt, smem, st>>>(a);
    else pass_rb_kernel<false><<<grid, nt, smem, st>>>(a);
    ARSO_CUDA(cudaGetLastError());
}

}  // namespace arso
