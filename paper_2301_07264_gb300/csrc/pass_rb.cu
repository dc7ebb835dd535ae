// Register-blocked fused tile pass (complex64, tiles of 2^t >= 2^10 amplitudes).
//
// A CTA of 2^(t-5) threads owns one tile of one trajectory; every thread
// keeps 32 amplitudes in registers. The tile-local index of register ri of
// thread tid is deposit(ri, R) | deposit(tid, complement of R), where R, the 5
// "register bits", changes only between phases (a swizzled shared-memory
// transpose). Register bit 0 is always tile bit 0, so registers 2k and 2k+1
// hold the neighbours j and j|1; they are kept split as two FP32x2 pairs,
// re[k] = (Re a_j, Re a_j|1) and im[k] = (Im a_j, Im a_j|1), and one packed
// instruction (FFMA2 / FMUL2 / FADD2) updates both. Within a phase:
//  * dense one-qubit gates, H and CX targets act on register bits, entirely
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
#include <cuda_fp16.h>

#include <algorithm>

#include "prof.h"
#include "sim_common.cuh"
#include "umma.cuh"

namespace arso {

__device__ __forceinline__ uint32_t swz(uint32_t j) { return j ^ (((j >> 4) ^ (j >> 8) ^ (j >> 12)) & 15u); }

// register bit b of a packed register set (the five bits are stored in ascending order)
__device__ __forceinline__ uint32_t rbit(uint32_t packed, int b) { return (packed >> (5 * b)) & 31u; }

// tid's bits deposited into the tile bits that are not register bits, ascending:
// a zero bit inserted at each register bit position, lowest first
__device__ __forceinline__ uint32_t thread_part(uint32_t tid, uint32_t packed) {
    uint32_t x = tid;
#pragma unroll
    for (int b = 0; b < REG_BITS; ++b) {
        const uint32_t r = rbit(packed, b);
        x = ((x >> r) << (r + 1)) | (x & ((1u << r) - 1u));
    }
    return x;
}


// register part of the local index of register ri (ri is a constant after unrolling)
__device__ __forceinline__ uint32_t reg_part(int ri, uint32_t packed) {
    uint32_t o = 0;
#pragma unroll
    for (int b = 0; b < REG_BITS; ++b)
        if ((ri >> b) & 1) o |= 1u << rbit(packed, b);
    return o;
}

// ----------------------------------------------------------- amplitudes ---
struct Amps {
    float2 re[16], im[16];  // re[k] = (Re of register 2k, Re of register 2k+1)
};

__device__ __forceinline__ float2 amp_get(const Amps &a, int ri) {
    const float2 r = a.re[ri >> 1], i = a.im[ri >> 1];
    return (ri & 1) ? make_float2(r.y, i.y) : make_float2(r.x, i.x);
}
__device__ __forceinline__ void amp_set(Amps &a, int ri, float2 v) {
    if (ri & 1) {
        a.re[ri >> 1].y = v.x;
        a.im[ri >> 1].y = v.y;
    } else {
        a.re[ri >> 1].x = v.x;
        a.im[ri >> 1].x = v.y;
    }
}

__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 swp2(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// ------------------------------------------------------- register gates ---
// Code size matters: the whole phase loop must stay resident in the
// instruction cache, so only dense one-qubit gates, H, phase gates and CZ are
// specialised per register position; everything else is position-free.

// U on register bit P >= 1: packed registers k and k | 2^(P-1) hold the pairs
template <int P>
__device__ __forceinline__ void rg_dense1(Amps &a, float2 u00, float2 u01, float2 u10, float2 u11) {
    const float2 u00r = bc2(u00.x), u00i = bc2(u00.y), n00i = bc2(-u00.y);
    const float2 u01r = bc2(u01.x), u01i = bc2(u01.y), n01i = bc2(-u01.y);
    const float2 u10r = bc2(u10.x), u10i = bc2(u10.y), n10i = bc2(-u10.y);
    const float2 u11r = bc2(u11.x), u11i = bc2(u11.y), n11i = bc2(-u11.y);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (k & (1 << (P - 1))) continue;
        const int k1 = k | (1 << (P - 1));
        const float2 r0 = a.re[k], i0 = a.im[k], r1 = a.re[k1], i1 = a.im[k1];
        a.re[k] = fma2(n01i, i1, fma2(u01r, r1, fma2(n00i, i0, mul2(u00r, r0))));
        a.im[k] = fma2(u01i, r1, fma2(u01r, i1, fma2(u00i, r0, mul2(u00r, i0))));
        a.re[k1] = fma2(n11i, i1, fma2(u11r, r1, fma2(n10i, i0, mul2(u10r, r0))));
        a.im[k1] = fma2(u11i, r1, fma2(u11r, i1, fma2(u10i, r0, mul2(u10r, i0))));
    }
}

// Special unitary U = [[a, b], [-conj b, conj a]] on register bit P >= 1:
// seven broadcast constants instead of twelve keep the phase loop spill-free.
template <int P> __device__ __forceinline__ void rg_su2(Amps &a, float2 ua, float2 ub) {
    const float2 ar = bc2(ua.x), ai = bc2(ua.y), nai = bc2(-ua.y);
    const float2 br = bc2(ub.x), bi = bc2(ub.y), nbi = bc2(-ub.y), nbr = bc2(-ub.x);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (k & (1 << (P - 1))) continue;
        const int k1 = k | (1 << (P - 1));
        const float2 r0 = a.re[k], i0 = a.im[k], r1 = a.re[k1], i1 = a.im[k1];
        a.re[k] = fma2(nbi, i1, fma2(br, r1, fma2(nai, i0, mul2(ar, r0))));
        a.im[k] = fma2(bi, r1, fma2(br, i1, fma2(ai, r0, mul2(ar, i0))));
        a.re[k1] = fma2(ai, i1, fma2(ar, r1, fma2(nbi, i0, mul2(nbr, r0))));
        a.im[k1] = fma2(nai, r1, fma2(ar, i1, fma2(bi, r0, mul2(nbr, i0))));
    }
}

// U on register bit 0: the pair sits in the two lanes of one packed register;
// lane 0 takes (u00, u01) against (a0, a1), lane 1 takes (u11, u10) against (a1, a0).
__device__ __forceinline__ void rg_dense1_lanes(Amps &a, float2 u00, float2 u01, float2 u10, float2 u11) {
    const float2 dr = make_float2(u00.x, u11.x), di = make_float2(u00.y, u11.y), ndi = make_float2(-u00.y, -u11.y);
    const float2 xr = make_float2(u01.x, u10.x), xi = make_float2(u01.y, u10.y), nxi = make_float2(-u01.y, -u10.y);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float2 r = a.re[k], i = a.im[k], rs = swp2(r), is = swp2(i);
        a.re[k] = fma2(nxi, is, fma2(xr, rs, fma2(ndi, i, mul2(dr, r))));
        a.im[k] = fma2(xi, rs, fma2(xr, is, fma2(di, r, mul2(dr, i))));
    }
}

// H on register bit P: (a0, a1) -> (a0 + a1, a0 - a1) / sqrt2 with 1/sqrt2
// applied as the compensated pair hi + lo. FLIP gives (a0 + a1, a1 - a0) /
// sqrt2, i.e. Z H, which is H on a qubit whose mask bit is set (H X = Z H:
// the caller then clears the mask bit).
template <int P, bool FLIP> __device__ __forceinline__ void rg_h(Amps &a) {
    const float2 hi = bc2(RSQRT2_HI), lo = bc2(RSQRT2_LO), m1 = bc2(-1.f);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (k & (1 << (P - 1))) continue;
        const int k1 = k | (1 << (P - 1));
        const float2 r0 = a.re[k], i0 = a.im[k], r1 = a.re[k1], i1 = a.im[k1];
        const float2 sr = add2(r0, r1), si = add2(i0, i1);
        const float2 dr = FLIP ? fma2(m1, r0, r1) : fma2(m1, r1, r0);
        const float2 di = FLIP ? fma2(m1, i0, i1) : fma2(m1, i1, i0);
        a.re[k] = fma2(hi, sr, mul2(lo, sr));
        a.im[k] = fma2(hi, si, mul2(lo, si));
        a.re[k1] = fma2(hi, dr, mul2(lo, dr));
        a.im[k1] = fma2(hi, di, mul2(lo, di));
    }
}
template <int P> __device__ __forceinline__ void rg_h(Amps &a, uint32_t flip) {
    if (flip) rg_h<P, true>(a);
    else rg_h<P, false>(a);
}
__device__ __forceinline__ void rg_h_lanes(Amps &a, float sg) {
    const float2 pm = make_float2(1.f, -1.f);
    const float2 h = make_float2(RSQRT2_HI, sg * RSQRT2_HI), l = make_float2(RSQRT2_LO, sg * RSQRT2_LO);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float2 tr = fma2(pm, a.re[k], swp2(a.re[k]));  // (a0 + a1, a0 - a1)
        const float2 ti = fma2(pm, a.im[k], swp2(a.im[k]));
        a.re[k] = fma2(h, tr, mul2(l, tr));
        a.im[k] = fma2(h, ti, mul2(l, ti));
    }
}

// CX on stored data, target register bit P; control is register bit cpos
// (0..4) or, when cpos == 15, the thread-level bit value cth.
template <int P> __device__ __forceinline__ void rg_cx(Amps &a, uint32_t cpos, uint32_t cth) {
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        if (ri & (1 << P)) continue;
        const uint32_t ctl = cpos < REG_BITS ? (((uint32_t)ri >> cpos) & 1u) : cth;
        const float2 a0 = amp_get(a, ri), a1 = amp_get(a, ri | (1 << P));
        amp_set(a, ri, ctl ? a1 : a0);
        amp_set(a, ri | (1 << P), ctl ? a0 : a1);
    }
}

// Value of tile bit q of the true index (stored index ^ m) for register ri:
// register bit pos < 5 -> (ri >> pos) ^ mq; else the thread-level value th.
__device__ __forceinline__ uint32_t bit_of(int ri, uint32_t pos, uint32_t mq, uint32_t th) {
    return pos < REG_BITS ? ((((uint32_t)ri >> pos) & 1u) ^ mq) : th;
}

struct TileCtx {
    uint32_t R;          // register bits of the current phase, 5 bits each (bit 0 of the tile first)
    uint32_t tpart;      // thread part of the local index
    uint32_t m;          // X mask (stored[j] = state[j ^ m])
    uint32_t gp;         // global phase i^gp
    uint32_t tid, nthr;  // thread index within the tile's thread group, group size
};

__device__ __forceinline__ uint32_t reg_pos(const TileCtx &c, uint32_t q) {
    uint32_t p = 15;
#pragma unroll
    for (int b = 0; b < REG_BITS; ++b)
        if (rbit(c.R, b) == q) p = (uint32_t)b;
    return p;
}
// true value of tile bit q held at thread level
__device__ __forceinline__ uint32_t thread_bit(const TileCtx &c, uint32_t q) { return ((c.tpart ^ c.m) >> q) & 1u; }

// diag(d0, d1) on tile bit q (true index) at register position pos (15: thread bit)
__device__ __forceinline__ void rg_diag1(Amps &a, const TileCtx &c, uint32_t q, uint32_t pos, float2 d0, float2 d1) {
    const uint32_t mq = (c.m >> q) & 1u, th = thread_bit(c, q);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t bx = bit_of(2 * k, pos, mq, th), by = bit_of(2 * k + 1, pos, mq, th);
        const float2 fr = make_float2(bx ? d1.x : d0.x, by ? d1.x : d0.x);
        const float2 fi = make_float2(bx ? d1.y : d0.y, by ? d1.y : d0.y);
        const float2 nfi = make_float2(-fi.x, -fi.y);
        const float2 r = a.re[k], i = a.im[k];
        a.re[k] = fma2(nfi, i, mul2(fr, r));
        a.im[k] = fma2(fi, r, mul2(fr, i));
    }
}

// diag(1, e^{i k pi/4}) on tile bit q, written per lane as kappa (A + i B)
// with A, B in {0, +-1} and kappa = 1/sqrt2 (odd k, compensated hi + lo) or 1.
// (R, I) -> kappa (A R - B I, B R + A I): the products by 0 and +-1 are exact,
// so lanes with (A, B, hi, lo) = (1, 0, 1, 0) pass through unchanged.
struct PhaseOp {
    float2 A, B, nB, H, L;
};
__device__ __forceinline__ void phase_pk(float2 &r, float2 &i, const PhaseOp &o) {
    float2 t1 = fma2(o.nB, i, mul2(o.A, r));
    float2 t2 = fma2(o.B, r, mul2(o.A, i));
    r = fma2(o.H, t1, mul2(o.L, t1));
    i = fma2(o.H, t2, mul2(o.L, t2));
}
__device__ __forceinline__ void omega_ab(uint32_t k, float &A, float &B, float &H, float &L) {
    const uint32_t q = (k >> 1) & 3u;
    const float cq = q == 0 ? 1.f : (q == 2 ? -1.f : 0.f), sq = q == 1 ? 1.f : (q == 3 ? -1.f : 0.f);
    if (k & 1u) {  // i^q (1 + i) / sqrt2
        A = cq - sq;
        B = cq + sq;
        H = RSQRT2_HI;
        L = RSQRT2_LO;
    } else {
        A = cq;
        B = sq;
        H = 1.f;
        L = 0.f;
    }
}
template <int P> __device__ __forceinline__ void rg_omega_half(Amps &a, const PhaseOp &op, uint32_t want) {
    if (want) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k & (1 << (P - 1))) phase_pk(a.re[k], a.im[k], op);
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (!(k & (1 << (P - 1)))) phase_pk(a.re[k], a.im[k], op);
    }
}
__device__ __forceinline__ void rg_omega(Amps &a, const TileCtx &c, uint32_t q, uint32_t pos, uint32_t k) {
    float A, B, H, L;
    omega_ab(k, A, B, H, L);
    if (pos >= REG_BITS) {
        if (thread_bit(c, q)) {
            const PhaseOp op{bc2(A), bc2(B), bc2(-B), bc2(H), bc2(L)};
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) phase_pk(a.re[kk], a.im[kk], op);
        }
        return;
    }
    const uint32_t want = ((c.m >> q) & 1u) ^ 1u;  // stored bit value whose true bit is 1
    if (pos == 0) {
        // lane `want` of every packed register
        const PhaseOp op = want ? PhaseOp{make_float2(1.f, A), make_float2(0.f, B), make_float2(0.f, -B),
                                          make_float2(1.f, H), make_float2(0.f, L)}
                                : PhaseOp{make_float2(A, 1.f), make_float2(B, 0.f), make_float2(-B, 0.f),
                                          make_float2(H, 1.f), make_float2(L, 0.f)};
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) phase_pk(a.re[kk], a.im[kk], op);
        return;
    }
    const PhaseOp op{bc2(A), bc2(B), bc2(-B), bc2(H), bc2(L)};
    switch (pos) {
        case 1: rg_omega_half<1>(a, op, want); break;
        case 2: rg_omega_half<2>(a, op, want); break;
        case 3: rg_omega_half<3>(a, op, want); break;
        default: rg_omega_half<4>(a, op, want); break;
    }
}

// Registers whose tile bit q (of the true index) is 1, as a 32-bit mask.
__device__ __forceinline__ uint32_t reg_pattern(uint32_t pos) {
    return pos == 0 ? 0xAAAAAAAAu : pos == 1 ? 0xCCCCCCCCu : pos == 2 ? 0xF0F0F0F0u : pos == 3 ? 0xFF00FF00u : 0xFFFF0000u;
}
__device__ __forceinline__ uint32_t bit_mask(const TileCtx &c, uint32_t q) {
    const uint32_t pos = reg_pos(c, q);
    if (pos < REG_BITS) return ((c.m >> q) & 1u) ? ~reg_pattern(pos) : reg_pattern(pos);
    return thread_bit(c, q) ? 0xFFFFFFFFu : 0u;
}
__device__ __forceinline__ uint32_t sign_bit(uint32_t mask, int ri) { return (mask << (31 - ri)) & 0x80000000u; }
// negate the registers selected by mask: flip the sign bits
__device__ __forceinline__ void negate_masked(Amps &a, uint32_t mask) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t sx = sign_bit(mask, 2 * k), sy = sign_bit(mask, 2 * k + 1);
        a.re[k].x = __uint_as_float(__float_as_uint(a.re[k].x) ^ sx);
        a.im[k].x = __uint_as_float(__float_as_uint(a.im[k].x) ^ sx);
        a.re[k].y = __uint_as_float(__float_as_uint(a.re[k].y) ^ sy);
        a.im[k].y = __uint_as_float(__float_as_uint(a.im[k].y) ^ sy);
    }
}

// CZ: negate the registers whose stored bits at positions PA and PB equal
// (WA, WB). Both bits in registers: 8 of the 32 amplitudes, fixed at compile
// time (40 variants); packed registers are negated with one FMUL2 by (-1, -1)
// or (-1, 1) per plane.
template <int PA, int PB, int WA, int WB> __device__ __forceinline__ void neg_quarter(Amps &a) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const bool nx = ((((2 * k) >> PA) & 1) == WA) && ((((2 * k) >> PB) & 1) == WB);
        const bool ny = ((((2 * k + 1) >> PA) & 1) == WA) && ((((2 * k + 1) >> PB) & 1) == WB);
        if (!nx && !ny) continue;
        const float2 s = make_float2(nx ? -1.f : 1.f, ny ? -1.f : 1.f);
        a.re[k] = mul2(s, a.re[k]);
        a.im[k] = mul2(s, a.im[k]);
    }
}
template <int P, int W> __device__ __forceinline__ void neg_half(Amps &a) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const bool nx = (((2 * k) >> P) & 1) == W, ny = (((2 * k + 1) >> P) & 1) == W;
        if (!nx && !ny) continue;
        const float2 s = make_float2(nx ? -1.f : 1.f, ny ? -1.f : 1.f);
        a.re[k] = mul2(s, a.re[k]);
        a.im[k] = mul2(s, a.im[k]);
    }
}
__host__ __device__ constexpr int cz_pa(int pp) { return pp < 4 ? 0 : pp < 7 ? 1 : pp < 9 ? 2 : 3; }
__host__ __device__ constexpr int cz_pb(int pp) {
    return pp < 4 ? pp + 1 : pp < 7 ? pp - 2 : pp < 9 ? pp - 4 : 4;
}
template <int IDX> __device__ __forceinline__ void cz_case(Amps &a) {
    neg_quarter<cz_pa(IDX >> 2), cz_pb(IDX >> 2), (IDX >> 1) & 1, IDX & 1>(a);
}

__device__ __forceinline__ void rg_diag2(Amps &a, const TileCtx &c, uint32_t qa, uint32_t qb,
                                         const float2 *__restrict__ d) {
    const uint32_t pa = reg_pos(c, qa), ma = (c.m >> qa) & 1u, ta = thread_bit(c, qa);
    const uint32_t pb = reg_pos(c, qb), mb = (c.m >> qb) & 1u, tb = thread_bit(c, qb);
    const float2 d0 = d[0], d1 = d[1], d2 = d[2], d3 = d[3];
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        const uint32_t k = bit_of(ri, pa, ma, ta) | (bit_of(ri, pb, mb, tb) << 1);
        const float2 f = k == 0 ? d0 : (k == 1 ? d1 : (k == 2 ? d2 : d3));
        amp_set(a, ri, cmul(f, amp_get(a, ri)));
    }
}

// Pauli error on tile bit q of the true state (Eq. (2)): Z -> phase -1 on
// bit q; X -> index mask; Y = i X Z.
__device__ __forceinline__ void rg_pauli(Amps &a, TileCtx &c, uint32_t q, uint32_t code) {
    if (code & 2u) {  // Z part (Z or Y): negate where bit q of the true index is 1
        const uint32_t mask = bit_mask(c, q);
        if (mask) negate_masked(a, mask);
    }
    if (code & 1u) c.m ^= 1u << q;          // X part (X or Y)
    if (code == 3u) c.gp = (c.gp + 1u) & 3u;  // Y = i X Z
}

// multiply every amplitude by i^gp (exact) and reset gp
__device__ __forceinline__ void apply_global_phase(Amps &a, TileCtx &c) {
    if (!c.gp) return;
    const float2 A = bc2(c.gp == 2 ? -1.f : (c.gp == 0 ? 1.f : 0.f)), B = bc2(c.gp == 1 ? 1.f : (c.gp == 3 ? -1.f : 0.f));
    const float2 nB = make_float2(-B.x, -B.y);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float2 r = a.re[k], i = a.im[k];
        a.re[k] = fma2(nB, i, mul2(A, r));
        a.im[k] = fma2(B, r, mul2(A, i));
    }
    c.gp = 0;
}

// stored index -> tile-local index bits for the load/store mapping
__device__ __forceinline__ void set_phase(TileCtx &c, uint32_t packed, int t) {
    c.R = packed;
    c.tpart = thread_part(c.tid, packed);
}

// Shared memory holds a tile as two planes of packed neighbour pairs:
// plane_re[swz(J)] = (Re a_2J, Re a_2J+1) and plane_im likewise, plane_im =
// plane_re + 2^(t-1). The swizzle is linear over XOR, so the slot of packed
// register k is swz(tpart >> 1) ^ (XOR of swz(2^(r[b]-1)) over the set bits
// b-1 of k); walking the registers in Gray-code order costs one XOR each.
__host__ __device__ constexpr int ctz4(int x) { return x & 1 ? 0 : x & 2 ? 1 : x & 4 ? 2 : 3; }

__device__ __forceinline__ void smem_basis(const TileCtx &c, uint32_t &base, uint32_t (&sw)[REG_BITS - 1]) {
    base = swz(c.tpart >> 1);
#pragma unroll
    for (int b = 1; b < REG_BITS; ++b) sw[b - 1] = swz(1u << (rbit(c.R, b) - 1));
}
__device__ __forceinline__ void to_smem(const Amps &a, float2 *sm, const TileCtx &c, int t) {
    uint32_t idx, sw[REG_BITS - 1];
    smem_basis(c, idx, sw);
    float2 *pim = sm + (1u << (t - 1));
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
        const int k = kk ^ (kk >> 1);
        sm[idx] = a.re[k];
        pim[idx] = a.im[k];
        if (kk < 15) idx ^= sw[ctz4(kk + 1)];
    }
}
__device__ __forceinline__ void from_smem(Amps &a, const float2 *sm, const TileCtx &c, int t) {
    uint32_t idx, sw[REG_BITS - 1];
    smem_basis(c, idx, sw);
    const float2 *pim = sm + (1u << (t - 1));
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
        const int k = kk ^ (kk >> 1);
        a.re[k] = sm[idx];
        a.im[k] = pim[idx];
        if (kk < 15) idx ^= sw[ctz4(kk + 1)];
    }
}

// SYNCED: the caller has just synced the CTA after the last shared-memory
// read (a phase start), so the first barrier is not needed.
template <bool SYNCED = false>
__device__ __forceinline__ void remap(Amps &a, float2 *sm, TileCtx &c, uint32_t packed, int t) {
    if (!SYNCED) __syncthreads();
    to_smem(a, sm, c, t);
    set_phase(c, packed, t);
    __syncthreads();
    from_smem(a, sm, c, t);
}

// Dense two-qubit gates and SWAP are rare: they run through shared memory on
// the stored data (U already conjugated by the mask) with runtime indices.
__device__ __forceinline__ void smem_dense2(float2 *sm, int t, uint32_t q0, uint32_t q1, const float2 *__restrict__ U,
                                            uint32_t tid, uint32_t nthr) {
    float *pre = reinterpret_cast<float *>(sm);
    float *pim = reinterpret_cast<float *>(sm + (1u << (t - 1)));
    const uint32_t lo = q0 < q1 ? q0 : q1, hi = q0 < q1 ? q1 : q0;
    const uint32_t m0 = 1u << q0, m1 = 1u << q1;
    float2 M[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) M[k] = U[k];
    for (uint32_t p = tid; p < (1u << (t - 2)); p += nthr) {
        const uint32_t i = insert_zero2(p, lo, hi);
        const uint32_t jx[4] = {i, i | m0, i | m1, i | m0 | m1};
        uint32_t ix[4];
        float2 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ix[k] = 2u * swz(jx[k] >> 1) + (jx[k] & 1u);
            v[k] = make_float2(pre[ix[k]], pim[ix[k]]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 acc = cmac2(M[4 * k], v[0], M[4 * k + 1], v[1]);
            const float2 acc2 = cmac2(M[4 * k + 2], v[2], M[4 * k + 3], v[3]);
            pre[ix[k]] = acc.x + acc2.x;
            pim[ix[k]] = acc.y + acc2.y;
        }
    }
}

// CZ from the host-resolved code: pair of register positions, or one
// register position and a thread bit; the mask bits of the qubits select the
// sign pattern (want = 1 ^ mask bit).
#define ARSO_CZ_CASE(i) case OP_CZ_RR + (i): cz_case<(i)>(a); break;
#define ARSO_CZ_CASE4(i) ARSO_CZ_CASE(4 * (i)) ARSO_CZ_CASE(4 * (i) + 1) ARSO_CZ_CASE(4 * (i) + 2) ARSO_CZ_CASE(4 * (i) + 3)
__device__ __forceinline__ void rg_cz_code(Amps &a, const TileCtx &c, const RegOp &op, uint32_t q0, uint32_t q1,
                                           uint32_t p0) {
    const uint32_t x = op.pad[0];
    const uint32_t ba = ((c.m >> q0) ^ (x >> 12)) & 1u, bb = ((c.m >> q1) ^ (x >> 13)) & 1u;
    const uint32_t code = (x & 255u) + ba * ((x >> 8) & 3u) + bb * ((x >> 10) & 3u);
    if (code >= (uint32_t)OP_CZ_RT) {
        if (code == (uint32_t)OP_CZ_TT) {
            if (thread_bit(c, q0) && thread_bit(c, q1)) {
                const float2 m1 = bc2(-1.f);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    a.re[k] = mul2(m1, a.re[k]);
                    a.im[k] = mul2(m1, a.im[k]);
                }
            }
            return;
        }
        if (!thread_bit(c, p0 < REG_BITS ? q1 : q0)) return;
        switch (code - OP_CZ_RT) {
            case 0: neg_half<0, 0>(a); break;
            case 1: neg_half<0, 1>(a); break;
            case 2: neg_half<1, 0>(a); break;
            case 3: neg_half<1, 1>(a); break;
            case 4: neg_half<2, 0>(a); break;
            case 5: neg_half<2, 1>(a); break;
            case 6: neg_half<3, 0>(a); break;
            case 7: neg_half<3, 1>(a); break;
            case 8: neg_half<4, 0>(a); break;
            default: neg_half<4, 1>(a); break;
        }
        return;
    }
    switch (code) {
        ARSO_CZ_CASE4(0) ARSO_CZ_CASE4(1) ARSO_CZ_CASE4(2) ARSO_CZ_CASE4(3) ARSO_CZ_CASE4(4)
        ARSO_CZ_CASE4(5) ARSO_CZ_CASE4(6) ARSO_CZ_CASE4(7) ARSO_CZ_CASE4(8) ARSO_CZ_CASE4(9)
        default: break;
    }
}
#undef ARSO_CZ_CASE
#undef ARSO_CZ_CASE4

// One dispatch per gate on the host-resolved base op code (class and
// register positions); mask-dependent details (H on a flipped qubit, the CZ
// sign pattern) are resolved inside the case, so cheap gates pay no extra
// decoding.
#define ARSO_P4(BASE, CALL) \
    case BASE + 1: CALL(1); break; \
    case BASE + 2: CALL(2); break; \
    case BASE + 3: CALL(3); break; \
    case BASE + 4: CALL(4); break;
__device__ __forceinline__ void apply_op(Amps &a, TileCtx &c, const RegOp &op, const float2 *__restrict__ mats,
                                         float2 *sm, float2 *ubuf, int t) {
    const uint32_t p0 = (op.w0 >> 8) & 15u;
    const uint32_t q0 = (op.w0 >> 16) & 255u, q1 = op.w0 >> 24;
    const float2 *M = mats + op.aux;
    // X U X for the qubit's mask bit: for SU(2) [[conj a, -conj b], [b, a]], the same form;
    // for a general U [[u11, u10], [u01, u00]]
#define ARSO_FLIP ((c.m >> q0) & 1u)
#define ARSO_UA (ARSO_FLIP ? make_float2(op.c0.x, -op.c0.y) : op.c0)
#define ARSO_UB (ARSO_FLIP ? make_float2(-op.c1.x, op.c1.y) : op.c1)
#define ARSO_SU2(P) rg_su2<P>(a, ARSO_UA, ARSO_UB)
#define ARSO_D1(P) \
    rg_dense1<P>(a, M[ARSO_FLIP ? 3 : 0], M[ARSO_FLIP ? 2 : 1], M[ARSO_FLIP ? 1 : 2], M[ARSO_FLIP ? 0 : 3])
    // H on a flipped qubit: H X = Z H, so apply Z H and clear the mask bit
#define ARSO_HADAMARD(P) rg_h<P>(a, ARSO_FLIP); c.m &= ~(1u << q0)
    // CX X^m = X^{m'} CX with m' = m ^ (target bit if the control bit is in m)
#define ARSO_CX(P) rg_cx<P>(a, p0, (c.tpart >> q0) & 1u); if (ARSO_FLIP) c.m ^= 1u << q1
    switch (op.pad[0] & 255u) {
        case OP_SU2: {
            const float2 ua = ARSO_UA, ub = ARSO_UB;
            rg_dense1_lanes(a, ua, ub, make_float2(-ub.x, ub.y), make_float2(ua.x, -ua.y));
            break;
        }
        ARSO_P4(OP_SU2, ARSO_SU2)
        case OP_DENSE1: {
            const uint32_t f = ARSO_FLIP;
            rg_dense1_lanes(a, M[f ? 3 : 0], M[f ? 2 : 1], M[f ? 1 : 2], M[f ? 0 : 3]);
            break;
        }
        ARSO_P4(OP_DENSE1, ARSO_D1)
        case OP_H: rg_h_lanes(a, ARSO_FLIP ? -1.f : 1.f); c.m &= ~(1u << q0); break;
        case OP_H + 2: ARSO_HADAMARD(1); break;
        case OP_H + 4: ARSO_HADAMARD(2); break;
        case OP_H + 6: ARSO_HADAMARD(3); break;
        case OP_H + 8: ARSO_HADAMARD(4); break;
        case OP_CZ_RR + 0: case OP_CZ_RR + 4: case OP_CZ_RR + 8: case OP_CZ_RR + 12: case OP_CZ_RR + 16:
        case OP_CZ_RR + 20: case OP_CZ_RR + 24: case OP_CZ_RR + 28: case OP_CZ_RR + 32: case OP_CZ_RR + 36:
        case OP_CZ_RT + 0: case OP_CZ_RT + 2: case OP_CZ_RT + 4: case OP_CZ_RT + 6: case OP_CZ_RT + 8:
        case OP_CZ_TT: rg_cz_code(a, c, op, q0, q1, p0); break;
        case OP_X: c.m ^= 1u << q0; break;
        case OP_OMEGA: rg_omega(a, c, q0, p0, op.aux); break;
        case OP_DIAG1: rg_diag1(a, c, q0, p0, op.c0, op.c1); break;
        case OP_DIAG2: rg_diag2(a, c, q0, q1, M); break;
        case OP_CX: ARSO_CX(0); break;
        ARSO_P4(OP_CX, ARSO_CX)
        case OP_DENSE2:
        case OP_SWAP: {
            const bool swap = (op.pad[0] & 255u) == OP_SWAP;
            const uint32_t mab = ((c.m >> q0) & 1u) | (((c.m >> q1) & 1u) << 1);
            if (c.tid < 16) {
                const uint32_t k = c.tid >> 2, l = c.tid & 3u;
                float2 u;
                if (swap) {
                    const uint32_t perm[4] = {0, 2, 1, 3};
                    u = make_float2(perm[k] == l ? 1.f : 0.f, 0.f);
                } else {
                    u = M[4 * (k ^ mab) + (l ^ mab)];
                }
                ubuf[c.tid] = u;
            }
            __syncthreads();
            to_smem(a, sm, c, t);
            __syncthreads();
            smem_dense2(sm, t, q0, q1, ubuf, c.tid, c.nthr);
            __syncthreads();
            from_smem(a, sm, c, t);
            __syncthreads();
            // SWAP X^m = X^{m with bits q0, q1 exchanged} SWAP
            if (swap && (((c.m >> q0) ^ (c.m >> q1)) & 1u)) c.m ^= (1u << q0) | (1u << q1);
            break;
        }
        default: break;
    }
#undef ARSO_FLIP
#undef ARSO_UA
#undef ARSO_UB
#undef ARSO_SU2
#undef ARSO_D1
#undef ARSO_HADAMARD
#undef ARSO_CX
}
#undef ARSO_P4

// Gates [g, ge) of one phase with the Pauli events that fall inside them;
// ops[0] is the record of gate g0 (the phase's first gate). The inner loop
// runs up to and including the next event's gate without touching the event
// state, which stays out of the hot registers. Records whose tensor role has
// its bit set in `skip` are passed over (tensor phases, which hold no event).
__device__ __forceinline__ void run_gates(Amps &v, TileCtx &c, uint32_t g, uint32_t ge, const RegOp *ops, uint32_t g0,
                                          const float2 *__restrict__ mats, float2 *sm, float2 *ubuf, int t,
                                          const uint32_t *&ev, const uint32_t *ev_end, uint32_t &next,
                                          uint32_t skip = 0u) {
    while (g < ge) {
        const uint32_t np = next == NO_EVENT ? ge : ev_pos(next);
        const uint32_t stop = np < ge ? np + 1 : ge;
        for (; g < stop; ++g) {
            const RegOp &op = ops[g - g0];
            if ((skip >> op.pad[1]) & 1u) continue;
            apply_op(v, c, op, mats, sm, ubuf, t);
        }
        if (np >= ge) break;
        const uint32_t w0 = ops[np - g0].w0;
        while (next != NO_EVENT && ev_pos(next) == np) {
            rg_pauli(v, c, ev_slot(next) ? (w0 >> 24) : ((w0 >> 16) & 255u), ev_code(next));
            ++ev;
            next = ev < ev_end ? *ev : NO_EVENT;
        }
    }
}

// A phase's gate records are staged in shared memory: stage_ops starts
// cp.async copies of the next phase's records (at most MAX_PHASE_OPS, 16 bytes
// per copy) while the current phase runs; stage_wait waits for this thread's
// copies and syncs the CTA, after which the staged records are visible to all
// threads and the other buffer is free again.
__device__ __forceinline__ void stage_ops(RegOp *dst, const RegOp *src, uint32_t n, uint32_t tid, uint32_t nthr) {
    n = n < (uint32_t)MAX_PHASE_OPS ? n : (uint32_t)MAX_PHASE_OPS;
    const char *s = reinterpret_cast<const char *>(src);
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    for (uint32_t i = tid; i < 2 * n; i += nthr)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d + 16 * i), "l"(s + 16 * i) : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void stage_wait() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
}

// ------------------------------------------------------- tensor phases ---
// A phase with a fused unitary U (see the tensor-phase notes of internal.h) as
// one contraction on the tensor cores. The tile is a matrix of 2^(t-5) rows
// (row = thread) by 64 reals (the thread's 32 amplitudes in packed-register
// order: for packed register p, Re a_2p, Re a_2p+1, Im a_2p, Im a_2p+1), and
// D = A B^T with B the real 64 x 64 form of U in the same order on both sides.
// FP32 accuracy from FP16 operands, with no bias from the tensor core's
// accumulation (which is not rounded to nearest): each row is scaled by a power
// of two so that its entries stay below 2^9 and split into the integer
// hi = rint(x) and lo = fp16(x - hi) (|lo| <= 1/2); B comes from the host scaled
// by 2^8 and split the same way (|hi| <= 256). The hi x hi products are integers
// below 2^17 and their sums below 2^23, so their accumulator D0 is exact; the
// other three products (hi lo, lo hi, lo lo) go to a second accumulator D1 about
// 2^-9 of D0's size, whose rounding is negligible; D0 + D1 is formed in
// registers. A (both terms) fills the tile's shared-memory buffer exactly; rows
// are grouped in blocks of 128 (MMAs of M = 128, N = 64), each block with its
// two accumulators in 128 tensor-memory columns.
constexpr uint32_t TP_ROWS = 128;
constexpr uint32_t TP_TERM_BYTES = TP_ROWS * 64 * 2;          // one term of one row block: 16 KiB
constexpr uint32_t TP_IMAGE_BYTES = TENSOR_IMAGE_HALVES * 2;  // B hi and lo: 16 KiB
constexpr uint32_t TP_IDESC = idesc_f16_f32(128, 64);

__device__ __forceinline__ uint32_t h2_bits(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);  // a in the low half (the lower K index)
    return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ float2 h2_value(uint32_t u) {
    const __half2 h = *reinterpret_cast<const __half2 *>(&u);
    return __half22float2(h);
}

// cp.async copies of one phase's B images (16 KiB) into shared memory, in the
// caller's commit group
__device__ __forceinline__ void stage_image(unsigned char *dst, const unsigned char *src, uint32_t tid, uint32_t nthr) {
    const uint32_t d = smem_u32(dst);
    for (uint32_t i = tid; i < TP_IMAGE_BYTES / 16; i += nthr)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d + 16 * i), "l"(src + 16 * i) : "memory");
}

// v <- U v for every row of the tile. Each block of 128 rows (four warps) is an
// independent group: it writes its rows of A, syncs on its own named barrier,
// and its first thread issues the block's MMAs and commits them to the block's
// mbarrier, which the group waits on before reading D back. The caller has
// synced the CTA after its last read of the tile buffer `abuf`; `img` holds
// this phase's staged B images (their cp.async copies waited for and synced).
// Returns false when the wait for the tensor cores gave up (v then holds no
// valid state).
__device__ __forceinline__ bool tensor_apply(Amps &v, unsigned char *abuf, const unsigned char *img, uint32_t nblk,
                                             uint32_t tmem, uint64_t *bars, uint32_t &parity) {
    const uint32_t tid = threadIdx.x, blk = tid >> 7, r = tid & (TP_ROWS - 1u);
    // row scale 2^k: sum of squares in [2^E, 2^(E+1)) bounds every entry below 2^ceil((E+1)/2)
    float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        s2 = fma2(v.re[p], v.re[p], s2);
        s2 = fma2(v.im[p], v.im[p], s2);
    }
    const int E = (int)((__float_as_uint(s2.x + s2.y) >> 23) & 255u) - 127;
    const int k = min(max(9 - ((E + 2) >> 1), -100), 100);
    const float2 sc = bc2(__uint_as_float((uint32_t)(127 + k) << 23));
    const float2 inv = bc2(__uint_as_float((uint32_t)(127 - k - 8) << 23));  // undoes the row and B scales
    {
        unsigned char *row_hi = abuf + blk * TP_TERM_BYTES + (r >> 3) * 1024u + (r & 7u) * 16u;
        unsigned char *row_lo = row_hi + nblk * TP_TERM_BYTES;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int p = 2 * u + (h >> 1);
                const float2 x = mul2(h & 1 ? v.im[p] : v.re[p], sc);
                const float2 rx = make_float2(rintf(x.x), rintf(x.y));
                hi[h] = h2_bits(rx.x, rx.y);
                lo[h] = h2_bits(x.x - rx.x, x.y - rx.y);
            }
            *reinterpret_cast<uint4 *>(row_hi + u * 128) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(row_lo + u * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
    fence_proxy_async_smem();  // A (and the staged B) visible to the tensor core
    tc_fence_before();         // the previous phase's tensor-memory loads precede the next MMA
    asm volatile("bar.sync %0, %1;\n" ::"r"(1u + blk), "r"(TP_ROWS) : "memory");
    if (r == 0) {
        tc_fence_after();
        // descriptors of K step 0; a K step of 16 advances every operand by 256 bytes (16 in
        // the descriptor's address field, which has room: shared addresses stay below 256 KiB)
        const uint32_t ah = smem_u32(abuf) + blk * TP_TERM_BYTES, b0 = smem_u32(img);
        const uint64_t dah = smem_desc_kmajor(ah, 128, 1024), dal = smem_desc_kmajor(ah + nblk * TP_TERM_BYTES, 128, 1024);
        const uint64_t dbh = smem_desc_kmajor(b0, 128, 1024), dbl = smem_desc_kmajor(b0 + TP_IMAGE_BYTES / 2, 128, 1024);
        const uint32_t d0 = tmem + blk * 128, d1 = d0 + 64;
#pragma unroll
        for (uint32_t s = 0; s < 4; ++s) {
            const uint64_t o = 16u * s;
            umma_bf16(d0, dah + o, dbh + o, TP_IDESC, s);
            umma_bf16(d1, dah + o, dbl + o, TP_IDESC, s);
            umma_bf16(d1, dal + o, dbh + o, TP_IDESC, 1);
            umma_bf16(d1, dal + o, dbl + o, TP_IDESC, 1);
        }
        umma_commit(bars + blk);
    }
    bool ok = mbar_wait_bounded(bars + blk, parity);
    if (!ok) (void)mbar_wait_bounded(bars + blk, parity);  // give a slow contraction one more bounded wait
    parity ^= 1u;
    tc_fence_after();
    // this thread's row: tensor-memory lane 32 (warp mod 4) + lane = tid mod 128, block tid / 128
    const uint32_t taddr = tmem + ((((tid >> 5) & 3u) * 32u) << 16) + blk * 128u;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t e[32], f[32];
        tmem_ld32_nowait(taddr + 32 * h, e);
        tmem_ld32_nowait(taddr + 64 + 32 * h, f);
        tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float2 er = make_float2(__uint_as_float(e[4 * i]), __uint_as_float(e[4 * i + 1]));
            const float2 ei = make_float2(__uint_as_float(e[4 * i + 2]), __uint_as_float(e[4 * i + 3]));
            const float2 fr = make_float2(__uint_as_float(f[4 * i]), __uint_as_float(f[4 * i + 1]));
            const float2 fi = make_float2(__uint_as_float(f[4 * i + 2]), __uint_as_float(f[4 * i + 3]));
            v.re[8 * h + i] = mul2(add2(er, fr), inv);
            v.im[8 * h + i] = mul2(add2(ei, fi), inv);
        }
    }
    return ok;
}

// Criterion partial of one thread's 32 amplitudes (true index of register ri:
// (tpart | register part) ^ m, mapped to memory by idx). Fidelity overlaps and
// outcome/binning probabilities are summed over the 32 registers in FP32 and
// then added to the FP64 partial (GB300's FP64 rate is a small fraction of its
// FP32 rate; the block and trajectory sums stay FP64); argmax compares FP64
// probabilities amplitude by amplitude.
template <class Index>
__device__ __forceinline__ void score_registers(Partial &acc, const DCrit &crit, const Amps &v, const TileCtx &c,
                                                const float2 *__restrict__ ref, Index idx) {
    if (crit.kind == ARSO_CRIT_ARGMAX) {
#pragma unroll
        for (int ri = 0; ri < 32; ++ri) accumulate(acc, crit, amp_get(v, ri), ref, idx((c.tpart | reg_part(ri, c.R)) ^ c.m));
        return;
    }
    float fa = 0.f, fb = 0.f;
#pragma unroll
    for (int ri = 0; ri < 32; ++ri) {
        const uint64_t gi = idx((c.tpart | reg_part(ri, c.R)) ^ c.m);
        const float2 x = amp_get(v, ri);
        if (crit.kind == ARSO_CRIT_FIDELITY) {
            const float2 r = ref[gi];
            fa = fmaf(r.x, x.x, fmaf(r.y, x.y, fa));
            fb = fmaf(r.x, x.y, fmaf(-r.y, x.x, fb));
        } else {
            const bool in = crit.kind == ARSO_CRIT_OUTCOME ? gi == crit.target
                                                            : ((crit.bitmap[gi >> 5] >> (gi & 31)) & 1u) != 0;
            if (in) fa = fmaf(x.x, x.x, fmaf(x.y, x.y, fa));
        }
    }
    acc.a += (double)fa;
    acc.b += (double)fb;
}

// global offset of the tile's first amplitude: the tile index deposited into
// the global bits outside the tile
__device__ __forceinline__ uint64_t tile_base(uint64_t rest_mask, uint64_t tile) {
    uint64_t base = 0;
    for (uint64_t mm = rest_mask; mm; mm &= mm - 1) {
        if (tile & 1) base |= mm & (~mm + 1);
        tile >>= 1;
    }
    return base;
}

// The phase loop holds the 64 amplitude registers; everything needed only
// before or after it (addresses, slot data) is recomputed there instead of
// being kept live.
// TENSOR: the launch has tensor phases (a separate instantiation, so that the
// gate-by-gate kernel's code is not shaped by the contraction path). SMALL:
// tiles of at most 2^12 amplitudes (at most 128 threads), compiled for five
// CTAs per SM (96 registers, a few more spills) instead of four: measured 5%
// faster on the 24-qubit benchmark at 12-qubit tiles.
template <bool LAST, bool TENSOR, bool SMALL = false>
__global__ void __launch_bounds__(SMALL ? 128 : 512, SMALL ? 5 : 1) pass_rb_kernel(PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    __shared__ Partial red[32];
    __shared__ float2 ubuf[16];
    __shared__ RegOp s_ops[2][MAX_PHASE_OPS];
    const int t = a.t;
    const uint32_t slot = blockIdx.y;
    const uint64_t N = 1ull << a.n;
    const uint32_t cmask = (1u << a.c) - 1u;
    auto gidx = [&](uint64_t base, uint32_t j) -> uint64_t { return base + a.offs[j >> a.c] + (j & cmask); };

    // load mapping R = {0, t-4, ..., t-1}: register ri = b0 | hi << 1 holds j = hi << (t-4) | tid << 1 | b0
    const uint32_t load_packed = 0u | ((uint32_t)(t - 4) << 5) | ((uint32_t)(t - 3) << 10) |
                                 ((uint32_t)(t - 2) << 15) | ((uint32_t)(t - 1) << 20);
    Amps v;
    const uint32_t *ev = nullptr, *ev_end = nullptr;
    {
        const float2 *src;
        if (a.ideal) {
            src = static_cast<const float2 *>(a.ideal_src);
        } else {
            const int start = a.start_pass[slot];
            if (a.pass < start || a.pass > a.end_pass[slot]) return;
            src = a.pass == start ? static_cast<const float2 *>(a.cache) + (size_t)a.cache_slot[start] * N
                                  : static_cast<const float2 *>(a.work) + (size_t)slot * N;
            // this pass's events: binary search for the first key at or after the pass's first gate
            const uint64_t tr = a.slot_traj[slot];
            const uint32_t *lo = a.keys + a.offsets[tr];
            const uint32_t *hi = a.keys + a.offsets[tr + 1];
            ev_end = hi;
            const uint32_t key_lo = a.gb << 3;
            while (lo < hi) {
                const uint32_t *mid = lo + (hi - lo) / 2;
                if (*mid < key_lo) lo = mid + 1;
                else hi = mid;
            }
            ev = lo;
        }
        const uint64_t base = tile_base(a.rest_mask, blockIdx.x);
#pragma unroll
        for (int hi = 0; hi < 16; ++hi) {
            const uint32_t j = ((uint32_t)hi << (t - 4)) | (threadIdx.x << 1);
            const float4 w = __ldg(reinterpret_cast<const float4 *>(src + gidx(base, j)));
            v.re[hi] = make_float2(w.x, w.z);
            v.im[hi] = make_float2(w.y, w.w);
        }
    }
    TileCtx c;
    c.m = 0;
    c.gp = 0;
    c.tid = threadIdx.x;
    c.nthr = blockDim.x;
    set_phase(c, load_packed, t);

    uint32_t next = ev < ev_end ? *ev : NO_EVENT;
    const float2 *mats = static_cast<const float2 *>(a.mats);
    // tensor phases: tensor memory for D0 and D1 (128 columns per block of 128 rows), one mbarrier
    // for the contractions' completion, and two 16 KiB buffers for the staged B images
    __shared__ uint64_t s_tbar[4];  // one per block of 128 rows
    __shared__ uint32_t s_tmem;
    constexpr bool tensor = TENSOR;
    const uint32_t nblk = blockDim.x / TP_ROWS;
    unsigned char *img = smem_raw + ((size_t)1 << t) * sizeof(float2);
    const unsigned char *tmats = static_cast<const unsigned char *>(a.tmats);
    uint32_t tmem = 0, tpar = 0;
    if (tensor) {
        if (threadIdx.x < 32) tmem_alloc(&s_tmem, nblk * 128u);
        if (threadIdx.x < nblk) {
            mbar_init(&s_tbar[threadIdx.x], 1);
            fence_mbar_init();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        tmem = s_tmem;
    }
    if (a.pb < a.pe) {
        if (tensor && a.ph_t[a.pb] != NO_TENSOR)
            stage_image(img, tmats + (size_t)a.ph_t[a.pb] * TP_IMAGE_BYTES, threadIdx.x, blockDim.x);
        stage_ops(s_ops[0], a.rops + a.ph_gb[a.pb], a.ph_gb[a.pb + 1] - a.ph_gb[a.pb], threadIdx.x, blockDim.x);
    }
    for (uint32_t ph = a.pb; ph < a.pe; ++ph) {
        const uint32_t buf = (ph - a.pb) & 1u;
        stage_wait();
        if (ph + 1 < a.pe) {
            if (tensor && a.ph_t[ph + 1] != NO_TENSOR)
                stage_image(img + (buf ^ 1u) * TP_IMAGE_BYTES, tmats + (size_t)a.ph_t[ph + 1] * TP_IMAGE_BYTES,
                            threadIdx.x, blockDim.x);
            stage_ops(s_ops[buf ^ 1u], a.rops + a.ph_gb[ph + 1], a.ph_gb[ph + 2] - a.ph_gb[ph + 1], threadIdx.x,
                      blockDim.x);
        }
        const uint32_t R = a.ph_R[ph];
        if (R != c.R) remap<true>(v, sm, c, R, t);
        const uint32_t g0 = a.ph_gb[ph], ge = a.ph_gb[ph + 1];
        if constexpr (TENSOR) {
            // the contraction applies U to the true amplitudes: no event of this trajectory in
            // the phase and no mask bit on a register bit (the CTA takes the same branch)
            uint32_t rm = 0;
#pragma unroll
            for (int b = 0; b < REG_BITS; ++b) rm |= 1u << rbit(R, b);
            const bool tp =
                a.ph_t[ph] != NO_TENSOR && (next == NO_EVENT || ev_pos(next) >= ge) && (c.m & rm) == 0u;
            const int rounds = tp ? 2 : 1;
#pragma unroll 1
            for (int rd = 0; rd < rounds; ++rd) {
                if (rd == 1) {
                    __syncthreads();  // every thread's reads of the tile buffer are done
                    if (!tensor_apply(v, smem_raw, img + buf * TP_IMAGE_BYTES, nblk, tmem, s_tbar, tpar))
                        atomicOr(a.terr, 1u);
                }
                const uint32_t skip =
                    tp ? (rd == 0 ? (1u << TR_CORE) | (1u << TR_AFTER) : (1u << TR_CORE) | (1u << TR_BEFORE)) : 0u;
                run_gates(v, c, g0, ge, s_ops[buf], g0, mats, sm, ubuf, t, ev, ev_end, next, skip);
            }
        } else {
            run_gates(v, c, g0, ge, s_ops[buf], g0, mats, sm, ubuf, t, ev, ev_end, next);
        }
    }
    if (tensor) {
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x < 32) {
            tc_fence_after();
            tmem_free(tmem, nblk * 128u);
        }
    }
    apply_global_phase(v, c);  // global phase i^gp
    const uint64_t base = tile_base(a.rest_mask, blockIdx.x);
    if (!a.ideal && !a.store_last && a.pass == a.end_pass[slot]) {
        const float2 *ref = static_cast<const float2 *>(a.ref_cache ? a.ref_cache : a.cache) +
                            (size_t)a.cache_slot[a.pass + 1] * N;
        Partial acc = empty_partial();
        score_registers(acc, a.crit, v, c, ref, [&](uint32_t j) { return gidx(base, j); });
        acc = block_reduce_partial(acc, red);
        if (threadIdx.x == 0) a.partials[(size_t)slot * gridDim.x + blockIdx.x] = acc;
        return;
    }
    if (c.R != load_packed) remap(v, sm, c, load_packed, t);
    float2 *dst = a.ideal ? static_cast<float2 *>(a.ideal_dst) : static_cast<float2 *>(a.work) + (size_t)slot * N;
    const uint32_t flip0 = c.m & 1u;
#pragma unroll
    for (int hi = 0; hi < 16; ++hi) {
        const uint32_t j = (((uint32_t)hi << (t - 4)) | (threadIdx.x << 1)) ^ (c.m & ~1u);
        const float2 r = flip0 ? swp2(v.re[hi]) : v.re[hi], i = flip0 ? swp2(v.im[hi]) : v.im[hi];
        reinterpret_cast<float4 *>(dst + gidx(base, j))[0] = make_float4(r.x, i.x, r.y, i.y);
    }
}

// ------------------------------------------------------------- resident ---
// Whole state (2^n, 10 <= n <= 13) in one CTA: each trajectory restarts from
// the cached error-free state at the checkpoint (phase boundary) at or before
// its first error and runs the remaining phases; ckpt_every counts phases.

__device__ __forceinline__ void rb_load_linear(Amps &v, const float2 *src, int t, uint32_t tid) {
#pragma unroll
    for (int hi = 0; hi < 16; ++hi) {
        const uint32_t j = ((uint32_t)hi << (t - 4)) | (tid << 1);
        const float4 w = __ldg(reinterpret_cast<const float4 *>(src + j));
        v.re[hi] = make_float2(w.x, w.z);
        v.im[hi] = make_float2(w.y, w.w);
    }
}

// store the true state (mask and global phase applied); leaves v in the load mapping
__device__ __forceinline__ void rb_store_linear(Amps &v, float2 *sm, TileCtx &c, uint32_t load_packed, float2 *dst,
                                                int t) {
    if (c.R != load_packed) remap(v, sm, c, load_packed, t);
    apply_global_phase(v, c);
    const uint32_t flip0 = c.m & 1u;
#pragma unroll
    for (int hi = 0; hi < 16; ++hi) {
        const uint32_t j = (((uint32_t)hi << (t - 4)) | (c.tid << 1)) ^ (c.m & ~1u);
        const float2 r = flip0 ? swp2(v.re[hi]) : v.re[hi], i = flip0 ? swp2(v.im[hi]) : v.im[hi];
        reinterpret_cast<float4 *>(dst + j)[0] = make_float4(r.x, i.x, r.y, i.y);
    }
}

template <int MODE>
__global__ void __launch_bounds__(512, 1) resident_rb_kernel(ResidentArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    __shared__ Partial red[32];
    __shared__ float2 ubuf[16];
    __shared__ RegOp s_ops[2][MAX_PHASE_OPS];
    const int t = a.n;
    const uint32_t N = 1u << t;
    const float2 *cache = static_cast<const float2 *>(a.cache);
    const float2 *mats = static_cast<const float2 *>(a.mats);
    const uint32_t load_packed = 0u | ((uint32_t)(t - 4) << 5) | ((uint32_t)(t - 3) << 10) |
                                 ((uint32_t)(t - 2) << 15) | ((uint32_t)(t - 1) << 20);
    const uint64_t count = MODE == 2 ? 1 : a.count;
    for (uint64_t b = blockIdx.x; b < count; b += gridDim.x) {
        Amps v;
        TileCtx c;
        c.m = 0;
        c.gp = 0;
        c.tid = threadIdx.x;
        c.nthr = blockDim.x;
        set_phase(c, load_packed, t);
        uint32_t ph0 = 0;
        const uint32_t *ev = nullptr, *ev_end = nullptr;
        uint64_t tr = 0;
        if (MODE == 2) {
#pragma unroll
            for (int k = 0; k < 16; ++k) v.re[k] = v.im[k] = make_float2(0.f, 0.f);
            if (threadIdx.x == 0) v.re[0].x = 1.f;
        } else {
            tr = a.ids ? a.ids[b] : a.first_traj + b;
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
        if (ph0 < a.n_phases)
            stage_ops(s_ops[0], a.rops + a.ph_gb[ph0], a.ph_gb[ph0 + 1] - a.ph_gb[ph0], threadIdx.x, blockDim.x);
        for (uint32_t ph = ph0; ph < a.n_phases; ++ph) {
            const uint32_t buf = (ph - ph0) & 1u;
            stage_wait();
            if (ph + 1 < a.n_phases)
                stage_ops(s_ops[buf ^ 1u], a.rops + a.ph_gb[ph + 1], a.ph_gb[ph + 2] - a.ph_gb[ph + 1], threadIdx.x,
                          blockDim.x);
            if (MODE == 2 && ph % (uint32_t)a.ckpt_every == 0) {
                float2 *dst = const_cast<float2 *>(cache) + (size_t)(ph / (uint32_t)a.ckpt_every) * N;
                rb_store_linear(v, sm, c, load_packed, dst, t);
            }
            const uint32_t R = a.ph_R[ph];
            if (R != c.R) remap<MODE != 2>(v, sm, c, R, t);
            const uint32_t g0 = a.ph_gb[ph];
            run_gates(v, c, g0, a.ph_gb[ph + 1], s_ops[buf], g0, mats, sm, ubuf, t, ev, ev_end, next);
        }
        if (MODE == 2) {
            rb_store_linear(v, sm, c, load_packed, const_cast<float2 *>(cache) + (size_t)(a.n_ckpt - 1) * N,
                            t);
        } else if (MODE == 1) {
            rb_store_linear(v, sm, c, load_packed, static_cast<float2 *>(a.states_out) + (size_t)b * N, t);
        } else {
            apply_global_phase(v, c);
            const float2 *ref = cache + (size_t)(a.n_ckpt - 1) * N;
            Partial acc = empty_partial();
            score_registers(acc, a.crit, v, c, ref, [](uint32_t j) { return (uint64_t)j; });
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

// One batched resident item (see above) run by the whole CTA.
__device__ __forceinline__ void batch_item(const BatchItem &it, const BatchCircuit &C, const uint64_t *__restrict__ ids,
                                           unsigned char *smem_raw, Partial *red, float2 (*ubuf)[16],
                                           RegOp (*s_ops)[MAX_PHASE_OPS]) {
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
    Amps v;
    rb_load_linear(v, C.cache + (size_t)it.ck * N, t, c.tid);
    const uint32_t *ev = C.keys + C.offsets[tr];
    const uint32_t *ev_end = C.keys + C.offsets[tr + 1];
    uint32_t next = ev < ev_end ? *ev : NO_EVENT;
    const uint32_t ph0 = it.ck * C.ckpt_every;
    if (ph0 < C.n_phases)
        stage_ops(s_ops[0], C.rops + C.ph_gb[ph0], C.ph_gb[ph0 + 1] - C.ph_gb[ph0], threadIdx.x, BATCH_THREADS);
    for (uint32_t ph = ph0; ph < C.n_phases; ++ph) {
        const uint32_t buf = (ph - ph0) & 1u;
        stage_wait();
        if (ph + 1 < C.n_phases)
            stage_ops(s_ops[buf ^ 1u], C.rops + C.ph_gb[ph + 1], C.ph_gb[ph + 2] - C.ph_gb[ph + 1], threadIdx.x,
                      BATCH_THREADS);
        const uint32_t R = C.ph_R[ph];
        if (R != c.R) remap<true>(v, sm, c, R, t);
        const uint32_t g0 = C.ph_gb[ph];
        run_gates(v, c, g0, C.ph_gb[ph + 1], s_ops[buf], g0, C.mats, sm, ubuf[sg], t, ev, ev_end, next);
    }
    apply_global_phase(v, c);
    const float2 *ref = C.cache + (size_t)(C.n_ckpt - 1) * N;
    Partial acc = empty_partial();
    score_registers(acc, C.crit, v, c, ref, [](uint32_t j) { return (uint64_t)j; });
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

__global__ void __launch_bounds__(BATCH_THREADS, 2)
    batch_resident_kernel(const BatchCircuit *__restrict__ circs, const BatchItem *__restrict__ items, uint32_t n_items,
                          uint32_t *counter, const uint64_t *__restrict__ ids) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_item;
    __shared__ Partial red[BATCH_THREADS / 32];
    __shared__ float2 ubuf[8][16];
    __shared__ RegOp s_ops[2][MAX_PHASE_OPS];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_items) return;
        const BatchItem it = items[item];
        batch_item(it, circs[it.circuit], ids, smem_raw, red, ubuf, s_ops);
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

// ------------------------------------------------- persistent mixed batch ---
// One launch over every unit of a batch of uneven circuits (MixArgs in kernels.h).
// A CTA of 256 threads takes sub-items from one counter in list order. Streaming
// sub-items wait (thread 0, bounded polls) for their slot's counter of finished
// tiles; since a unit's dependencies always sit earlier in the list, the lowest
// sub-item in progress never waits on a later one and the launch cannot deadlock.
// A wait that gives up sets the error word; every CTA then stops at its next item.
constexpr int MIX_THREADS = BATCH_THREADS;  // one 2^13-amplitude tile: 256 threads x 32 registers

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// thread 0: wait until *ctr >= need + extra (extra is 0 except in the failure-path test);
// false if the wait gave up or another CTA's did
__device__ bool mix_wait(const uint32_t *ctr, uint32_t need, uint32_t extra, uint32_t limit, uint32_t *err) {
    const uint64_t target = (uint64_t)need + extra;
    for (uint32_t it = 0;; ++it) {
        if ((uint64_t)ld_acquire_u32(ctr) >= target) return true;
        if (it >= limit || ld_acquire_u32(err) != 0u) {
            atomicOr(err, 1u);
            return false;
        }
        __nanosleep(256);
    }
}

__device__ __forceinline__ Partial ld_partial_cg(const Partial *p) {
    Partial v;
    v.a = __ldcg(&p->a);
    v.b = __ldcg(&p->b);
    v.maxp = __ldcg(&p->maxp);
    v.idx = __ldcg(&p->idx);
    return v;
}

// First unit u >= lo with unit_end[u] > i (warp 0; unit_end ascending, unit_end[lo - 1] <= i
// by the caller's previous item): 32-way search, each round one load per lane.
__device__ uint32_t mix_find_unit(const uint64_t *__restrict__ unit_end, uint32_t n_units, uint32_t lo, uint64_t i) {
    if (__ldg(unit_end + lo) > i) return lo;
    uint32_t hi = n_units - 1;  // unit_end[hi] = total > i; invariant unit_end[lo] <= i < unit_end[hi]
    const uint32_t lane = threadIdx.x & 31u;
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t probe = min(lo + step * (lane + 1), hi);
        const unsigned m = __ballot_sync(0xffffffffu, __ldg(unit_end + probe) > i);
        const uint32_t f = (uint32_t)(__ffs(m) - 1);  // lane 31 probes hi, so m != 0
        const uint32_t nhi = min(lo + step * (f + 1), hi);
        lo = f == 0 ? lo : lo + step * f;
        hi = nhi;
    }
    return hi;
}

// MIX_REF: chunk `chunk` of psi_R scored; the last chunk adds the chunk partials in
// order and gives that score to every error-free trajectory of the circuit.
__device__ __noinline__ void mix_ref(const MixRef &R, uint32_t chunk, Partial *red, uint32_t *s_flag, double *s_val) {
    const uint32_t N = 1u << R.n, j0 = chunk << 13, j1 = min(N, j0 + 8192u);
    Partial acc = empty_partial();
    for (uint32_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) accumulate(acc, R.crit, R.psi_R[j], R.psi_R, j);
    acc = block_reduce_partial(acc, red);
    if (threadIdx.x == 0) {
        R.partials[chunk] = acc;
        __threadfence();
        *s_flag = atomicAdd(R.done, 1u) == R.chunks - 1;
    }
    __syncthreads();
    if (!*s_flag) return;
    __threadfence();
    if (threadIdx.x == 0) {
        Partial sum = empty_partial();
        for (uint32_t k = 0; k < R.chunks; ++k) {
            const Partial q = ld_partial_cg(R.partials + k);
            sum.a += q.a;
            sum.b += q.b;
            argmax_merge(sum.maxp, sum.idx, q.maxp, q.idx);
        }
        *s_val = finish_score(R.crit, sum);
    }
    __syncthreads();
    const double sc = *s_val;
    for (uint64_t t = threadIdx.x; t < R.n_traj; t += blockDim.x)
        if (R.first[t] == NO_EVENT) {
            R.score[t] = sc;
            if (R.pass_flags) R.pass_flags[t] = sc >= R.crit.threshold;
        }
}

// MIX_SMALL: up to 32 trajectories of one circuit of n <= 9 qubits side by side in
// shared memory as one state of n + log2(count) qubits (gates touch only the low n
// bits, so one update covers every trajectory); each trajectory's Pauli errors are
// applied to its own block; 8 threads score each trajectory.
__device__ __noinline__ void mix_small(const MixSmall &C, const BatchItem &it, const uint64_t *__restrict__ ids, float2 *s) {
    __shared__ const uint32_t *s_ev[MIX_SMALL_MAX];
    __shared__ const uint32_t *s_end[MIX_SMALL_MAX];
    __shared__ uint32_t s_pe[MIX_SMALL_MAX];
    const int n = C.n;
    const uint32_t N = 1u << n, cnt = it.count;
    int tb = n;
    while ((1u << (tb - n)) < cnt) ++tb;  // n + ceil(log2 cnt) <= 13
    const float2 *src = C.cache + (size_t)it.ck * N;
    for (uint32_t i = threadIdx.x; i < (1u << tb); i += blockDim.x)
        s[i] = (i >> n) < cnt ? src[i & (N - 1)] : make_float2(0.f, 0.f);
    if (threadIdx.x < cnt) {
        const uint64_t tr = ids[it.off + threadIdx.x];
        s_ev[threadIdx.x] = C.keys + C.offsets[tr];
        s_end[threadIdx.x] = C.keys + C.offsets[tr + 1];
    }
    __syncthreads();
    const uint32_t g0 = min(C.G, it.ck * C.ckpt_every);
    for (uint32_t g = g0; g < C.G; ++g) {
        const DGate gate = C.gates[g];
        if (gate.cls != GC_NOP) tile_gate(s, tb, gate, C.mats + gate.mat);
        // this gate's error events of each trajectory: up to two, (valid | qubit << 2 | code) per half
        bool any = false;
        if (threadIdx.x < cnt) {
            const uint32_t *e = s_ev[threadIdx.x], *ee = s_end[threadIdx.x];
            uint32_t pe = 0, sh = 0;
            while (e < ee && ev_pos(*e) == g) {
                const uint32_t q = ev_slot(*e) ? gate.q1 : gate.q0;
                pe |= (0x8000u | (q << 2) | ev_code(*e)) << sh;
                sh = 16;
                ++e;
            }
            s_ev[threadIdx.x] = e;
            s_pe[threadIdx.x] = pe;
            any = pe != 0;
        }
        if (__syncthreads_or(any)) {
            for (int w = 0; w < 2; ++w) {
                for (uint32_t p = threadIdx.x; p < (cnt << (n - 1)); p += blockDim.x) {
                    const uint32_t k = p >> (n - 1), e = (s_pe[k] >> (16 * w)) & 0xFFFFu;
                    if (!(e & 0x8000u)) continue;
                    const uint32_t q = (e >> 2) & 63u, code = e & 3u, bit = 1u << q;
                    const uint32_t i0 = (k << n) | insert_zero(p & ((N >> 1) - 1), q), i1 = i0 | bit;
                    const float2 a0 = s[i0], a1 = s[i1];
                    if (code == 1) {
                        s[i0] = a1;
                        s[i1] = a0;
                    } else if (code == 2) {
                        s[i1] = cneg(a1);
                    } else {  // Y: (a0, a1) -> (-i a1, i a0), Eq. (2)
                        s[i0] = make_float2(a1.y, -a1.x);
                        s[i1] = make_float2(-a0.y, a0.x);
                    }
                }
                __syncthreads();
            }
        }
    }
    // score: 8 threads per trajectory, FP64 sums, shuffles within each group of 8
    const uint32_t k = threadIdx.x >> 3, r = threadIdx.x & 7u;
    const float2 *ref = C.cache + (size_t)(C.n_ckpt - 1) * N;
    Partial acc = empty_partial();
    if (k < cnt)
        for (uint32_t j = r; j < N; j += 8) accumulate(acc, C.crit, s[(k << n) + j], ref, j);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        const double a2 = __shfl_down_sync(0xffffffffu, acc.a, o, 8);
        const double b2 = __shfl_down_sync(0xffffffffu, acc.b, o, 8);
        const double mp = __shfl_down_sync(0xffffffffu, acc.maxp, o, 8);
        const unsigned long long mi = __shfl_down_sync(0xffffffffu, acc.idx, o, 8);
        acc.a += a2;
        acc.b += b2;
        argmax_merge(acc.maxp, acc.idx, mp, mi);
    }
    if (r == 0 && k < cnt) {
        const uint64_t tr = ids[it.off + k];
        const double sc = finish_score(C.crit, acc);
        C.score[tr] = sc;
        if (C.pass_flags) C.pass_flags[tr] = sc >= C.crit.threshold;
    }
}

__device__ __noinline__ void mix_res(const BatchItem &it, const BatchCircuit &C, const uint64_t *__restrict__ ids,
                                    unsigned char *smem_raw, Partial *red, float2 (*ubuf)[16],
                                    RegOp (*s_ops)[MAX_PHASE_OPS]) {
    batch_item(it, C, ids, smem_raw, red, ubuf, s_ops);
}

// MIX_STR: one tile of pass j of trajectory k of stream S (the body of pass_rb_kernel
// with explicit coordinates), after the slot's dependencies. The item's coordinates live
// in shared memory (`it`) and the stream's descriptor too: read where needed rather than
// held in registers, since the phase loop already uses all 128 (kept in registers they
// spilled into the loop).
struct MixTile {
    uint32_t k, j, tile;
};

__device__ __forceinline__ uint64_t mix_gidx(const MixStream &S, uint32_t j, uint64_t base, uint32_t jj) {
    return base + S.passes[j].offs[jj >> S.c] + (jj & ((1u << S.c) - 1u));
}

__device__ __forceinline__ void mix_tile(const MixArgs &A, const MixStream &S, const MixTile &it,
                                         unsigned char *smem_raw, Partial *red, float2 *ubuf,
                                         RegOp (*s_ops)[MAX_PHASE_OPS], uint32_t *s_flag) {
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    if (threadIdx.x == 0) {
        const MixTraj &T = S.trajs[it.k];
        *s_flag = mix_wait(S.slot_done + T.slot, T.base + (uint32_t)((int)it.j - T.start) * S.tiles,
                           A.stall_extra, A.wait_limit, A.err);
    }
    __syncthreads();  // thread 0's acquire load, then the barrier, order the tile loads after it
    if (!*s_flag) return;
    const int t = S.t;
    Amps v;
    const uint32_t *ev, *ev_end;
    {
        const uint32_t k = it.k, j = it.j;
        const MixTraj &T = S.trajs[k];
        const uint64_t N = 1ull << S.n;
        const bool from_cache = (int)j == T.start;
        const float2 *src = from_cache ? S.cache + (size_t)S.cache_slot[j] * N : S.work + (size_t)T.slot * N;
        const uint64_t base = tile_base(S.passes[j].rest_mask, it.tile);
#pragma unroll
        for (int hi = 0; hi < 16; ++hi) {
            const uint32_t jj = ((uint32_t)hi << (t - 4)) | (threadIdx.x << 1);
            const float4 *pa = reinterpret_cast<const float4 *>(src + mix_gidx(S, j, base, jj));
            // the working slot was written by other CTAs of this launch: read it through L2
            const float4 w = from_cache ? __ldg(pa) : __ldcg(pa);
            v.re[hi] = make_float2(w.x, w.z);
            v.im[hi] = make_float2(w.y, w.w);
        }
        // this pass's events: binary search for the first key at or after the pass's first gate
        const uint32_t *lo = S.keys + S.offsets[T.tr], *hi_ = S.keys + S.offsets[T.tr + 1];
        ev_end = hi_;
        const uint32_t key_lo = S.passes[j].gb << 3;
        while (lo < hi_) {
            const uint32_t *mid = lo + (hi_ - lo) / 2;
            if (*mid < key_lo) lo = mid + 1;
            else hi_ = mid;
        }
        ev = lo;
    }
    TileCtx c;
    c.m = 0;
    c.gp = 0;
    c.tid = threadIdx.x;
    c.nthr = blockDim.x;
    set_phase(c, 0u | ((uint32_t)(t - 4) << 5) | ((uint32_t)(t - 3) << 10) | ((uint32_t)(t - 2) << 15) |
                     ((uint32_t)(t - 1) << 20),
              t);
    uint32_t next = ev < ev_end ? *ev : NO_EVENT;
    {
        const uint32_t pb = S.passes[it.j].pb;
        if (pb < S.passes[it.j].pe)
            stage_ops(s_ops[0], S.rops + S.ph_gb[pb], S.ph_gb[pb + 1] - S.ph_gb[pb], threadIdx.x, blockDim.x);
    }
    for (uint32_t ph = S.passes[it.j].pb, buf = 0; ph < S.passes[it.j].pe; ++ph, buf ^= 1u) {
        stage_wait();
        if (ph + 1 < S.passes[it.j].pe)
            stage_ops(s_ops[buf ^ 1u], S.rops + S.ph_gb[ph + 1], S.ph_gb[ph + 2] - S.ph_gb[ph + 1], threadIdx.x,
                      blockDim.x);
        const uint32_t R = S.ph_R[ph];
        if (R != c.R) remap<true>(v, sm, c, R, t);
        const uint32_t g0 = S.ph_gb[ph];
        run_gates(v, c, g0, S.ph_gb[ph + 1], s_ops[buf], g0, S.mats, sm, ubuf, t, ev, ev_end, next);
    }
    apply_global_phase(v, c);
    const uint32_t k = it.k, j = it.j;
    const MixTraj &T = S.trajs[k];
    const uint64_t N = 1ull << S.n;
    const uint64_t base = tile_base(S.passes[j].rest_mask, it.tile);
    const bool scored = (int)j == T.end;
    if (scored) {
        const float2 *ref = S.ref_cache + (size_t)S.cache_slot[j + 1] * N;
        Partial acc = empty_partial();
        score_registers(acc, S.crit, v, c, ref, [&](uint32_t jj) { return mix_gidx(S, j, base, jj); });
        acc = block_reduce_partial(acc, red);
        if (threadIdx.x == 0) S.partials[(size_t)k * S.tiles + it.tile] = acc;
    } else {
        const uint32_t load_packed = 0u | ((uint32_t)(t - 4) << 5) | ((uint32_t)(t - 3) << 10) |
                                     ((uint32_t)(t - 2) << 15) | ((uint32_t)(t - 1) << 20);
        if (c.R != load_packed) remap(v, sm, c, load_packed, t);
        float2 *dst = S.work + (size_t)T.slot * N;
        const uint32_t flip0 = c.m & 1u;
#pragma unroll
        for (int hi = 0; hi < 16; ++hi) {
            const uint32_t jj = (((uint32_t)hi << (t - 4)) | (threadIdx.x << 1)) ^ (c.m & ~1u);
            const float2 r = flip0 ? swp2(v.re[hi]) : v.re[hi], i = flip0 ? swp2(v.im[hi]) : v.im[hi];
            reinterpret_cast<float4 *>(dst + mix_gidx(S, j, base, jj))[0] = make_float4(r.x, i.x, r.y, i.y);
        }
    }
    // publish: the barrier orders every thread's stores before thread 0's fence and
    // counter increments (the release the waiting CTAs acquire)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(S.slot_done + T.slot, 1u);
        *s_flag = scored && atomicAdd(S.traj_done + k, 1u) == S.tiles - 1 ? 2u : 1u;
    }
    __syncthreads();
    if (*s_flag != 2u) return;
    // last tile of the scored pass: the trajectory's partials added in the order of
    // finish_partials_kernel, so the score equals the one of the per-pass launches
    __threadfence();
    Partial acc = empty_partial();
    for (uint32_t i = threadIdx.x; i < S.tiles; i += blockDim.x) {
        const Partial q = ld_partial_cg(S.partials + (size_t)k * S.tiles + i);
        acc.a += q.a;
        acc.b += q.b;
        argmax_merge(acc.maxp, acc.idx, q.maxp, q.idx);
    }
    acc = block_reduce_partial(acc, red);
    if (threadIdx.x == 0) {
        const double sc = finish_score(S.crit, acc);
        S.score[T.tr] = sc;
        if (S.pass_flags) S.pass_flags[T.tr] = sc >= S.crit.threshold;
    }
}

__global__ void __launch_bounds__(MIX_THREADS, 2) mix_kernel(const __grid_constant__ MixArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long s_i;
    __shared__ uint32_t s_u, s_flag;
    __shared__ double s_val;
    __shared__ Partial red[MIX_THREADS / 32];
    __shared__ float2 ubuf[8][16];
    __shared__ RegOp s_ops[2][MAX_PHASE_OPS];
    // the current streaming circuit's descriptor: read from shared memory in the phase loop
    // instead of being held in registers (the loop already uses all 128)
    __shared__ MixStream s_stream;
    __shared__ uint32_t s_stream_idx;
    __shared__ MixTile s_tile;
    if (threadIdx.x == 0) s_u = 0, s_stream_idx = ~0u;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_i = ld_acquire_u32(a.err) ? a.n_sub : atomicAdd(a.counter, 1ull);
        __syncthreads();
        const unsigned long long i = s_i;
        if (i >= a.n_sub) return;
        if (threadIdx.x < 32) {
            const uint32_t u = mix_find_unit(a.unit_end, a.n_units, s_u, i);
            if (threadIdx.x == 0) s_u = u;
        }
        __syncthreads();
        const uint32_t u = s_u;
        const MixUnit un = a.units[u];
        const uint32_t sub = (uint32_t)(i - (u ? a.unit_end[u - 1] : 0ull));
        if (un.kind == MIX_REF) {
            mix_ref(a.refs[un.idx], sub, red, &s_flag, &s_val);
        } else if (un.kind == MIX_SMALL) {
            const BatchItem it = a.items[un.idx];
            mix_small(a.smalls[it.circuit], it, a.ids, reinterpret_cast<float2 *>(smem_raw));
        } else if (un.kind == MIX_RES) {
            const BatchItem it = a.items[un.idx];
            mix_res(it, a.rcircs[it.circuit], a.ids, smem_raw, red, ubuf, s_ops);
        } else {
            if (threadIdx.x == 0) {
                if (s_stream_idx != un.idx) {
                    s_stream = a.streams[un.idx];
                    s_stream_idx = un.idx;
                }
                s_tile = MixTile{un.a, un.b, sub};
            }
            __syncthreads();
            mix_tile(a, s_stream, s_tile, smem_raw, red, ubuf[0], s_ops, &s_flag);
        }
    }
}

void launch_mix(const MixArgs &a, double bytes, double flops, double smem_bytes, cudaStream_t st) {
    if (!a.n_sub) return;
    ProfScope ps_(ARSO_K_MIX, bytes, st, flops, smem_bytes);
    const size_t smem = (size_t(1) << 13) * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        ARSO_CUDA(cudaFuncSetAttribute(mix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    int per_sm = 1, dev = 0, sms = 152;
    ARSO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mix_kernel, MIX_THREADS, smem));
    ARSO_CUDA(cudaGetDevice(&dev));
    ARSO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)std::min<uint64_t>(a.n_sub, (uint64_t)std::max(per_sm, 1) * sms);
    mix_kernel<<<grid, MIX_THREADS, smem, st>>>(a);
    ARSO_CUDA(cudaGetLastError());
}

// Raise the dynamic shared-memory limit of both pass variants once, before any
// launch (and outside stream capture).
void prepare_pass_rb() {
    static bool done = false;
    if (done) return;
    const int smem = (1 << MAX_TILE_QUBITS) * (int)sizeof(float2) + 2 * (int)TP_IMAGE_BYTES;
    ARSO_CUDA(cudaFuncSetAttribute(pass_rb_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ARSO_CUDA(cudaFuncSetAttribute(pass_rb_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ARSO_CUDA(cudaFuncSetAttribute(pass_rb_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ARSO_CUDA(cudaFuncSetAttribute(pass_rb_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ARSO_CUDA(cudaFuncSetAttribute(pass_rb_kernel<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ARSO_CUDA(cudaFuncSetAttribute(pass_rb_kernel<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    done = true;
}

void launch_pass_rb(const PassArgs &a, bool last, uint32_t slots, double bytes, cudaStream_t st, double flops,
                    double smem_bytes) {
    ProfScope ps_(last && !a.store_last ? ARSO_K_PASS_LAST : ARSO_K_PASS, bytes, st, flops, smem_bytes);
    prepare_pass_rb();
    const uint32_t tiles = 1u << (a.n - a.t);
    const int nt = 1 << (a.t - REG_BITS);
    const size_t smem = (size_t(1) << a.t) * sizeof(float2) + (a.ph_t ? 2 * TP_IMAGE_BYTES : 0);
    if (a.ph_t) ARSO_REQUIRE(a.t >= 12 && a.t <= MAX_TILE_QUBITS, "tensor phases need 12-14-qubit tiles");
    dim3 grid(tiles, slots);
    if (a.ph_t) {
        if (last) pass_rb_kernel<true, true><<<grid, nt, smem, st>>>(a);
        else pass_rb_kernel<false, true><<<grid, nt, smem, st>>>(a);
    } else if (nt <= 128) {
        if (last) pass_rb_kernel<true, false, true><<<grid, nt, smem, st>>>(a);
        else pass_rb_kernel<false, false, true><<<grid, nt, smem, st>>>(a);
    } else {
        if (last) pass_rb_kernel<true, false><<<grid, nt, smem, st>>>(a);
        else pass_rb_kernel<false, false><<<grid, nt, smem, st>>>(a);
    }
    ARSO_CUDA(cudaGetLastError());
}

}  // namespace arso
