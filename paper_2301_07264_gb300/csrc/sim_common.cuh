// Device helpers shared by the simulation kernels: complex arithmetic, gate
// and Pauli application on a shared-memory tile, block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "kernels.h"

namespace arso {

template <typename R> struct CT;
template <> struct CT<float> {
    using T = float2;
};
template <> struct CT<double> {
    using T = double2;
};

template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
    T r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a*x + b*y
template <typename T> __device__ __forceinline__ T cmac2(T a, T x, T b, T y) {
    T r;
    r.x = a.x * x.x - a.y * x.y + b.x * y.x - b.y * y.y;
    r.y = a.x * x.y + a.y * x.x + b.x * y.y + b.y * y.x;
    return r;
}
template <typename T> __device__ __forceinline__ T cneg(T a) {
    a.x = -a.x;
    a.y = -a.y;
    return a;
}

// x / sqrt(2): FP32 uses the two-float constant (fma(hi, x, lo * x)), so the
// product carries only the unbiased rounding of the operations.
__device__ __forceinline__ float mul_rsqrt2(float x) { return fmaf(RSQRT2_HI, x, RSQRT2_LO * x); }
__device__ __forceinline__ double mul_rsqrt2(double x) { return x * RSQRT2_D; }

// v * e^{i k pi / 4}
template <typename T> __device__ __forceinline__ T omega_mul(T v, uint32_t k) {
    T r = v;
    if (k & 1u) {  // e^{i pi/4} (x + iy) = (x - y)/sqrt2 + i (x + y)/sqrt2
        r.x = mul_rsqrt2(v.x - v.y);
        r.y = mul_rsqrt2(v.x + v.y);
    }
    const uint32_t q = (k >> 1) & 3u;  // remaining factor i^q
    T o = r;
    if (q == 1) { o.x = -r.y; o.y = r.x; }
    else if (q == 2) { o.x = -r.x; o.y = -r.y; }
    else if (q == 3) { o.x = r.y; o.y = -r.x; }
    return o;
}

__device__ __forceinline__ uint32_t insert_zero(uint32_t p, uint32_t b) {
    const uint32_t lo = (1u << b) - 1u;
    return ((p & ~lo) << 1) | (p & lo);
}
// insert zeros at bit positions lo < hi (positions in the result)
__device__ __forceinline__ uint32_t insert_zero2(uint32_t p, uint32_t lo, uint32_t hi) {
    return insert_zero(insert_zero(p, lo), hi);
}

// Apply gate g to a tile of 2^t amplitudes in shared memory. All threads of
// the block take part; the caller synchronises afterwards.
template <typename T>
__device__ __forceinline__ void tile_gate(T *s, int t, const DGate &g, const T *__restrict__ M) {
    const uint32_t nt = blockDim.x, tid = threadIdx.x;
    switch (g.cls) {
        case GC_DENSE1:
        case GC_SU2: {
            const T u00 = M[0], u01 = M[1], u10 = M[2], u11 = M[3];
            const uint32_t b = g.q0, bit = 1u << b;
            for (uint32_t p = tid; p < (1u << (t - 1)); p += nt) {
                const uint32_t i0 = insert_zero(p, b), i1 = i0 | bit;
                const T a0 = s[i0], a1 = s[i1];
                s[i0] = cmac2(u00, a0, u01, a1);
                s[i1] = cmac2(u10, a0, u11, a1);
            }
            break;
        }
        case GC_DIAG1: {
            const T d0 = M[0], d1 = M[1];
            const uint32_t b = g.q0, bit = 1u << b;
            for (uint32_t p = tid; p < (1u << (t - 1)); p += nt) {
                const uint32_t i0 = insert_zero(p, b), i1 = i0 | bit;
                s[i0] = cmul(d0, s[i0]);
                s[i1] = cmul(d1, s[i1]);
            }
            break;
        }
        case GC_H: {
            const uint32_t b = g.q0, bit = 1u << b;
            for (uint32_t p = tid; p < (1u << (t - 1)); p += nt) {
                const uint32_t i0 = insert_zero(p, b), i1 = i0 | bit;
                const T a0 = s[i0], a1 = s[i1];
                T r0, r1;
                r0.x = mul_rsqrt2(a0.x + a1.x);
                r0.y = mul_rsqrt2(a0.y + a1.y);
                r1.x = mul_rsqrt2(a0.x - a1.x);
                r1.y = mul_rsqrt2(a0.y - a1.y);
                s[i0] = r0;
                s[i1] = r1;
            }
            break;
        }
        case GC_OMEGA: {
            const uint32_t b = g.q0, bit = 1u << b, k = g.mat;
            for (uint32_t p = tid; p < (1u << (t - 1)); p += nt) {
                const uint32_t i1 = insert_zero(p, b) | bit;
                s[i1] = omega_mul(s[i1], k);
            }
            break;
        }
        case GC_X: {
            const uint32_t b = g.q0, bit = 1u << b;
            for (uint32_t p = tid; p < (1u << (t - 1)); p += nt) {
                const uint32_t i0 = insert_zero(p, b), i1 = i0 | bit;
                const T a0 = s[i0];
                s[i0] = s[i1];
                s[i1] = a0;
            }
            break;
        }
        case GC_CZ: {
            const uint32_t lo = g.q0 < g.q1 ? g.q0 : g.q1, hi = g.q0 < g.q1 ? g.q1 : g.q0;
            const uint32_t both = (1u << g.q0) | (1u << g.q1);
            for (uint32_t p = tid; p < (1u << (t - 2)); p += nt) {
                const uint32_t i = insert_zero2(p, lo, hi) | both;
                s[i] = cneg(s[i]);
            }
            break;
        }
        case GC_DENSE2:
        case GC_DIAG2:
        case GC_CX:
        case GC_SWAP: {
            const uint32_t b0 = g.q0, b1 = g.q1;
            const uint32_t lo = b0 < b1 ? b0 : b1, hi = b0 < b1 ? b1 : b0;
            const uint32_t m0 = 1u << b0, m1 = 1u << b1;
            for (uint32_t p = tid; p < (1u << (t - 2)); p += nt) {
                const uint32_t i = insert_zero2(p, lo, hi);
                const uint32_t idx[4] = {i, i | m0, i | m1, i | m0 | m1};
                if (g.cls == GC_DENSE2) {
                    T a[4], r[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) a[k] = s[idx[k]];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        T acc = cmac2(M[4 * k + 0], a[0], M[4 * k + 1], a[1]);
                        const T acc2 = cmac2(M[4 * k + 2], a[2], M[4 * k + 3], a[3]);
                        acc.x += acc2.x;
                        acc.y += acc2.y;
                        r[k] = acc;
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) s[idx[k]] = r[k];
                } else if (g.cls == GC_DIAG2) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) s[idx[k]] = cmul(M[k], s[idx[k]]);
                } else if (g.cls == GC_CX) {
                    const T a = s[idx[1]];
                    s[idx[1]] = s[idx[3]];
                    s[idx[3]] = a;
                } else {
                    const T a = s[idx[1]];
                    s[idx[1]] = s[idx[2]];
                    s[idx[2]] = a;
                }
            }
            break;
        }
        default: break;  // GC_NOP
    }
}

// Pauli error gate on tile-local bit b, as Eq. (2): X (a0,a1)->(a1,a0);
// Z (a0,a1)->(a0,-a1); Y (a0,a1)->(-i a1, i a0). code 1 = X, 2 = Z, 3 = Y.
template <typename T> __device__ __forceinline__ void tile_pauli(T *s, int t, uint32_t b, uint32_t code) {
    const uint32_t nt = blockDim.x, bit = 1u << b;
    for (uint32_t p = threadIdx.x; p < (1u << (t - 1)); p += nt) {
        const uint32_t i0 = insert_zero(p, b), i1 = i0 | bit;
        const T a0 = s[i0], a1 = s[i1];
        T r0, r1;
        if (code == 1) {
            r0 = a1;
            r1 = a0;
        } else if (code == 2) {
            r0 = a0;
            r1 = cneg(a1);
        } else {
            r0.x = a1.y;   // -i * a1
            r0.y = -a1.x;
            r1.x = -a0.y;  // i * a0
            r1.y = a0.x;
        }
        s[i0] = r0;
        s[i1] = r1;
    }
}

__device__ __forceinline__ void argmax_merge(double &mp, unsigned long long &mi, double op, unsigned long long oi) {
    if (op > mp || (op == mp && oi < mi)) {
        mp = op;
        mi = oi;
    }
}

// Block-wide reduction of one Partial per thread; result valid in thread 0.
// Uses `red` (shared, >= 32 Partials). Deterministic for a fixed block size.
__device__ __forceinline__ Partial block_reduce_partial(Partial v, Partial *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double a = __shfl_down_sync(0xffffffffu, v.a, o);
        const double b = __shfl_down_sync(0xffffffffu, v.b, o);
        const double mp = __shfl_down_sync(0xffffffffu, v.maxp, o);
        const unsigned long long mi = __shfl_down_sync(0xffffffffu, v.idx, o);
        v.a += a;
        v.b += b;
        argmax_merge(v.maxp, v.idx, mp, mi);
    }
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        Partial w = lane < nw ? red[lane] : Partial{0.0, 0.0, -1.0, ~0ull};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double a = __shfl_down_sync(0xffffffffu, w.a, o);
            const double b = __shfl_down_sync(0xffffffffu, w.b, o);
            const double mp = __shfl_down_sync(0xffffffffu, w.maxp, o);
            const unsigned long long mi = __shfl_down_sync(0xffffffffu, w.idx, o);
            w.a += a;
            w.b += b;
            argmax_merge(w.maxp, w.idx, mp, mi);
        }
        v = w;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ void accumulate(Partial &acc, const DCrit &c, T v, const T *__restrict__ ref,
                                           unsigned long long gi) {
    if (c.kind == ARSO_CRIT_FIDELITY) {
        const T r = ref[gi];
        acc.a += (double)r.x * (double)v.x + (double)r.y * (double)v.y;
        acc.b += (double)r.x * (double)v.y - (double)r.y * (double)v.x;
    } else {
        const double p = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        if (c.kind == ARSO_CRIT_OUTCOME) {
            if (gi == c.target) acc.a += p;
        } else if (c.kind == ARSO_CRIT_BINNING) {
            if ((c.bitmap[gi >> 5] >> (gi & 31)) & 1u) acc.a += p;
        } else {
            argmax_merge(acc.maxp, acc.idx, p, gi);
        }
    }
}

__device__ __forceinline__ double finish_score(const DCrit &c, const Partial &p) {
    if (c.kind == ARSO_CRIT_FIDELITY) return p.a * p.a + p.b * p.b;
    if (c.kind == ARSO_CRIT_ARGMAX) return p.idx == c.target ? 1.0 : 0.0;
    return p.a;
}

__device__ __forceinline__ Partial empty_partial() { return Partial{0.0, 0.0, -1.0, ~0ull}; }

}  // namespace arso
