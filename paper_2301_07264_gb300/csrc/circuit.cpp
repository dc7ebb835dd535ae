// Circuit compiler: gate matrices, error-location table, fused pass schedule.
//
// A circuit (Sec. II) is a list of one- and two-qubit gates. Every gate gets
// one error location per qubit (Sec. IV-B.2: a two-qubit gate draws an error
// on each of its qubits), so L = k + 2m (Eq. (3)).
//
// Engines:
//  * resident  - the whole 2^n state lives in one CTA's shared memory for the
//                entire circuit (n <= 13 for complex64, 12 for complex128);
//  * streaming - the state lives in HBM and is swept by fused passes. A pass
//                is a set of t "tile qubits" (always including the low qubits
//                0..c-1 so that global accesses stay contiguous) and a list of
//                gates acting only on tile qubits; each CTA loads one tile of
//                2^t amplitudes into shared memory, applies all of the pass's
//                gates (and the trajectory's error gates that follow them),
//                and writes the tile back: one HBM round trip per pass.
//
// The pass builder chooses each pass's tile qubits, then places gates in
// circuit order: a gate joins the pass when its qubits are tile qubits and none
// is blocked; otherwise its qubits become blocked for the rest of the pass, and
// so does every later gate that touches a blocked qubit. The set of gates
// placed in a pass is therefore closed under the circuit's dependencies, and
// concatenating the passes gives an engine order that is a valid topological
// reordering of the circuit. Error gates stay attached to the gate they
// follow, which keeps them correct: a gate moved ahead of gate g never touches
// g's qubits after g. The tile set starts from the low qubits and the qubits of
// the first unplaced gate and grows one qubit at a time, each time by the qubit
// whose addition places the most gates (lowest index on ties); when no single
// qubit adds a gate, it takes the qubits of the earliest gate still left out.
#include <algorithm>
#include <set>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace arso {

using cd = std::complex<double>;

void matrix_for(const arso_gate &g, HostGate &h) {
    const double s2 = 1.0 / std::sqrt(2.0);
    const double th = g.param;
    const cd I(0, 1);
    for (auto &v : h.m) v = 0;
    auto set2 = [&](cd a, cd b, cd c, cd d) { h.m[0] = a; h.m[1] = b; h.m[2] = c; h.m[3] = d; };
    switch (g.kind) {
        case ARSO_GATE_ID: set2(1, 0, 0, 1); h.cls = GC_NOP; break;
        case ARSO_GATE_H: set2(s2, s2, s2, -s2); h.cls = GC_H; break;
        case ARSO_GATE_X: set2(0, 1, 1, 0); h.cls = GC_X; break;
        case ARSO_GATE_Y: set2(0, -I, I, 0); h.cls = GC_DENSE1; break;
        // diag(1, e^{i k pi/4}): Z (k=4), S (2), SDG (6), T (1), TDG (7)
        case ARSO_GATE_Z: set2(1, 0, 0, -1); h.cls = GC_OMEGA; h.omega_k = 4; break;
        case ARSO_GATE_S: set2(1, 0, 0, I); h.cls = GC_OMEGA; h.omega_k = 2; break;
        case ARSO_GATE_SDG: set2(1, 0, 0, -I); h.cls = GC_OMEGA; h.omega_k = 6; break;
        case ARSO_GATE_T: set2(1, 0, 0, std::polar(1.0, M_PI / 4)); h.cls = GC_OMEGA; h.omega_k = 1; break;
        case ARSO_GATE_TDG: set2(1, 0, 0, std::polar(1.0, -M_PI / 4)); h.cls = GC_OMEGA; h.omega_k = 7; break;
        case ARSO_GATE_RX:
            set2(std::cos(th / 2), -I * std::sin(th / 2), -I * std::sin(th / 2), std::cos(th / 2));
            h.cls = GC_DENSE1;
            break;
        case ARSO_GATE_RY:
            set2(std::cos(th / 2), -std::sin(th / 2), std::sin(th / 2), std::cos(th / 2));
            h.cls = GC_DENSE1;
            break;
        case ARSO_GATE_RZ: set2(std::polar(1.0, -th / 2), 0, 0, std::polar(1.0, th / 2)); h.cls = GC_DIAG1; break;
        case ARSO_GATE_P: set2(1, 0, 0, std::polar(1.0, th)); h.cls = GC_DIAG1; break;
        case ARSO_GATE_U:
            ARSO_REQUIRE(g.matrix != nullptr, "U gate needs a 2x2 matrix");
            for (int i = 0; i < 4; ++i) h.m[i] = cd(g.matrix[2 * i], g.matrix[2 * i + 1]);
            h.cls = GC_DENSE1;
            break;
        case ARSO_GATE_CX:
            for (int i = 0; i < 4; ++i) h.m[5 * i] = 1;
            h.m[5] = 0; h.m[15] = 0; h.m[1 * 4 + 3] = 1; h.m[3 * 4 + 1] = 1;
            h.cls = GC_CX;
            break;
        case ARSO_GATE_CZ:
            h.m[0] = 1; h.m[5] = 1; h.m[10] = 1; h.m[15] = -1; h.cls = GC_CZ; break;
        case ARSO_GATE_CP:
            h.m[0] = 1; h.m[5] = 1; h.m[10] = 1; h.m[15] = std::polar(1.0, th); h.cls = GC_DIAG2; break;
        case ARSO_GATE_SWAP:
            h.m[0] = 1; h.m[15] = 1; h.m[1 * 4 + 2] = 1; h.m[2 * 4 + 1] = 1; h.cls = GC_SWAP; break;
        case ARSO_GATE_U2:
            ARSO_REQUIRE(g.matrix != nullptr, "U2 gate needs a 4x4 matrix");
            for (int i = 0; i < 16; ++i) h.m[i] = cd(g.matrix[2 * i], g.matrix[2 * i + 1]);
            h.cls = GC_DENSE2;
            break;
        default: throw Error(ARSO_EINVAL, "unknown gate kind " + std::to_string(g.kind));
    }
    for (int i = 0; i < (h.arity == 1 ? 4 : 16); ++i)
        ARSO_REQUIRE(std::isfinite(h.m[i].real()) && std::isfinite(h.m[i].imag()), "non-finite gate matrix entry");
}

// gates [first, G) that a pass with tile set in_s would place (circuit order,
// blocked-qubit rule); returns their number and, when `out` is given, their indices
static size_t pass_closure(const arso_circuit *c, const std::vector<char> &done, size_t first,
                           const std::vector<char> &in_s, std::vector<uint32_t> *out) {
    const uint32_t n = c->n;
    std::vector<char> blocked(n, 0);
    uint32_t n_blocked = 0;
    size_t cnt = 0;
    for (size_t g = first; g < c->gates.size() && n_blocked < n; ++g) {
        if (done[g]) continue;
        const HostGate &h = c->gates[g];
        const uint32_t qs[2] = {h.q0, h.q1};
        bool ok = true;
        for (int j = 0; j < h.arity; ++j) ok &= !blocked[qs[j]] && in_s[qs[j]];
        if (ok) {
            ++cnt;
            if (out) out->push_back((uint32_t)g);
        } else {
            for (int j = 0; j < h.arity; ++j)
                if (!blocked[qs[j]]) blocked[qs[j]] = 1, ++n_blocked;
        }
    }
    return cnt;
}

static void schedule_streaming(arso_circuit *c) {
    const uint32_t n = c->n, t = c->tile_qubits, lowq = c->low_qubits;
    const size_t G = c->gates.size();
    std::vector<char> done(G, 0);
    size_t remaining = G, first = 0;
    c->passes.clear();
    c->perm.clear();
    do {
        std::vector<char> in_s(n, 0);
        uint32_t cnt = 0;
        auto add = [&](uint32_t q) {
            if (!in_s[q]) in_s[q] = 1, ++cnt;
        };
        for (uint32_t q = 0; q < lowq; ++q) add(q);
        if (first < G) {
            add(c->gates[first].q0);
            add(c->gates[first].q1);
        }
        size_t placed = pass_closure(c, done, first, in_s, nullptr);
        while (cnt < t) {
            size_t best = placed;
            uint32_t bq = n;
            for (uint32_t q = 0; q < n; ++q) {
                if (in_s[q]) continue;
                in_s[q] = 1;
                const size_t k = pass_closure(c, done, first, in_s, nullptr);
                in_s[q] = 0;
                if (k > best) best = k, bq = q;
            }
            if (bq < n) {
                add(bq);
                placed = best;
                continue;
            }
            // no single qubit places another gate: the earliest gate left out that fits
            std::vector<uint32_t> in_pass;
            pass_closure(c, done, first, in_s, &in_pass);
            std::vector<char> placed_g(G, 0);
            for (uint32_t g : in_pass) placed_g[g] = 1;
            bool grown = false;
            for (size_t g = first; g < G && !grown; ++g) {
                if (done[g] || placed_g[g]) continue;
                const HostGate &h = c->gates[g];
                const uint32_t fresh = (in_s[h.q0] ? 0u : 1u) + (h.arity == 2 && !in_s[h.q1] ? 1u : 0u);
                if (fresh && cnt + fresh <= t) {
                    add(h.q0);
                    add(h.q1);
                    grown = true;
                }
            }
            if (!grown) break;
            placed = pass_closure(c, done, first, in_s, nullptr);
        }
        // pad the tile to exactly t qubits (lowest unused qubits first)
        for (uint32_t q = 0; q < n && cnt < t; ++q) add(q);
        Pass p;
        p.gb = (uint32_t)c->perm.size();
        std::vector<uint32_t> in_pass;
        pass_closure(c, done, first, in_s, &in_pass);
        ARSO_REQUIRE(!in_pass.empty() || G == 0, "internal: the pass builder placed no gate");
        for (uint32_t g : in_pass) {
            done[g] = 1;
            --remaining;
            c->perm.push_back(g);
        }
        while (first < G && done[first]) ++first;
        for (uint32_t q = 0; q < n; ++q)
            if (in_s[q]) p.tile_qubits.push_back(q);
        p.ge = (uint32_t)c->perm.size();
        c->passes.push_back(std::move(p));
    } while (remaining > 0);
}

// Register-bit phases of each pass. A gate that mixes amplitudes needs its
// mixing qubit among the REG_BITS register bits (dense one-qubit gates and H:
// their qubit; CX: its target); diagonal gates, X, and the dense two-qubit
// gates and SWAP (run through shared memory) act on any bit. Tile bit 0 is a
// register bit in every phase (the register kernels pack amplitudes j and
// j|1 into one FP32x2 register pair).
//
// Within a pass the gates may run in any order that respects their qubit
// dependencies. The planner list-schedules them: with register set R it runs
// every ready gate whose need is in R, repeatedly; when none is left it picks
// the next R among all sets of tile bit 0 and four other tile bits by the
// weighted number of gates the closure under R would run. Passes start and
// end in the load/store mapping {0, t-4, t-3, t-2, t-1}, whose thread bits
// 1..t-5 keep global accesses contiguous.
static constexpr uint32_t NO_NEED = 0xFFFFFFFFu;

static uint32_t need_of(const HostGate &h, uint32_t lq0, uint32_t lq1) {
    switch (h.cls) {
        case GC_DENSE1: case GC_H: return lq0;
        case GC_CX: return lq1;
        default: return NO_NEED;
    }
}

// relative cost of a gate in the register kernels (the planner's objective)
static double gate_weight(const HostGate &h) {
    switch (h.cls) {
        case GC_DENSE1: case GC_H: return 1.0;
        case GC_DENSE2: case GC_SWAP: return 2.0;
        case GC_DIAG1: case GC_OMEGA: return 0.5;
        default: return 0.25;
    }
}

namespace {
// Dependency DAG of one pass and a list scheduler with trial closures.
struct PassScheduler {
    uint32_t G;
    std::vector<uint32_t> need;
    std::vector<double> weight;
    std::vector<std::vector<uint32_t>> succ;
    std::vector<uint32_t> indeg;
    std::set<uint32_t> ready;  // unscheduled gates whose predecessors are all scheduled
    std::vector<uint32_t> order;
    // Tensor-phase rules: a gate runs under R when all its qubits are in R (a
    // diagonal one always, another one while none of its qubits is frozen) or
    // when it is diagonal. A diagonal gate with qubits in and out of R freezes
    // its qubits in R that a non-diagonal gate of the phase already acted on.
    bool tensor = false;
    std::vector<uint8_t> diag;    // diagonal in the computational basis
    std::vector<uint32_t> qmask;  // tile-local qubits of the gate

    static bool in(const std::vector<uint32_t> &R, uint32_t q) {
        return q == NO_NEED || std::find(R.begin(), R.end(), q) != R.end();
    }
    bool runs(uint32_t g, const std::vector<uint32_t> &R, uint32_t Rm, uint32_t frozen) const {
        if (!tensor) return in(R, need[g]);
        if ((qmask[g] & ~Rm) == 0) return diag[g] || !(qmask[g] & frozen);
        return diag[g] != 0;
    }
    // Run every ready gate that runs under R, repeatedly. With `trial` the
    // state is restored afterwards and only the weight is returned.
    double closure(const std::vector<uint32_t> &R, bool trial) {
        std::vector<std::pair<uint32_t, uint32_t>> undo;  // (gate, old indeg)
        std::set<uint32_t> rd = ready;
        double w = 0.0;
        uint32_t Rm = 0, started = 0, frozen = 0;
        for (uint32_t q : R) Rm |= 1u << q;
        bool progress = true;
        while (progress) {
            progress = false;
            for (auto it = rd.begin(); it != rd.end();) {
                const uint32_t g = *it;
                if (!runs(g, R, Rm, frozen)) {
                    ++it;
                    continue;
                }
                it = rd.erase(it);
                w += weight[g];
                if (tensor) {
                    if ((qmask[g] & ~Rm) == 0) started |= diag[g] ? 0u : qmask[g];
                    else frozen |= qmask[g] & Rm & started;
                }
                if (!trial) order.push_back(g);
                for (uint32_t s : succ[g]) {
                    if (trial) undo.emplace_back(s, indeg[s]);
                    if (--indeg[s] == 0) rd.insert(s);
                }
                progress = true;
                it = rd.begin();  // lowest index first
            }
        }
        if (trial) {
            for (auto u = undo.rbegin(); u != undo.rend(); ++u) indeg[u->first] = u->second;
        } else {
            ready.swap(rd);
        }
        return w;
    }
};
}  // namespace

// algorithmic FP32 flops per amplitude of one gate (see the tracing section of arso.h)
static double gate_flops(const HostGate &h) {
    switch (h.cls) {
        case GC_DENSE1: return 14.0;
        case GC_DENSE2: return 30.0;
        case GC_DIAG1: case GC_DIAG2: return 6.0;
        case GC_H: return 4.0;
        case GC_OMEGA: return (h.omega_k & 1u) ? 2.0 : 0.0;
        default: return 0.0;
    }
}

static bool is_diagonal(const HostGate &h) {
    switch (h.cls) {
        case GC_NOP: case GC_DIAG1: case GC_DIAG2: case GC_OMEGA: case GC_CZ: return true;
        default: return false;
    }
}

// U <- G U for gate h on register positions p0 (and p1) of the 32-dimensional
// register index (two-qubit matrices index bit(q0) + 2 bit(q1), row-major)
static void left_apply(std::vector<std::complex<double>> &U, const HostGate &h, uint32_t p0, uint32_t p1) {
    const uint32_t b0 = 1u << p0, b1 = 1u << p1;
    for (uint32_t col = 0; col < 32; ++col) {
        auto at = [&](uint32_t row) -> std::complex<double> & { return U[row * 32 + col]; };
        for (uint32_t l = 0; l < 32; ++l) {
            if (h.arity == 1) {
                if (l & b0) continue;
                const std::complex<double> x0 = at(l), x1 = at(l | b0);
                at(l) = h.m[0] * x0 + h.m[1] * x1;
                at(l | b0) = h.m[2] * x0 + h.m[3] * x1;
            } else {
                if (l & (b0 | b1)) continue;
                const uint32_t ix[4] = {l, l | b0, l | b1, l | b0 | b1};
                std::complex<double> x[4], y[4];
                for (int k = 0; k < 4; ++k) x[k] = at(ix[k]);
                for (int r = 0; r < 4; ++r) {
                    y[r] = 0;
                    for (int k = 0; k < 4; ++k) y[r] += h.m[4 * r + k] * x[k];
                }
                for (int k = 0; k < 4; ++k) at(ix[k]) = y[k];
            }
        }
    }
}

// Nearest binary16 value of x (ties to even; |x| < 65504), as bits; *v gets its value.
static uint16_t f16_bits(double x, double *v) {
    const double ax = std::fabs(x);
    const uint16_t sign = std::signbit(x) ? 0x8000u : 0u;
    if (ax == 0.0) {
        *v = 0.0;
        return sign;
    }
    int e;
    std::frexp(ax, &e);                      // ax in [2^(e-1), 2^e)
    const int E = std::max(e - 1, -14);      // below 2^-14 the spacing stays 2^-24 (subnormals)
    const double q = std::ldexp(1.0, E - 10);
    const double r = std::nearbyint(ax / q) * q;  // round to nearest, ties to even
    *v = sign ? -r : r;
    if (r < std::ldexp(1.0, -14)) return (uint16_t)(sign | (uint16_t)std::ldexp(r, 24));
    int er;
    const double fr = std::frexp(r, &er);    // r = fr 2^er, fr in [0.5, 1)
    const uint32_t mant = (uint32_t)std::ldexp(fr, 11) - 1024u;
    return (uint16_t)(sign | (uint16_t)((er - 1 + 15) << 10) | (uint16_t)mant);
}

// Roles of the records of phase ph (positions [gb, ge), tile-local qubits lq0/lq1
// indexed from pass_gb) and, when the phase qualifies, its operand images: the
// real 64 x 64 form of U in packed-register order on both sides (index 4p + 2c +
// lane for register 2p + lane, c = 0 real part, 1 imaginary part), B[n][k] with
// D[row][n] = sum_k A[row][k] B[n][k], scaled by 2^8 and split into the integer
// hi = rint(2^8 B) (|hi| <= 256, exact in fp16) and lo = fp16(2^8 B - hi).
static void tensor_phase(arso_circuit *c, uint32_t ph, uint32_t gb, uint32_t ge, uint32_t pass_gb,
                         const std::vector<uint32_t> &lq0, const std::vector<uint32_t> &lq1) {
    uint32_t R[REG_BITS], Rm = 0;
    int rp[32];
    std::fill(rp, rp + 32, -1);
    for (int b = 0; b < REG_BITS; ++b) {
        R[b] = (c->ph_R[ph] >> (5 * b)) & 31u;
        Rm |= 1u << R[b];
        rp[R[b]] = b;
    }
    std::vector<std::complex<double>> U(32 * 32, 0.0);
    for (int i = 0; i < 32; ++i) U[i * 33] = 1.0;
    uint32_t started = 0, frozen = 0;
    int dense = 0;
    bool ok = true;
    for (uint32_t pos = gb; pos < ge; ++pos) {
        const HostGate &h = c->gates[c->perm[pos]];
        const uint32_t a = lq0[pos - pass_gb], b = lq1[pos - pass_gb];
        const uint32_t qm = (1u << a) | (1u << b);
        const bool dg = is_diagonal(h);
        if ((qm & ~Rm) == 0) {
            c->role[pos] = TR_CORE;
            if (!dg) {
                ok &= (qm & frozen) == 0;
                started |= qm;
                ++dense;
            }
            left_apply(U, h, (uint32_t)rp[a], (uint32_t)rp[b]);
        } else {
            ok &= dg;
            const bool after = (qm & Rm & started) != 0;
            c->role[pos] = after ? TR_AFTER : TR_BEFORE;
            frozen |= qm & Rm & started;
        }
    }
    if (!ok || dense < TENSOR_MIN_DENSE) return;
    c->ph_t[ph] = (uint32_t)(c->tmats.size() / TENSOR_IMAGE_HALVES);
    const size_t base = c->tmats.size();
    c->tmats.resize(base + TENSOR_IMAGE_HALVES);
    uint16_t *hi = c->tmats.data() + base, *lo = hi + TENSOR_IMAGE_HALVES / 2;
    for (uint32_t n = 0; n < 64; ++n)
        for (uint32_t k = 0; k < 64; ++k) {
            const uint32_t j = 2 * (n >> 2) + (n & 1u), l = 2 * (k >> 2) + (k & 1u);
            const uint32_t co = (n >> 1) & 1u, ci = (k >> 1) & 1u;
            const std::complex<double> u = U[j * 32 + l];
            const double val = co == 0 ? (ci == 0 ? u.real() : -u.imag()) : (ci == 0 ? u.imag() : u.real());
            double vh, vl;
            const uint32_t off = ((n >> 3) * 1024 + (k >> 3) * 128 + (n & 7u) * 16 + (k & 7u) * 2) / 2;
            const double x = std::ldexp(val, 8), xi = std::nearbyint(x);
            hi[off] = f16_bits(xi, &vh);
            lo[off] = f16_bits(x - xi, &vl);
        }
}

static void plan_phases(arso_circuit *c) {
    const uint32_t t = c->tile_qubits;
    c->reg_blocked = c->precision == ARSO_C64 && t >= (uint32_t)RB_MIN_TILE;
    c->ph_gb.clear();
    c->ph_R.clear();
    c->rpos.assign(c->perm.size(), 0xFF);
    c->tensor = c->reg_blocked && c->engine == 1 && t >= 12 && (c->flags & ARSO_OPT_TENSOR_PHASES);
    c->ph_t.clear();
    c->tmats.clear();
    c->role.assign(c->perm.size(), (uint8_t)TR_CORE);
    if (!c->reg_blocked) return;
    const std::vector<uint32_t> load_map = {0, t - 4, t - 3, t - 2, t - 1};
    for (Pass &ps : c->passes) {
        std::vector<int> local(c->n, -1);
        for (size_t i = 0; i < ps.tile_qubits.size(); ++i) local[ps.tile_qubits[i]] = (int)i;
        const uint32_t G = ps.ge - ps.gb;
        PassScheduler S;
        S.G = G;
        S.tensor = c->tensor;
        S.diag.resize(G);
        S.qmask.resize(G);
        S.need.resize(G);
        S.weight.resize(G);
        S.succ.assign(G, {});
        S.indeg.assign(G, 0);
        std::vector<int> last(t, -1);
        for (uint32_t i = 0; i < G; ++i) {
            const HostGate &h = c->gates[c->perm[ps.gb + i]];
            const uint32_t a = (uint32_t)local[h.q0], b = (uint32_t)local[h.q1];
            S.need[i] = need_of(h, a, b);
            S.weight[i] = gate_weight(h);
            S.diag[i] = is_diagonal(h) ? 1 : 0;
            S.qmask[i] = (1u << a) | (1u << b);
            const int pa = last[a], pb = h.arity == 2 ? last[b] : -1;
            if (pa >= 0) S.succ[pa].push_back(i), ++S.indeg[i];
            if (pb >= 0 && pb != pa) S.succ[pb].push_back(i), ++S.indeg[i];
            last[a] = (int)i;
            if (h.arity == 2) last[b] = (int)i;
        }
        for (uint32_t i = 0; i < G; ++i)
            if (!S.indeg[i]) S.ready.insert(i);
        ps.pb = (uint32_t)c->ph_R.size();
        std::vector<uint32_t> cur = load_map;
        std::vector<std::pair<uint32_t, std::vector<uint32_t>>> phases;  // (start in order, R)
        for (;;) {
            const size_t before = S.order.size();
            S.closure(cur, false);
            if (S.order.size() > before) phases.emplace_back((uint32_t)before, cur);
            if (S.order.size() == G) break;
            // next register set: tile bit 0 and the 4 other tile bits whose closure runs
            // the largest weight of gates (all C(t-1, 4) sets are tried; ties keep the first)
            std::vector<uint32_t> R{0, 1, 2, 3, 4}, best;
            double best_w = -1.0;
            for (uint32_t a = 1; a < t; ++a)
                for (uint32_t b = a + 1; b < t; ++b)
                    for (uint32_t d = b + 1; d < t; ++d)
                        for (uint32_t e = d + 1; e < t; ++e) {
                            R[1] = a, R[2] = b, R[3] = d, R[4] = e;
                            const double w = S.closure(R, true);
                            if (w > best_w + 1e-12) best_w = w, best = R;
                        }
            R = best;
            std::sort(R.begin(), R.end());
            // tensor rules: a new phase under the same set starts with nothing frozen
            ARSO_REQUIRE(best_w > 0.0 && (R != cur || S.tensor), "internal: the phase planner made no progress");
            cur = R;
        }
        if (phases.empty()) phases.emplace_back(0u, load_map);
        // the pass's new engine order
        std::vector<uint32_t> perm_new(G);
        for (uint32_t k = 0; k < G; ++k) perm_new[k] = c->perm[ps.gb + S.order[k]];
        std::copy(perm_new.begin(), perm_new.end(), c->perm.begin() + ps.gb);
        std::vector<uint32_t> lq0(G), lq1(G);
        for (uint32_t i = 0; i < G; ++i) {
            const HostGate &h = c->gates[c->perm[ps.gb + i]];
            lq0[i] = (uint32_t)local[h.q0];
            lq1[i] = (uint32_t)local[h.q1];
        }
        // phases longer than MAX_PHASE_OPS gates continue with the same register set
        for (size_t k = 0; k < phases.size(); ++k) {
            ARSO_REQUIRE(phases[k].second[0] == 0, "internal: a register set without tile bit 0");
            const uint32_t end = k + 1 < phases.size() ? phases[k + 1].first : G;
            for (uint32_t b = phases[k].first; b < end || b == phases[k].first; b += MAX_PHASE_OPS) {
                c->ph_gb.push_back(ps.gb + b);
                c->ph_R.push_back(pack_rbits(phases[k].second.data()));
            }
        }
        ps.pe = (uint32_t)c->ph_R.size();
        // register positions of each gate's qubits within its phase
        for (uint32_t ph = ps.pb; ph < ps.pe; ++ph) {
            uint32_t R[REG_BITS];
            for (int b = 0; b < REG_BITS; ++b) R[b] = (c->ph_R[ph] >> (5 * b)) & 31u;
            const uint32_t ge = ph + 1 < ps.pe ? c->ph_gb[ph + 1] : ps.ge;
            for (uint32_t pos = c->ph_gb[ph]; pos < ge; ++pos) {
                uint32_t p0 = 15, p1 = 15;
                for (int b = 0; b < REG_BITS; ++b) {
                    if (R[b] == lq0[pos - ps.gb]) p0 = (uint32_t)b;
                    if (R[b] == lq1[pos - ps.gb]) p1 = (uint32_t)b;
                }
                c->rpos[pos] = (uint8_t)(p0 | (p1 << 4));
            }
        }
        if (c->tensor) {
            c->ph_t.resize(ps.pe, NO_TENSOR);
            for (uint32_t ph = ps.pb; ph < ps.pe; ++ph)
                tensor_phase(c, ph, c->ph_gb[ph], ph + 1 < ps.pe ? c->ph_gb[ph + 1] : ps.ge, ps.gb, lq0, lq1);
        }
    }
    for (Pass &ps : c->passes) {
        ps.flops_per_amp = 0.0;
        for (uint32_t pos = ps.gb; pos < ps.ge; ++pos) ps.flops_per_amp += gate_flops(c->gates[c->perm[pos]]);
        // shared-memory transposes of one sweep: every change of register set, from the load layout
        const uint32_t load_packed = pack_rbits(load_map.data());
        uint32_t prev = load_packed;
        ps.remaps = 0;
        for (uint32_t ph = ps.pb; ph < ps.pe; ++ph) {
            ps.remaps += c->ph_R[ph] != prev;
            prev = c->ph_R[ph];
        }
        ps.end_remap = prev != load_packed;
    }
    c->chg_prefix.assign(c->ph_R.size() + 1, 0);
    for (size_t ph = 0; ph < c->ph_R.size(); ++ph)
        c->chg_prefix[ph + 1] = c->chg_prefix[ph] + (ph > 0 && c->ph_R[ph] != c->ph_R[ph - 1]);
    c->ph_gb.push_back(c->passes.empty() ? 0 : c->passes.back().ge);  // sentinel
    c->phase_of_pos.assign(c->perm.size(), 0);
    for (size_t ph = 0; ph + 1 < c->ph_gb.size(); ++ph)
        for (uint32_t pos = c->ph_gb[ph]; pos < c->ph_gb[ph + 1]; ++pos) c->phase_of_pos[pos] = (uint32_t)ph;
}

void build_circuit(arso_circuit *c, uint32_t n, const arso_gate *gates, size_t n_gates,
                   const arso_compile_opts *opts) {
    ARSO_REQUIRE(n >= 1 && n <= 30, "n_qubits must be in [1, 30]");
    ARSO_REQUIRE(n_gates == 0 || gates != nullptr, "gates is NULL");
    ARSO_REQUIRE(n_gates < (1u << 28), "too many gates");
    c->n = n;
    c->precision = opts ? (int)opts->precision : ARSO_C64;
    ARSO_REQUIRE(c->precision == ARSO_C64 || c->precision == ARSO_C128, "bad precision");
    c->gates.resize(n_gates);
    c->k = c->m = 0;
    for (size_t i = 0; i < n_gates; ++i) {
        const arso_gate &g = gates[i];
        HostGate &h = c->gates[i];
        h.kind = g.kind;
        h.arity = g.kind >= ARSO_GATE_CX ? 2 : 1;
        h.q0 = g.q[0];
        h.q1 = h.arity == 2 ? g.q[1] : g.q[0];
        ARSO_REQUIRE(h.q0 < n && h.q1 < n, "gate " + std::to_string(i) + ": qubit out of range");
        ARSO_REQUIRE(h.arity == 1 || h.q0 != h.q1, "gate " + std::to_string(i) + ": repeated qubit");
        matrix_for(g, h);
        if (h.arity == 1) ++c->k; else ++c->m;
    }
    c->L = c->k + 2 * c->m;
    ARSO_REQUIRE(c->L < (1ull << 29), "too many error locations");
    c->loc_gate.clear();
    c->loc_gate.reserve(c->L);
    for (size_t i = 0; i < n_gates; ++i)
        for (int j = 0; j < c->gates[i].arity; ++j) c->loc_gate.push_back((uint32_t)i);

    const int rmax = c->precision == ARSO_C128 ? RESIDENT_MAX_N_C128 : RESIDENT_MAX_N_C64;
    c->engine = (int)n <= rmax ? 0 : 1;
    uint32_t tq = opts && opts->tile_qubits ? opts->tile_qubits : (c->precision == ARSO_C128 ? 12u : 13u);
    uint32_t lq = opts && opts->low_qubits ? opts->low_qubits : 4u;
    c->max_batch = opts ? opts->max_batch : 0;
    c->flags = opts ? opts->flags : 0;
    c->cache_budget = opts && opts->cache_bytes ? opts->cache_bytes : (uint64_t)16 << 30;
    if (c->engine == 0) {
        c->tile_qubits = n;
        c->low_qubits = n;
        c->perm.resize(n_gates);
        for (size_t i = 0; i < n_gates; ++i) c->perm[i] = (uint32_t)i;
        Pass p;
        p.gb = 0;
        p.ge = (uint32_t)n_gates;
        for (uint32_t q = 0; q < n; ++q) p.tile_qubits.push_back(q);
        c->passes.assign(1, p);
    } else {
        const uint32_t tmax = c->precision == ARSO_C128 ? 13u : (uint32_t)MAX_TILE_QUBITS;
        ARSO_REQUIRE(tq >= 6 && tq <= tmax, "tile_qubits out of range");
        tq = std::min(tq, n);
        lq = std::min(std::max(lq, 1u), tq);
        c->tile_qubits = tq;
        c->low_qubits = lq;
        schedule_streaming(c);
    }
    plan_phases(c);  // may reorder gates within a pass
    c->flops_prefix.assign(n_gates + 1, 0.0);
    for (size_t pos = 0; pos < n_gates; ++pos) c->flops_prefix[pos + 1] = c->flops_prefix[pos] + gate_flops(c->gates[c->perm[pos]]);
    c->pos_of.assign(n_gates, 0);
    for (size_t pos = 0; pos < c->perm.size(); ++pos) c->pos_of[c->perm[pos]] = (uint32_t)pos;
    c->pass_of_pos.assign(n_gates, 0);
    for (size_t p = 0; p < c->passes.size(); ++p)
        for (uint32_t pos = c->passes[p].gb; pos < c->passes[p].ge; ++pos) c->pass_of_pos[pos] = (uint32_t)p;
}

}  // namespace arso

namespace arso {

// 32 surrogate features: n, G, L, k, m, depth, two-qubit layers, log10 L,
// log10 G, two-qubit fraction, counts per gate kind (18), criterion one-hot (4).
std::vector<float> circuit_features(const arso_circuit *c, const arso_criterion *crit) {
    std::vector<float> f(ARSO_N_FEATURES, 0.f);
    const size_t G = c->gates.size();
    std::vector<uint32_t> level(c->n, 0);
    uint32_t depth = 0;
    std::vector<char> layer_has_2q;
    static const uint32_t kinds[18] = {ARSO_GATE_H, ARSO_GATE_X, ARSO_GATE_Y, ARSO_GATE_Z, ARSO_GATE_S,
                                       ARSO_GATE_SDG, ARSO_GATE_T, ARSO_GATE_TDG, ARSO_GATE_RX, ARSO_GATE_RY,
                                       ARSO_GATE_RZ, ARSO_GATE_P, ARSO_GATE_U, ARSO_GATE_CX, ARSO_GATE_CZ,
                                       ARSO_GATE_CP, ARSO_GATE_SWAP, ARSO_GATE_U2};
    float counts[18] = {0};
    for (const HostGate &h : c->gates) {
        uint32_t lv = level[h.q0];
        if (h.arity == 2) lv = std::max(lv, level[h.q1]);
        lv += 1;
        level[h.q0] = lv;
        if (h.arity == 2) level[h.q1] = lv;
        depth = std::max(depth, lv);
        if (layer_has_2q.size() < lv + 1) layer_has_2q.resize(lv + 1, 0);
        if (h.arity == 2) layer_has_2q[lv] = 1;
        for (int i = 0; i < 18; ++i)
            if (kinds[i] == h.kind) counts[i] += 1.f;
    }
    uint32_t layers2 = 0;
    for (char b : layer_has_2q) layers2 += b ? 1 : 0;
    f[0] = (float)c->n;
    f[1] = (float)G;
    f[2] = (float)c->L;
    f[3] = (float)c->k;
    f[4] = (float)c->m;
    f[5] = (float)depth;
    f[6] = (float)layers2;
    f[7] = (float)std::log10(std::max<double>(1.0, (double)c->L));
    f[8] = (float)std::log10(std::max<double>(1.0, (double)G));
    f[9] = G ? (float)c->m / (float)G : 0.f;
    for (int i = 0; i < 18; ++i) f[10 + i] = counts[i];
    if (crit && crit->kind <= ARSO_CRIT_ARGMAX) f[28 + crit->kind] = 1.f;
    return f;
}

}  // namespace arso
