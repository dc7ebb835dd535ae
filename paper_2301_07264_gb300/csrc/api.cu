// C-ABI entry points: circuit upload, prefix cache, error sampling,
// trajectory engines, success probability (Sec. IV-C, Eq. (4)) and the
// tolerable error rate (Sec. IV-D, Eq. (5), Fig. 3).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>

#include "kernels.h"
#include "prof.h"

namespace arso {

static thread_local std::string g_last_error;
void set_last_error(const std::string &m) { g_last_error = m; }

template <class F> static arso_status guard(F &&f) {
    try {
        f();
        return ARSO_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return ARSO_ENOMEM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return ARSO_ECUDA;
    }
}

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Stream-ordered scratch buffer.
struct Scratch {
    void *ptr = nullptr;
    cudaStream_t st;
    explicit Scratch(cudaStream_t s, size_t bytes) : st(s) {
        if (bytes) ARSO_CUDA(cudaMallocAsync(&ptr, bytes, st));
    }
    ~Scratch() {
        if (ptr) cudaFreeAsync(ptr, st);
    }
    Scratch(const Scratch &) = delete;
    template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

static void copy_h2d(void *dst, const void *src, size_t bytes, cudaStream_t st) {
    ARSO_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    prof_count_h2d(bytes);
}
static void copy_d2h(void *dst, const void *src, size_t bytes, cudaStream_t st) {
    ARSO_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
    prof_count_d2h(bytes);
}
template <typename T> static void h2d(void *dst, const std::vector<T> &v, cudaStream_t st) {
    if (!v.empty()) copy_h2d(dst, v.data(), v.size() * sizeof(T), st);
}

// ------------------------------------------------------------ upload -------
// op code and mask-adjustment fields of a register-kernel gate record
static uint32_t reg_opcode(uint32_t cls, uint32_t p0, uint32_t p1) {
    auto enc = [](uint32_t opc, uint32_t sa, uint32_t sb, uint32_t xa, uint32_t xb) {
        return opc | sa << 8 | sb << 10 | xa << 12 | xb << 13;
    };
    const uint32_t R = (uint32_t)REG_BITS;
    switch (cls) {
        case GC_SU2: return enc(OP_SU2 + p0, 0, 0, 0, 0);
        case GC_DENSE1: return enc(OP_DENSE1 + p0, 0, 0, 0, 0);
        case GC_H: return enc(OP_H + 2 * p0, 1, 0, 0, 0);  // + flip = bit q0 of m
        case GC_CZ: {
            if (p0 < R && p1 < R) {
                const uint32_t lo = std::min(p0, p1), hi = std::max(p0, p1);
                const uint32_t pp = lo == 0 ? hi - 1 : lo == 1 ? hi + 2 : lo == 2 ? hi + 4 : 9;
                // want = 1 ^ mask bit; the lower position carries weight 2
                return p0 < p1 ? enc(OP_CZ_RR + 4 * pp, 2, 1, 1, 1) : enc(OP_CZ_RR + 4 * pp, 1, 2, 1, 1);
            }
            if (p0 < R) return enc(OP_CZ_RT + 2 * p0, 1, 0, 1, 0);
            if (p1 < R) return enc(OP_CZ_RT + 2 * p1, 0, 1, 0, 1);
            return enc(OP_CZ_TT, 0, 0, 0, 0);
        }
        case GC_X: return enc(OP_X, 0, 0, 0, 0);
        case GC_OMEGA: return enc(OP_OMEGA, 0, 0, 0, 0);
        case GC_DIAG1: return enc(OP_DIAG1, 0, 0, 0, 0);
        case GC_DIAG2: return enc(OP_DIAG2, 0, 0, 0, 0);
        case GC_CX: return enc(OP_CX + std::min(p1, R - 1), 0, 0, 0, 0);
        case GC_DENSE2: return enc(OP_DENSE2, 0, 0, 0, 0);
        case GC_SWAP: return enc(OP_SWAP, 0, 0, 0, 0);
        default: return enc(OP_NOP, 0, 0, 0, 0);
    }
}

static void upload_circuit(arso_circuit *c) {
    const size_t G = c->gates.size();
    std::vector<DGate> dg(std::max<size_t>(G, 1));
    std::vector<std::complex<double>> pool;
    for (size_t p = 0; p < c->passes.size(); ++p) {
        const Pass &ps = c->passes[p];
        std::vector<int> local(c->n, -1);
        for (size_t i = 0; i < ps.tile_qubits.size(); ++i) local[ps.tile_qubits[i]] = (int)i;
        for (uint32_t pos = ps.gb; pos < ps.ge; ++pos) {
            const HostGate &h = c->gates[c->perm[pos]];
            DGate d{};
            d.cls = h.cls;
            d.arity = (uint8_t)h.arity;
            d.q0 = (uint8_t)local[h.q0];
            d.q1 = (uint8_t)local[h.q1];
            d.mat = h.cls == GC_OMEGA ? h.omega_k : (uint32_t)pool.size();
            switch (h.cls) {
                case GC_DENSE1: for (int i = 0; i < 4; ++i) pool.push_back(h.m[i]); break;
                case GC_DIAG1: pool.push_back(h.m[0]); pool.push_back(h.m[3]); break;
                case GC_DENSE2: for (int i = 0; i < 16; ++i) pool.push_back(h.m[i]); break;
                case GC_DIAG2: for (int i = 0; i < 4; ++i) pool.push_back(h.m[5 * i]); break;
                default: break;
            }
            // register kernels: a dense gate whose complex64 entries have the special
            // unitary form [[a, b], [-conj b, conj a]] exactly runs on a and b alone
            if (h.cls == GC_DENSE1 && c->reg_blocked) {
                const std::complex<float> a((float)h.m[0].real(), (float)h.m[0].imag());
                const std::complex<float> b((float)h.m[1].real(), (float)h.m[1].imag());
                const std::complex<float> u10((float)h.m[2].real(), (float)h.m[2].imag());
                const std::complex<float> u11((float)h.m[3].real(), (float)h.m[3].imag());
                if (u10 == -std::conj(b) && u11 == std::conj(a)) d.cls = GC_SU2;
            }
            dg[pos] = d;
        }
    }
    c->d_gates.ensure(dg.size() * sizeof(DGate));
    ARSO_CUDA(cudaMemcpy(c->d_gates.ptr, dg.data(), dg.size() * sizeof(DGate), cudaMemcpyHostToDevice));
    const size_t esz = c->precision == ARSO_C128 ? 16 : 8;
    c->d_mats.ensure(std::max<size_t>(pool.size(), 1) * esz);
    if (!pool.empty()) {
        if (c->precision == ARSO_C128) {
            std::vector<double2> v(pool.size());
            for (size_t i = 0; i < pool.size(); ++i) v[i] = make_double2(pool[i].real(), pool[i].imag());
            ARSO_CUDA(cudaMemcpy(c->d_mats.ptr, v.data(), v.size() * esz, cudaMemcpyHostToDevice));
        } else {
            std::vector<float2> v(pool.size());
            for (size_t i = 0; i < pool.size(); ++i)
                v[i] = make_float2((float)pool[i].real(), (float)pool[i].imag());
            ARSO_CUDA(cudaMemcpy(c->d_mats.ptr, v.data(), v.size() * esz, cudaMemcpyHostToDevice));
        }
    }
    std::vector<uint32_t> first_loc(G + 1, 0);
    for (size_t g = 0; g < G; ++g) first_loc[g + 1] = first_loc[g] + c->gates[g].arity;
    std::vector<uint32_t> lk(std::max<uint64_t>(c->L, 1));
    for (uint64_t l = 0; l < c->L; ++l) {
        const uint32_t g = c->loc_gate[l];
        lk[l] = (c->pos_of[g] << 1) | (uint32_t)(l - first_loc[g]);
    }
    c->d_loc_key.ensure(lk.size() * 4);
    ARSO_CUDA(cudaMemcpy(c->d_loc_key.ptr, lk.data(), lk.size() * 4, cudaMemcpyHostToDevice));
    if (c->engine == 1) {
        const uint32_t t = c->tile_qubits, cl = c->low_qubits;
        std::vector<uint32_t> offs;
        c->offs_base.clear();
        for (const Pass &ps : c->passes) {
            c->offs_base.push_back(offs.size());
            for (uint32_t jh = 0; jh < (1u << (t - cl)); ++jh) {
                uint64_t o = 0;
                for (uint32_t i = cl; i < t; ++i)
                    if ((jh >> (i - cl)) & 1u) o |= 1ull << ps.tile_qubits[i];
                ARSO_REQUIRE(o < (1ull << 32), "tile offset overflow");
                offs.push_back((uint32_t)o);
            }
        }
        c->d_offs.ensure(offs.size() * 4);
        ARSO_CUDA(cudaMemcpy(c->d_offs.ptr, offs.data(), offs.size() * 4, cudaMemcpyHostToDevice));
    }
    if (c->reg_blocked) {
        c->d_ph_gb.ensure(c->ph_gb.size() * 4);
        ARSO_CUDA(cudaMemcpy(c->d_ph_gb.ptr, c->ph_gb.data(), c->ph_gb.size() * 4, cudaMemcpyHostToDevice));
        c->d_ph_R.ensure(std::max<size_t>(c->ph_R.size(), 1) * 4);
        if (!c->ph_R.empty())
            ARSO_CUDA(cudaMemcpy(c->d_ph_R.ptr, c->ph_R.data(), c->ph_R.size() * 4, cudaMemcpyHostToDevice));
        std::vector<RegOp> ops(std::max<size_t>(dg.size(), 1));
        for (size_t pos = 0; pos < c->rpos.size(); ++pos) {
            const DGate &d = dg[pos];
            RegOp &o = ops[pos];
            o.w0 = (uint32_t)d.cls | (uint32_t)(c->rpos[pos] & 15u) << 8 | (uint32_t)(c->rpos[pos] >> 4) << 12 |
                   (uint32_t)d.q0 << 16 | (uint32_t)d.q1 << 24;
            o.aux = d.mat;
            const HostGate &h = c->gates[c->perm[pos]];
            o.pad[0] = reg_opcode(d.cls, c->rpos[pos] & 15u, c->rpos[pos] >> 4);
            o.pad[1] = c->tensor ? (uint32_t)c->role[pos] : (uint32_t)TR_CORE;
            if (d.cls == GC_SU2) {
                o.c0 = make_float2((float)h.m[0].real(), (float)h.m[0].imag());
                o.c1 = make_float2((float)h.m[1].real(), (float)h.m[1].imag());
            } else if (d.cls == GC_DIAG1) {
                o.c0 = make_float2((float)h.m[0].real(), (float)h.m[0].imag());
                o.c1 = make_float2((float)h.m[3].real(), (float)h.m[3].imag());
            }
        }
        c->d_rops.ensure(ops.size() * sizeof(RegOp));
        ARSO_CUDA(cudaMemcpy(c->d_rops.ptr, ops.data(), ops.size() * sizeof(RegOp), cudaMemcpyHostToDevice));
        if (c->tensor) {
            c->d_ph_t.ensure(std::max<size_t>(c->ph_t.size(), 1) * 4);
            if (!c->ph_t.empty())
                ARSO_CUDA(cudaMemcpy(c->d_ph_t.ptr, c->ph_t.data(), c->ph_t.size() * 4, cudaMemcpyHostToDevice));
            c->d_tmats.ensure(std::max<size_t>(c->tmats.size(), 8) * 2);
            if (!c->tmats.empty())
                ARSO_CUDA(cudaMemcpy(c->d_tmats.ptr, c->tmats.data(), c->tmats.size() * 2, cudaMemcpyHostToDevice));
            c->d_terr.ensure(4);
            ARSO_CUDA(cudaMemset(c->d_terr.ptr, 0, 4));
        }
        c->d_phase_of_pos.ensure(std::max<size_t>(c->phase_of_pos.size(), 1) * 4);
        if (!c->phase_of_pos.empty())
            ARSO_CUDA(cudaMemcpy(c->d_phase_of_pos.ptr, c->phase_of_pos.data(), c->phase_of_pos.size() * 4,
                                 cudaMemcpyHostToDevice));
    }
}

// resident arguments common to every launch
static ResidentArgs resident_args(const arso_circuit *c) {
    ResidentArgs a{};
    a.n = (int)c->n;
    a.G = (uint32_t)c->gates.size();
    a.gates = c->d_gates.as<DGate>();
    a.mats = c->d_mats.ptr;
    a.cache = c->d_cache.ptr;
    a.ckpt_every = c->ckpt_every;
    a.n_ckpt = c->n_ckpt;
    if (c->reg_blocked) {
        a.n_phases = (uint32_t)c->ph_R.size();
        a.ph_gb = c->d_ph_gb.as<uint32_t>();
        a.ph_R = c->d_ph_R.as<uint32_t>();
        a.rops = c->d_rops.as<RegOp>();
        a.phase_of_pos = c->d_phase_of_pos.as<uint32_t>();
    }
    return a;
}

static void launch_resident_any(const arso_circuit *c, const ResidentArgs &a, int mode, double bytes, cudaStream_t st) {
    if (c->reg_blocked) launch_resident_rb(a, mode, bytes, st);
    else launch_resident(a, mode == 2, c->precision, bytes, st);
}

// streaming pass launch: register-blocked kernel when the schedule has phases.
// sweeps = how many states the launch reads and writes once (active slots).
static void run_pass(const arso_circuit *c, const PassArgs &a, bool last, uint32_t slots, double sweeps,
                     cudaStream_t st) {
    const double bytes = 2.0 * (double)c->state_bytes() * sweeps;
    if (c->reg_blocked) {
        PassArgs b = a;
        b.pb = c->passes[a.pass].pb;
        b.pe = c->passes[a.pass].pe;
        b.ph_gb = c->d_ph_gb.as<uint32_t>();
        b.ph_R = c->d_ph_R.as<uint32_t>();
        b.rops = c->d_rops.as<RegOp>();
        if (c->tensor) {
            b.ph_t = c->d_ph_t.as<uint32_t>();
            b.tmats = c->d_tmats.ptr;
            b.terr = c->d_terr.as<uint32_t>();
        }
        const Pass &ps = c->passes[a.pass];
        launch_pass_rb(b, last, slots, bytes, st, ps.flops_per_amp * std::ldexp(sweeps, (int)c->n),
                       (double)(ps.remaps + ps.end_remap) * 16.0 * std::ldexp(sweeps, (int)c->n));
    } else {
        launch_pass(a, last, c->precision, slots, bytes, st);
    }
}

// Synchronises; ARSO_ETIMEOUT when a tensor-phase wait of the circuit's pass
// launches gave up since the last check (the word is cleared).
static void check_tensor(const arso_circuit *c, cudaStream_t st) {
    uint32_t err = 0;
    if (c->tensor) copy_d2h(&err, c->d_terr.ptr, 4, st);
    ARSO_CUDA(cudaStreamSynchronize(st));
    if (err) {
        ARSO_CUDA(cudaMemsetAsync(c->d_terr.ptr, 0, 4, st));
        ARSO_CUDA(cudaStreamSynchronize(st));
        throw Error(ARSO_ETIMEOUT, "tensor phase: a wait for the tensor cores gave up");
    }
}

// ----------------------------------------------------------- prefix cache --
static void ensure_cache(arso_circuit *c, cudaStream_t st) {
    if (c->cache_ready) return;
    const size_t sb = c->state_bytes();
    const uint64_t G = c->gates.size();
    if (c->engine == 0) {
        // checkpoints every `every` gates (or phases when register-blocked)
        const uint64_t units = c->reg_blocked ? c->ph_R.size() : G;
        const uint64_t budget = std::min<uint64_t>(c->cache_budget, 512ull << 20);
        uint64_t every = std::max<uint64_t>(1, ((units + 1) * sb + budget - 1) / budget);
        c->ckpt_every = every;
        c->n_ckpt = (uint32_t)(units / every + 1 + (units % every ? 1 : 0));
        c->d_cache.ensure((size_t)c->n_ckpt * sb);
        launch_resident_any(c, resident_args(c), 2, (double)c->n_ckpt * sb, st);
    } else {
        const uint32_t P = (uint32_t)c->passes.size();
        // boundaries 0..P; cache every s-th boundary and the last one
        uint32_t s = 1;
        while ((uint64_t)((P + s - 1) / s + 2) * sb > c->cache_budget && s < P) ++s;
        c->ckpt_pass.assign(P + 1, NO_EVENT);
        uint32_t slots = 0;
        for (uint32_t j = 0; j <= P; ++j)
            if (j % s == 0 || j == P) c->ckpt_pass[j] = slots++;
        c->n_ckpt = slots;
        c->d_cache.ensure((size_t)slots * sb);
        Scratch work(st, s > 1 ? sb : 0);
        char *base = c->d_cache.as<char>();
        launch_init_zero_state(base, (int)c->n, c->precision, st);
        for (uint32_t j = 0; j < P; ++j) {
            PassArgs a{};
            a.n = (int)c->n;
            a.t = (int)c->tile_qubits;
            a.c = (int)c->low_qubits;
            uint64_t tm = 0;
            for (uint32_t q : c->passes[j].tile_qubits) tm |= 1ull << q;
            a.rest_mask = ((c->n == 64 ? 0 : (1ull << c->n)) - 1) & ~tm;
            a.offs = c->d_offs.as<uint32_t>() + c->offs_base[j];
            a.gb = c->passes[j].gb;
            a.ge = c->passes[j].ge;
            a.pass = (int)j;
            a.gates = c->d_gates.as<DGate>();
            a.mats = c->d_mats.ptr;
            a.ideal = 1;
            a.ideal_src = c->ckpt_pass[j] != NO_EVENT ? base + (size_t)c->ckpt_pass[j] * sb : work.ptr;
            a.ideal_dst = c->ckpt_pass[j + 1] != NO_EVENT ? base + (size_t)c->ckpt_pass[j + 1] * sb : work.ptr;
            run_pass(c, a, false, 1, 1.0, st);
        }
    }
    ARSO_CUDA(cudaStreamSynchronize(st));
    c->cache_ready = true;
}

static const void *ref_state_ptr(const arso_circuit *c) {
    return c->d_cache.as<char>() + (size_t)(c->n_ckpt - 1) * c->state_bytes();
}

// A host gate in the form of the single-gate HBM kernels (global qubits; H and the
// omega phases as dense / diagonal gates, CZ as a diagonal), or its adjoint.
static void hbm_gate(const HostGate &h, bool adjoint, DGate &d, M16 &m) {
    d = DGate{};
    d.cls = h.cls == GC_H ? (uint8_t)GC_DENSE1
          : h.cls == GC_OMEGA ? (uint8_t)GC_DIAG1 : h.cls == GC_CZ ? (uint8_t)GC_DIAG2 : h.cls;
    d.arity = (uint8_t)h.arity;
    d.q0 = (uint8_t)h.q0;
    d.q1 = (uint8_t)h.q1;
    const int dim = h.arity == 1 ? 2 : 4;
    auto e = [&](int r, int col) { return adjoint ? std::conj(h.m[col * dim + r]) : h.m[r * dim + col]; };
    auto f2 = [](std::complex<double> v) { return make_float2((float)v.real(), (float)v.imag()); };
    m = M16{};
    if (h.arity == 1 && d.cls == GC_DIAG1) {
        m.m[0] = f2(e(0, 0));
        m.m[1] = f2(e(1, 1));
    } else if (d.cls != GC_NOP) {
        for (int r = 0; r < dim; ++r)
            for (int col = 0; col < dim; ++col) m.m[r * dim + col] = f2(e(r, col));
    }
}

// Backward states for the outcome criterion's suffix reuse (streaming, complex64):
// phi_j = (gates of passes j..P-1)^dagger |target> at every cached pass boundary j,
// built from |target> by the adjoint gates in reverse engine order.
static bool bwd_supported(const arso_circuit *c) { return c->engine == 1 && c->precision == ARSO_C64; }

static void ensure_bwd_cache(arso_circuit *c, uint64_t target, cudaStream_t st) {
    if (c->bwd_ready && c->bwd_target == target) return;
    ensure_cache(c, st);
    const size_t sb = c->state_bytes();
    const uint32_t P = (uint32_t)c->passes.size();
    c->bwd_ready = false;
    c->d_bwd.ensure((size_t)c->n_ckpt * sb);
    char *base = c->d_bwd.as<char>();
    Scratch work(st, sb);
    const float2 one = make_float2(1.f, 0.f);
    ARSO_CUDA(cudaMemsetAsync(work.ptr, 0, sb, st));
    copy_h2d(work.as<float2>() + target, &one, sizeof(float2), st);
    ARSO_CUDA(cudaMemcpyAsync(base + (size_t)c->ckpt_pass[P] * sb, work.ptr, sb, cudaMemcpyDeviceToDevice, st));
    for (uint32_t j = P; j-- > 0;) {
        for (uint32_t pos = c->passes[j].ge; pos-- > c->passes[j].gb;) {
            const HostGate &h = c->gates[c->perm[pos]];
            if (h.cls == GC_NOP) continue;
            DGate d;
            M16 m;
            hbm_gate(h, true, d, m);
            launch_gate_pairs(work.as<float2>(), (int)c->n, d, m, st);
        }
        if (c->ckpt_pass[j] != NO_EVENT)
            ARSO_CUDA(cudaMemcpyAsync(base + (size_t)c->ckpt_pass[j] * sb, work.ptr, sb, cudaMemcpyDeviceToDevice, st));
    }
    ARSO_CUDA(cudaStreamSynchronize(st));
    c->bwd_target = target;
    c->bwd_ready = true;
}

// whether the trajectories of `crit` stop after their last error's pass (fidelity,
// and outcome probability through the backward states)
static bool suffix_wanted(const arso_circuit *c, const DCrit &crit) {
    if (c->flags & ARSO_OPT_NO_SUFFIX_REUSE) return false;
    return crit.kind == ARSO_CRIT_FIDELITY || (crit.kind == ARSO_CRIT_OUTCOME && bwd_supported(c));
}

// ------------------------------------------------------------ criterion ----
struct DevCrit {
    DCrit d{};
    uint32_t aggregate = 0;
    DeviceBuffer bitmap;
};

static void make_crit(const arso_circuit *c, const arso_criterion *crit, DevCrit &out, cudaStream_t st) {
    ARSO_REQUIRE(crit != nullptr, "criterion is NULL");
    ARSO_REQUIRE(crit->kind <= ARSO_CRIT_ARGMAX, "bad criterion kind");
    ARSO_REQUIRE(crit->aggregate <= ARSO_AGG_PASS, "bad aggregate");
    const uint64_t N = 1ull << c->n;
    if (crit->kind == ARSO_CRIT_OUTCOME || crit->kind == ARSO_CRIT_ARGMAX)
        ARSO_REQUIRE(crit->target < N, "criterion target out of range");
    out.d.kind = crit->kind;
    out.d.threshold = crit->threshold;
    out.d.target = crit->target;
    out.d.bitmap = nullptr;
    out.aggregate = crit->aggregate;
    if (crit->kind == ARSO_CRIT_BINNING) {
        ARSO_REQUIRE(crit->set_len == 0 || crit->set != nullptr, "binning set is NULL");
        std::vector<uint32_t> bm((N + 31) / 32, 0);
        for (size_t i = 0; i < crit->set_len; ++i) {
            ARSO_REQUIRE(crit->set[i] < N, "binning outcome out of range");
            bm[crit->set[i] >> 5] |= 1u << (crit->set[i] & 31);
        }
        out.bitmap.ensure(bm.size() * 4);
        copy_h2d(out.bitmap.ptr, bm.data(), bm.size() * 4, st);
        ARSO_CUDA(cudaStreamSynchronize(st));
        out.d.bitmap = out.bitmap.as<uint32_t>();
    }
}

// score of an arbitrary device state into a device scalar
static void score_into(const void *psi, const void *ref, int n, int precision, const DCrit &crit, double *d_out,
                       cudaStream_t st) {
    Scratch parts(st, 152 * 8 * sizeof(Partial));
    const uint32_t blocks = launch_score_partials(psi, ref, n, precision, crit, parts.as<Partial>(), 152 * 8, st);
    launch_finish_partials(parts.as<Partial>(), blocks, 1, nullptr, crit, d_out, nullptr, st);
}

// -------------------------------------------------------------- engines ----
static PassArgs pass_args(const arso_circuit *c, uint32_t j) {
    PassArgs a{};
    a.n = (int)c->n;
    a.t = (int)c->tile_qubits;
    a.c = (int)c->low_qubits;
    uint64_t tm = 0;
    for (uint32_t q : c->passes[j].tile_qubits) tm |= 1ull << q;
    a.rest_mask = ((1ull << c->n) - 1) & ~tm;
    a.offs = c->d_offs.as<uint32_t>() + c->offs_base[j];
    a.gb = c->passes[j].gb;
    a.ge = c->passes[j].ge;
    a.pass = (int)j;
    a.gates = c->d_gates.as<DGate>();
    a.mats = c->d_mats.ptr;
    return a;
}

struct GraphKey {
    int jmin, jmax;
    uint32_t slots;
    bool operator<(const GraphKey &o) const {
        return jmin != o.jmin ? jmin < o.jmin : jmax != o.jmax ? jmax < o.jmax : slots < o.slots;
    }
};
// Stream capture of one batch's launches. If capture cannot start, launches go
// directly to the stream; if anything throws while capturing, the capture is
// ended and discarded so the caller's stream is left usable.
struct CaptureGuard {
    cudaStream_t st;
    bool active = false;
    CaptureGuard(cudaStream_t s, bool want) : st(s) {
        if (!want) return;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            active = true;
            prof_suspend(true);
        } else {
            cudaGetLastError();
        }
    }
    cudaGraphExec_t finish() {
        prof_suspend(false);
        active = false;
        cudaGraph_t g = nullptr;
        ARSO_CUDA(cudaStreamEndCapture(st, &g));
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        ARSO_CUDA(ie);
        return ex;
    }
    ~CaptureGuard() {
        if (!active) return;
        prof_suspend(false);
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(st, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    }
};

struct GraphCache : std::map<GraphKey, cudaGraphExec_t> {
    ~GraphCache() {
        for (auto &kv : *this) cudaGraphExecDestroy(kv.second);
    }
};

// Streaming engine over trajectories `ids` of the error list. states_out
// (non-null) receives final states in the order of `ids` instead of scores.
static void run_streaming(arso_circuit *c, const arso_error_list *e, const std::vector<uint64_t> &ids,
                          const std::vector<uint32_t> &first_pos, const std::vector<uint32_t> &last_pos,
                          const DCrit &crit, double *d_score, uint8_t *d_pass, void *states_out, cudaStream_t st) {
    if (ids.empty()) return;
    const uint32_t P = (uint32_t)c->passes.size();
    const size_t sb = c->state_bytes();
    const uint32_t tiles = 1u << (c->n - c->tile_qubits);
    // start: the last cached boundary at or before the first error's pass.
    // end: the pass whose output is scored. Fidelity is invariant under the
    // error-free suffix W that follows the last error (<W a|W b> = <a|b>), so
    // the trajectory is scored right after its last error's pass against the
    // cached error-free state at that boundary (the first cached one after
    // it); other criteria need the final state (end = P - 1).
    // The outcome probability |<t|psi>|^2 is scored the same way, as the overlap with
    // the backward state W^dagger |t> at that boundary (|<t|W a>| = |<W^dagger t|a>|).
    const bool suffix = !states_out && suffix_wanted(c, crit);
    const bool outcome_overlap = suffix && crit.kind == ARSO_CRIT_OUTCOME;
    if (outcome_overlap) ARSO_REQUIRE(c->bwd_ready && c->bwd_target == crit.target, "backward states not built");
    DCrit kcrit = crit;  // what the kernels score: the overlap for the outcome criterion
    if (outcome_overlap) kcrit.kind = ARSO_CRIT_FIDELITY;
    std::vector<int> start(ids.size()), end(ids.size());
    for (size_t i = 0; i < ids.size(); ++i) {
        uint32_t fp = first_pos[i] == NO_EVENT ? P - 1 : c->pass_of_pos[first_pos[i]];
        while (c->ckpt_pass[fp] == NO_EVENT) --fp;
        start[i] = (int)fp;
        uint32_t lp = P - 1;
        if (suffix && last_pos[i] != NO_EVENT) {
            lp = c->pass_of_pos[last_pos[i]];
            while (c->ckpt_pass[lp + 1] == NO_EVENT) ++lp;
        }
        end[i] = (int)lp;
    }
    std::vector<size_t> order(ids.size());
    std::iota(order.begin(), order.end(), 0);
    if (!states_out)
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
            return start[x] != start[y] ? start[x] < start[y] : end[x] < end[y];
        });
    uint64_t B = c->max_batch ? c->max_batch : std::max<uint64_t>(1, (8ull << 30) / sb);
    B = std::min<uint64_t>(B, std::min<uint64_t>(ids.size(), 65535));
    if (states_out) B = ids.size();
    ARSO_REQUIRE(B <= 65535, "too many states requested at once");
    Scratch work(st, states_out ? 0 : B * sb);
    Scratch parts(st, states_out ? 0 : B * tiles * sizeof(Partial));
    Scratch d_slot_traj(st, B * 8), d_start(st, B * 4), d_end(st, B * 4);
    std::vector<uint32_t> cslot(c->ckpt_pass.begin(), c->ckpt_pass.end());
    Scratch d_cslot(st, cslot.size() * 4);
    h2d(d_cslot.ptr, cslot, st);
    // captured pass sequences of this call, replayed for batches of the same shape
    GraphCache graphs;
    // the legacy default stream cannot be captured
    const bool use_graphs = !states_out && c->reg_blocked && !(c->flags & ARSO_OPT_NO_GRAPHS) && st != nullptr &&
                            st != cudaStreamLegacy && st != cudaStreamPerThread;
    if (use_graphs) prepare_pass_rb();
    for (size_t b0 = 0; b0 < ids.size(); b0 += B) {
        const size_t nb = std::min<size_t>(B, ids.size() - b0);
        std::vector<uint64_t> st_traj(nb);
        std::vector<int> st_start(nb), st_end(nb);
        int jmin = (int)P, jmax = 0;
        for (size_t i = 0; i < nb; ++i) {
            st_traj[i] = ids[order[b0 + i]];
            st_start[i] = start[order[b0 + i]];
            st_end[i] = end[order[b0 + i]];
            jmin = std::min(jmin, st_start[i]);
            jmax = std::max(jmax, st_end[i]);
        }
        h2d(d_slot_traj.ptr, st_traj, st);
        h2d(d_start.ptr, st_start, st);
        h2d(d_end.ptr, st_end, st);
        double batch_bytes = 0, batch_flops = 0, batch_smem = 0;
        for (uint32_t j = (uint32_t)jmin; j <= (uint32_t)jmax; ++j)
            for (size_t i = 0; i < nb; ++i)
                if (st_start[i] <= (int)j && (int)j <= st_end[i]) {
                    batch_bytes += 2.0 * sb;
                    batch_flops += c->reg_blocked ? c->passes[j].flops_per_amp * std::ldexp(1.0, (int)c->n) : 0.0;
                    batch_smem += c->reg_blocked ? (double)(c->passes[j].remaps + c->passes[j].end_remap) * 16.0 *
                                                       std::ldexp(1.0, (int)c->n)
                                                 : 0.0;
                }
        const uint64_t n_launch = (uint64_t)(jmax - jmin + 1) + (states_out ? 0 : 1);
        const GraphKey key{jmin, jmax, (uint32_t)nb};
        auto hit = graphs.find(key);
        if (hit != graphs.end()) {  // replay: the slot tables above are the only inputs that changed
            {
                ProfScope ps_(ARSO_K_PASS, batch_bytes, st, batch_flops, batch_smem);
                ARSO_CUDA(cudaGraphLaunch(hit->second, st));
            }
            prof_add_launches(ARSO_K_PASS, n_launch - 1);
            ARSO_CUDA(cudaStreamSynchronize(st));
            continue;
        }
        CaptureGuard capture(st, use_graphs);
        for (uint32_t j = (uint32_t)jmin; j <= (uint32_t)jmax; ++j) {
            PassArgs a = pass_args(c, j);
            a.cache = c->d_cache.ptr;
            a.ref_cache = outcome_overlap ? c->d_bwd.ptr : nullptr;
            a.cache_slot = d_cslot.as<uint32_t>();
            a.ref_slot = c->n_ckpt - 1;
            a.work = states_out ? states_out : work.ptr;
            a.start_pass = d_start.as<int>();
            a.end_pass = d_end.as<int>();
            a.slot_traj = d_slot_traj.as<uint64_t>();
            a.offsets = e->d_offsets.as<uint64_t>();
            a.keys = e->d_key.as<uint32_t>();
            a.crit = kcrit;
            a.partials = parts.as<Partial>();
            a.store_last = states_out ? 1 : 0;
            uint32_t active = 0;
            for (size_t i = 0; i < nb; ++i) active += st_start[i] <= (int)j && (int)j <= st_end[i];
            run_pass(c, a, j == P - 1, (uint32_t)nb, (double)active, st);
        }
        if (!states_out)
            launch_finish_partials(parts.as<Partial>(), tiles, (uint32_t)nb, d_slot_traj.as<uint64_t>(), kcrit,
                                   d_score, d_pass, st);
        if (capture.active) {
            cudaGraphExec_t ex = capture.finish();
            graphs[key] = ex;
            {
                ProfScope ps_(ARSO_K_PASS, batch_bytes, st, batch_flops, batch_smem);
                ARSO_CUDA(cudaGraphLaunch(ex, st));
            }
            prof_add_launches(ARSO_K_PASS, n_launch - 1);
        }
        ARSO_CUDA(cudaStreamSynchronize(st));  // host vectors and slot tables are reused per batch
    }
}

static void run_all(arso_circuit *c, const arso_error_list *e, const DevCrit &dc, cudaStream_t st, double *d_score,
                    uint8_t *d_pass) {
    ensure_cache(c, st);
    Scratch ref(st, sizeof(double));
    score_into(ref_state_ptr(c), ref_state_ptr(c), (int)c->n, c->precision, dc.d, ref.as<double>(), st);
    if (e->n_traj == 0) return;
    if (c->engine == 0) {
        ResidentArgs a = resident_args(c);
        a.first_traj = 0;
        a.count = e->n_traj;
        a.offsets = e->d_offsets.as<uint64_t>();
        a.keys = e->d_key.as<uint32_t>();
        a.first = e->d_first.as<uint32_t>();
        a.crit = dc.d;
        a.ref_score = ref.as<double>();
        a.score = d_score;
        a.pass_flags = d_pass;
        launch_resident_any(c, a, 0, (double)e->n_traj * c->state_bytes(), st);
        ARSO_CUDA(cudaStreamSynchronize(st));
        return;
    }
    launch_fill_error_free(e->d_first.as<uint32_t>(), e->n_traj, ref.as<double>(), dc.d.threshold, d_score, d_pass, st);
    if (dc.d.kind == ARSO_CRIT_OUTCOME && suffix_wanted(c, dc.d)) ensure_bwd_cache(c, dc.d.target, st);
    std::vector<uint32_t> first(e->n_traj), last(e->n_traj);
    copy_d2h(first.data(), e->d_first.ptr, e->n_traj * 4, st);
    copy_d2h(last.data(), e->d_last.ptr, e->n_traj * 4, st);
    ARSO_CUDA(cudaStreamSynchronize(st));
    std::vector<uint64_t> ids;
    std::vector<uint32_t> fp, lp;
    for (uint64_t i = 0; i < e->n_traj; ++i)
        if (first[i] != NO_EVENT) ids.push_back(i), fp.push_back(first[i]), lp.push_back(last[i]);
    run_streaming(c, e, ids, fp, lp, dc.d, d_score, d_pass, nullptr, st);
    check_tensor(c, st);
}

// ------------------------------------------------------------ sampling -----
static arso_error_list *new_list(const arso_circuit *c, uint64_t n_traj) {
    auto *e = new arso_error_list();
    e->circ = c;
    e->n_traj = n_traj;
    e->d_offsets.ensure((n_traj + 1) * 8);
    e->d_first.ensure(std::max<uint64_t>(n_traj, 1) * 4);
    e->d_last.ensure(std::max<uint64_t>(n_traj, 1) * 4);
    return e;
}

static void finish_list(const arso_circuit *c, arso_error_list *e, cudaStream_t st) {
    bool identity = true;
    for (size_t i = 0; i < c->perm.size() && identity; ++i) identity = c->perm[i] == i;
    if (!identity) launch_sort_keys(e->d_offsets.as<uint64_t>(), e->n_traj, e->d_key.as<uint32_t>(), st);
    launch_first_event(e->d_offsets.as<uint64_t>(), e->n_traj, e->d_key.as<uint32_t>(), e->d_first.as<uint32_t>(),
                       e->d_last.as<uint32_t>(), st);
    ARSO_CUDA(cudaStreamSynchronize(st));
}

static void sample(const arso_circuit *c, double px, double pz, double py, uint64_t seed, uint64_t begin,
                   uint64_t n_traj, cudaStream_t st, arso_error_list **out) {
    ARSO_REQUIRE(px >= 0 && pz >= 0 && py >= 0, "error probabilities must be >= 0");
    const double pt = px + pz + py;
    ARSO_REQUIRE(pt <= 1.0, "p_x + p_z + p_y must be <= 1");
    ARSO_REQUIRE(begin + n_traj >= begin, "trajectory range overflows");
    std::unique_ptr<arso_error_list> e(new_list(c, n_traj));
    SampleArgs a{};
    a.seed = seed;
    a.traj_begin = begin;
    a.n_traj = n_traj;
    a.L = (uint32_t)c->L;
    if (pt > 0) {
        const double two32 = 4294967296.0;
        a.thr = (uint32_t)std::min(std::floor(pt * two32), 4294967295.0);
        const double cx = std::floor(px / pt * two32), cxz = std::floor((px + pz) / pt * two32);
        a.cut_x_all = cx >= two32;
        a.cut_xz_all = cxz >= two32;
        a.cut_x = a.cut_x_all ? 0 : (uint32_t)cx;
        a.cut_xz = a.cut_xz_all ? 0 : (uint32_t)cxz;
    }
    Scratch counts(st, std::max<uint64_t>(n_traj, 1) * 4);
    if (a.thr == 0 || c->L == 0) {
        ARSO_CUDA(cudaMemsetAsync(counts.ptr, 0, std::max<uint64_t>(n_traj, 1) * 4, st));
    } else {
        launch_sample_count(a, counts.as<uint32_t>(), st);
    }
    launch_exclusive_scan(counts.as<uint32_t>(), n_traj, e->d_offsets.as<uint64_t>(), st);
    uint64_t total = 0;
    copy_d2h(&total, e->d_offsets.as<uint64_t>() + n_traj, 8, st);
    ARSO_CUDA(cudaStreamSynchronize(st));
    e->n_events = total;
    e->d_loc.ensure(std::max<uint64_t>(total, 1) * 4);
    e->d_key.ensure(std::max<uint64_t>(total, 1) * 4);
    if (total) launch_sample_fill(a, e->d_offsets.as<uint64_t>(), c->d_loc_key.as<uint32_t>(), e->d_loc.as<uint32_t>(),
                                  e->d_key.as<uint32_t>(), st);
    finish_list(c, e.get(), st);
    *out = e.release();
}

static SampleArgs sample_args(const arso_circuit *c, double px, double pz, double py, uint64_t seed, uint64_t begin,
                              uint64_t n_traj) {
    ARSO_REQUIRE(px >= 0 && pz >= 0 && py >= 0, "error probabilities must be >= 0");
    const double pt = px + pz + py;
    ARSO_REQUIRE(pt <= 1.0, "p_x + p_z + p_y must be <= 1");
    ARSO_REQUIRE(begin + n_traj >= begin, "trajectory range overflows");
    SampleArgs a{};
    a.seed = seed;
    a.traj_begin = begin;
    a.n_traj = n_traj;
    a.L = (uint32_t)c->L;
    if (pt > 0 && c->L > 0) {
        const double two32 = 4294967296.0;
        a.thr = (uint32_t)std::min(std::floor(pt * two32), 4294967295.0);
        const double cx = std::floor(px / pt * two32), cxz = std::floor((px + pz) / pt * two32);
        a.cut_x_all = cx >= two32;
        a.cut_xz_all = cxz >= two32;
        a.cut_x = a.cut_x_all ? 0 : (uint32_t)cx;
        a.cut_xz = a.cut_xz_all ? 0 : (uint32_t)cxz;
    }
    return a;
}

// Error lists of many circuits with one launch of each sampling kernel.
static void sample_batch(size_t count, const arso_circuit *const *circuits, const double *px, const double *pz,
                         const double *py, const uint64_t *seeds, const uint64_t *begins, const uint64_t *n_traj,
                         cudaStream_t st, arso_error_list **out) {
    std::vector<std::unique_ptr<arso_error_list>> lists(count);
    std::vector<SampleJob> jobs(count);
    uint64_t total = 0;
    for (size_t i = 0; i < count; ++i) {
        const arso_circuit *c = circuits[i];
        ARSO_REQUIRE(c != nullptr, "NULL circuit");
        SampleJob &J = jobs[i];
        J.a = sample_args(c, px[i], pz[i], py[i], seeds[i], begins[i], n_traj[i]);
        lists[i].reset(new_list(c, n_traj[i]));
        J.traj0 = total;
        total += n_traj[i];
        J.offsets = lists[i]->d_offsets.as<uint64_t>();
        J.loc_key = c->d_loc_key.as<uint32_t>();
        J.first = lists[i]->d_first.as<uint32_t>();
        J.last = lists[i]->d_last.as<uint32_t>();
        bool identity = true;
        for (size_t g = 0; g < c->perm.size() && identity; ++g) identity = c->perm[g] == g;
        J.identity = identity;
    }
    if (count) {
        Scratch d_jobs(st, count * sizeof(SampleJob)), counts(st, std::max<uint64_t>(total, 1) * 4),
            totals(st, count * 8);
        copy_h2d(d_jobs.ptr, jobs.data(), count * sizeof(SampleJob), st);
        launch_sample_batch_count(d_jobs.as<SampleJob>(), (uint32_t)count, total, counts.as<uint32_t>(),
                                  totals.as<uint64_t>(), st);
        std::vector<uint64_t> ev(count);
        copy_d2h(ev.data(), totals.ptr, count * 8, st);
        ARSO_CUDA(cudaStreamSynchronize(st));
        bool any = false;
        for (size_t i = 0; i < count; ++i) {
            lists[i]->n_events = ev[i];
            lists[i]->d_loc.ensure(std::max<uint64_t>(ev[i], 1) * 4);
            lists[i]->d_key.ensure(std::max<uint64_t>(ev[i], 1) * 4);
            jobs[i].ev_loc = lists[i]->d_loc.as<uint32_t>();
            jobs[i].ev_key = lists[i]->d_key.as<uint32_t>();
            any |= ev[i] > 0;
        }
        copy_h2d(d_jobs.ptr, jobs.data(), count * sizeof(SampleJob), st);
        launch_sample_batch_fill(d_jobs.as<SampleJob>(), (uint32_t)count, total, any, st);
        ARSO_CUDA(cudaStreamSynchronize(st));
    }
    for (size_t i = 0; i < count; ++i) out[i] = lists[i].release();
}

static void list_from_host(const arso_circuit *c, uint64_t n_traj, const uint64_t *offsets, const uint32_t *events,
                           cudaStream_t st, arso_error_list **out) {
    ARSO_REQUIRE(offsets != nullptr, "offsets is NULL");
    ARSO_REQUIRE(offsets[0] == 0, "offsets[0] must be 0");
    for (uint64_t t = 0; t < n_traj; ++t) {
        ARSO_REQUIRE(offsets[t + 1] >= offsets[t], "offsets must be non-decreasing");
        for (uint64_t i = offsets[t]; i < offsets[t + 1]; ++i) {
            ARSO_REQUIRE((events[i] >> 2) < c->L, "event location out of range");
            ARSO_REQUIRE((events[i] & 3u) != 0, "event code must be 1 (X), 2 (Z) or 3 (Y)");
            ARSO_REQUIRE(i == offsets[t] || (events[i] >> 2) > (events[i - 1] >> 2),
                         "events must be strictly increasing in location within a trajectory");
        }
    }
    const uint64_t total = offsets[n_traj];
    ARSO_REQUIRE(total == 0 || events != nullptr, "events is NULL");
    std::unique_ptr<arso_error_list> e(new_list(c, n_traj));
    e->n_events = total;
    e->d_loc.ensure(std::max<uint64_t>(total, 1) * 4);
    e->d_key.ensure(std::max<uint64_t>(total, 1) * 4);
    copy_h2d(e->d_offsets.ptr, offsets, (n_traj + 1) * 8, st);
    if (total) {
        copy_h2d(e->d_loc.ptr, events, total * 4, st);
        launch_keys_from_loc(e->d_loc.as<uint32_t>(), total, c->d_loc_key.as<uint32_t>(), e->d_key.as<uint32_t>(), st);
    }
    finish_list(c, e.get(), st);
    *out = e.release();
}

// --------------------------------------------------- success probability ---
struct McOut {
    double mean, pass_frac, sd_mean, sd_pass;
};

static McOut mc_run(arso_circuit *c, const DevCrit &dc, double p, uint64_t n_traj, uint64_t seed, cudaStream_t st) {
    arso_error_list *raw = nullptr;
    sample(c, p / 3, p / 3, p / 3, seed, 0, n_traj, st, &raw);
    std::unique_ptr<arso_error_list> e(raw);
    Scratch sc(st, std::max<uint64_t>(n_traj, 1) * 8), pf(st, std::max<uint64_t>(n_traj, 1));
    Scratch sums(st, 3 * 8);
    run_all(c, e.get(), dc, st, sc.as<double>(), pf.as<uint8_t>());
    launch_sum_scores(sc.as<double>(), pf.as<uint8_t>(), n_traj, sums.as<double>(), st);
    double h[3];
    copy_d2h(h, sums.ptr, 24, st);
    ARSO_CUDA(cudaStreamSynchronize(st));
    McOut o{};
    const double N = (double)std::max<uint64_t>(n_traj, 1);
    o.mean = h[0] / N;
    o.pass_frac = h[2] / N;
    const double var_s = n_traj > 1 ? std::max(0.0, (h[1] - h[0] * h[0] / N) / (N - 1)) : 0.0;
    const double var_p = n_traj > 1 ? std::max(0.0, (h[2] - h[2] * h[2] / N) / (N - 1)) : 0.0;
    o.sd_mean = std::sqrt(var_s / N);
    o.sd_pass = std::sqrt(var_p / N);
    return o;
}

// Probes of one search share (seed, n_traj) and draw the same random numbers:
// a trajectory's error set at p is contained in its set at any p' > p (the
// error test compares one draw with a threshold increasing in p, and with
// p_X = p_Z = p_Y the type cut points do not depend on p). So a trajectory
// with as many events at p as at an earlier probe has exactly that probe's
// events, and its score there is reused; only the others are simulated.
struct ProbeMemo {
    struct Rec {
        double p;
        std::vector<uint32_t> count;
        std::vector<double> score;
        std::vector<uint8_t> pass;
    };
    std::vector<Rec> recs;
    bool enabled = true;
};

static bool memo_supported(const arso_circuit *c) { return c->engine == 1 || c->reg_blocked; }

static McOut mc_run_memo(arso_circuit *c, const DevCrit &dc, double p, uint64_t n_traj, uint64_t seed, cudaStream_t st,
                         ProbeMemo *memo) {
    if (!memo || !memo->enabled || !memo_supported(c) || n_traj == 0) return mc_run(c, dc, p, n_traj, seed, st);
    arso_error_list *raw = nullptr;
    sample(c, p / 3, p / 3, p / 3, seed, 0, n_traj, st, &raw);
    std::unique_ptr<arso_error_list> e(raw);
    ensure_cache(c, st);
    std::vector<uint64_t> off(n_traj + 1);
    copy_d2h(off.data(), e->d_offsets.ptr, (n_traj + 1) * 8, st);
    Scratch ref(st, sizeof(double));
    score_into(ref_state_ptr(c), ref_state_ptr(c), (int)c->n, c->precision, dc.d, ref.as<double>(), st);
    double ref_h = 0.0;
    copy_d2h(&ref_h, ref.ptr, 8, st);
    ARSO_CUDA(cudaStreamSynchronize(st));
    ProbeMemo::Rec rec;
    rec.p = p;
    rec.count.resize(n_traj);
    rec.score.resize(n_traj);
    rec.pass.resize(n_traj);
    // the nearest earlier probes below and above p
    const ProbeMemo::Rec *below = nullptr, *above = nullptr;
    for (const ProbeMemo::Rec &r : memo->recs) {
        if (r.count.size() != n_traj) continue;
        if (r.p <= p && (!below || r.p > below->p)) below = &r;
        if (r.p >= p && (!above || r.p < above->p)) above = &r;
    }
    std::vector<uint64_t> ids;
    for (uint64_t t = 0; t < n_traj; ++t) {
        const uint32_t k = (uint32_t)(off[t + 1] - off[t]);
        rec.count[t] = k;
        const ProbeMemo::Rec *from = nullptr;
        if (k == 0) {
            rec.score[t] = ref_h;
            rec.pass[t] = ref_h >= dc.d.threshold;
            continue;
        }
        if (below && below->count[t] == k) from = below;
        else if (above && above->count[t] == k) from = above;
        if (from) {
            rec.score[t] = from->score[t];
            rec.pass[t] = from->pass[t];
        } else {
            ids.push_back(t);
        }
    }
    if (!ids.empty()) {
        Scratch sc(st, n_traj * 8), pf(st, n_traj);
        if (c->engine == 0) {
            Scratch d_ids(st, ids.size() * 8);
            copy_h2d(d_ids.ptr, ids.data(), ids.size() * 8, st);
            ResidentArgs a = resident_args(c);
            a.first_traj = 0;
            a.count = ids.size();
            a.ids = d_ids.as<uint64_t>();
            a.offsets = e->d_offsets.as<uint64_t>();
            a.keys = e->d_key.as<uint32_t>();
            a.first = e->d_first.as<uint32_t>();
            a.crit = dc.d;
            a.ref_score = ref.as<double>();
            a.score = sc.as<double>();
            a.pass_flags = pf.as<uint8_t>();
            launch_resident_rb(a, 0, (double)ids.size() * c->state_bytes(), st);
        } else {
            std::vector<uint32_t> first(n_traj), last(n_traj), fp, lp;
            copy_d2h(first.data(), e->d_first.ptr, n_traj * 4, st);
            copy_d2h(last.data(), e->d_last.ptr, n_traj * 4, st);
            ARSO_CUDA(cudaStreamSynchronize(st));
            for (uint64_t t : ids) fp.push_back(first[t]), lp.push_back(last[t]);
            if (dc.d.kind == ARSO_CRIT_OUTCOME && suffix_wanted(c, dc.d)) ensure_bwd_cache(c, dc.d.target, st);
            run_streaming(c, e.get(), ids, fp, lp, dc.d, sc.as<double>(), pf.as<uint8_t>(), nullptr, st);
        }
        std::vector<double> sh(n_traj);
        std::vector<uint8_t> ph(n_traj);
        copy_d2h(sh.data(), sc.ptr, n_traj * 8, st);
        copy_d2h(ph.data(), pf.ptr, n_traj, st);
        ARSO_CUDA(cudaStreamSynchronize(st));
        for (uint64_t t : ids) rec.score[t] = sh[t], rec.pass[t] = ph[t];
    }
    double s1 = 0.0, s2 = 0.0, np = 0.0;
    for (uint64_t t = 0; t < n_traj; ++t) {
        s1 += rec.score[t];
        s2 += rec.score[t] * rec.score[t];
        np += rec.pass[t];
    }
    memo->recs.push_back(std::move(rec));
    McOut o{};
    const double N = (double)n_traj;
    o.mean = s1 / N;
    o.pass_frac = np / N;
    const double var_s = n_traj > 1 ? std::max(0.0, (s2 - s1 * s1 / N) / (N - 1)) : 0.0;
    const double var_p = n_traj > 1 ? std::max(0.0, (np - np * np / N) / (N - 1)) : 0.0;
    o.sd_mean = std::sqrt(var_s / N);
    o.sd_pass = std::sqrt(var_p / N);
    return o;
}

// Exhaustive single-error analysis: values per location and per type
// (Eq. (3)); P[4] = {P_R, P_X, P_Z, P_Y} for the given aggregate.
// Fidelity of every single-error state from one error-free sweep: the state
// with error P on qubit q after gate g scores <psi_g|P|psi_g>^2 (the rest of the
// circuit maps psi_g to psi_R). Scores in the exhaustive order (X block, Z
// block, Y block, each in location order). Returns false where the sweep is
// not available (streaming complex128), leaving the trajectory route.
static bool single_error_fidelities(arso_circuit *c, cudaStream_t st, std::vector<double> &s) {
    const uint64_t L = c->L, G = c->gates.size();
    if (c->engine != 0 && c->precision != ARSO_C64) return false;
    std::vector<double> xyz(3 * std::max<uint64_t>(L, 1));
    if (L) {
        std::vector<uint32_t> first(G);
        for (uint64_t l = L; l-- > 0;) first[c->loc_gate[l]] = (uint32_t)l;
        Scratch d_out(st, 3 * L * 8);
        if (c->engine == 0) {
            // one CTA per segment between cached checkpoints (every ckpt_every gates,
            // or phases when register-blocked), all segments in parallel
            ensure_cache(c, st);
            const uint64_t units = c->reg_blocked ? c->ph_R.size() : G;
            std::vector<uint32_t> seg;
            for (uint64_t u = 0; u < units; u += c->ckpt_every)
                seg.push_back(c->reg_blocked ? c->ph_gb[u] : (uint32_t)u);
            seg.push_back((uint32_t)G);
            std::vector<uint32_t> fl(G);
            for (uint64_t pos = 0; pos < G; ++pos) fl[pos] = first[c->perm[pos]];
            Scratch d_fl(st, G * 4), d_seg(st, seg.size() * 4);
            copy_h2d(d_fl.ptr, fl.data(), G * 4, st);
            copy_h2d(d_seg.ptr, seg.data(), seg.size() * 4, st);
            launch_expect_resident(c->d_gates.as<DGate>(), c->d_mats.ptr, (int)c->n, c->precision, c->d_cache.ptr,
                                   d_seg.as<uint32_t>(), (uint32_t)(seg.size() - 1), d_fl.as<uint32_t>(),
                                   d_out.as<double>(), st);
            copy_d2h(xyz.data(), d_out.ptr, 3 * L * 8, st);
            ARSO_CUDA(cudaStreamSynchronize(st));
        } else {
            // complex64 state in HBM: each gate in engine order fused with the expectations
            // of its qubits on the amplitudes it writes; block partials of up to CH gates at a
            // time, then one ordered reduction per chunk
            const int n = (int)c->n;
            const uint32_t blocks = expect_hbm_blocks(n);
            const uint64_t CH = 1024;
            std::vector<uint32_t> loc(G);
            std::vector<uint8_t> ar(G);
            for (uint64_t pos = 0; pos < G; ++pos) {
                loc[pos] = first[c->perm[pos]];
                ar[pos] = (uint8_t)c->gates[c->perm[pos]].arity;
            }
            Scratch psi(st, c->state_bytes()), part(st, CH * blocks * 6 * 8), d_loc(st, G * 4), d_ar(st, G);
            copy_h2d(d_loc.ptr, loc.data(), G * 4, st);
            copy_h2d(d_ar.ptr, ar.data(), G, st);
            launch_init_zero_state(psi.ptr, n, ARSO_C64, st);
            for (uint64_t c0 = 0; c0 < G; c0 += CH) {
                const uint64_t c1 = std::min<uint64_t>(G, c0 + CH);
                for (uint64_t pos = c0; pos < c1; ++pos) {
                    const HostGate &h = c->gates[c->perm[pos]];
                    DGate d{};
                    d.cls = h.cls == GC_H ? (uint8_t)GC_DENSE1
                          : h.cls == GC_OMEGA ? (uint8_t)GC_DIAG1 : h.cls == GC_CZ ? (uint8_t)GC_DIAG2 : h.cls;
                    d.arity = (uint8_t)h.arity;
                    d.q0 = (uint8_t)h.q0;
                    d.q1 = (uint8_t)h.q1;
                    M16 m{};
                    if (h.arity == 1 && d.cls == GC_DIAG1) {
                        m.m[0] = make_float2((float)h.m[0].real(), (float)h.m[0].imag());
                        m.m[1] = make_float2((float)h.m[3].real(), (float)h.m[3].imag());
                    } else if (h.cls != GC_NOP) {
                        for (int i = 0; i < (h.arity == 1 ? 4 : 16); ++i)
                            m.m[i] = make_float2((float)h.m[i].real(), (float)h.m[i].imag());
                    }
                    launch_gate_expect(psi.as<float2>(), n, d, m, part.as<double>() + (pos - c0) * blocks * 6, st);
                }
                launch_gate_expect_reduce(part.as<double>(), (uint32_t)(c1 - c0), blocks, d_loc.as<uint32_t>() + c0,
                                          d_ar.as<uint8_t>() + c0, d_out.as<double>(), st);
            }
            copy_d2h(xyz.data(), d_out.ptr, 3 * L * 8, st);
            ARSO_CUDA(cudaStreamSynchronize(st));
        }
    }
    s.assign(3 * L, 0.0);
    for (uint64_t l = 0; l < L; ++l)
        for (int k = 0; k < 3; ++k) s[k * L + l] = xyz[3 * l + k] * xyz[3 * l + k];  // X, Z, Y blocks
    return true;
}

// Outcome probability of every single-error state from one backward sweep of the
// error-free state and the backward state (both carried from the circuit's end by
// the adjoint gates): the state with P on qubit q after gate g scores
// |<phi_g|P|psi_g>|^2 with phi_g = W^dagger |target> for the rest W of the circuit.
// Same output order as single_error_fidelities. Returns false for streaming
// complex128 circuits (trajectory route).
static bool single_error_outcomes(arso_circuit *c, uint64_t target, cudaStream_t st, std::vector<double> &s) {
    const uint64_t L = c->L, G = c->gates.size();
    if (c->engine != 0 && c->precision != ARSO_C64) return false;
    std::vector<double> v6(6 * std::max<uint64_t>(L, 1), 0.0);
    if (L) {
        ensure_cache(c, st);
        std::vector<uint32_t> first(G);
        for (uint64_t l = L; l-- > 0;) first[c->loc_gate[l]] = (uint32_t)l;
        std::vector<uint32_t> loc(G);
        std::vector<uint8_t> ar(G);
        for (uint64_t pos = 0; pos < G; ++pos) {
            loc[pos] = first[c->perm[pos]];
            ar[pos] = (uint8_t)c->gates[c->perm[pos]].arity;
        }
        Scratch d_out(st, 6 * L * 8), d_loc(st, G * 4);
        copy_h2d(d_loc.ptr, loc.data(), G * 4, st);
        if (c->engine == 0) {
            // adjoint gate table in engine order (global qubits) and its matrix pool
            std::vector<DGate> adj(std::max<uint64_t>(G, 1));
            std::vector<std::complex<double>> pool;
            for (uint64_t pos = 0; pos < G; ++pos) {
                const HostGate &h = c->gates[c->perm[pos]];
                DGate d{};
                d.cls = h.cls;
                d.arity = (uint8_t)h.arity;
                d.q0 = (uint8_t)h.q0;
                d.q1 = (uint8_t)h.q1;
                d.mat = h.cls == GC_OMEGA ? (8u - h.omega_k) & 7u : (uint32_t)pool.size();
                const int dim = h.arity == 1 ? 2 : 4;
                switch (h.cls) {
                    case GC_DENSE1:
                    case GC_DENSE2:
                        for (int r = 0; r < dim; ++r)
                            for (int col = 0; col < dim; ++col) pool.push_back(std::conj(h.m[col * dim + r]));
                        break;
                    case GC_DIAG1: pool.push_back(std::conj(h.m[0])); pool.push_back(std::conj(h.m[3])); break;
                    case GC_DIAG2: for (int i = 0; i < 4; ++i) pool.push_back(std::conj(h.m[5 * i])); break;
                    default: break;  // NOP, X, H, CX, SWAP, CZ are their own adjoints; omega: k -> -k
                }
                adj[pos] = d;
            }
            const size_t esz = c->precision == ARSO_C128 ? 16 : 8;
            Scratch d_adj(st, adj.size() * sizeof(DGate)), d_pool(st, std::max<size_t>(pool.size(), 1) * esz);
            copy_h2d(d_adj.ptr, adj.data(), adj.size() * sizeof(DGate), st);
            if (c->precision == ARSO_C128) {
                std::vector<double2> v(pool.size());
                for (size_t i = 0; i < pool.size(); ++i) v[i] = make_double2(pool[i].real(), pool[i].imag());
                if (!v.empty()) copy_h2d(d_pool.ptr, v.data(), v.size() * esz, st);
            } else {
                std::vector<float2> v(pool.size());
                for (size_t i = 0; i < pool.size(); ++i) v[i] = make_float2((float)pool[i].real(), (float)pool[i].imag());
                if (!v.empty()) copy_h2d(d_pool.ptr, v.data(), v.size() * esz, st);
            }
            launch_dual_expect_resident(d_adj.as<DGate>(), d_pool.ptr, (uint32_t)G, (int)c->n, c->precision,
                                        ref_state_ptr(c), target, d_loc.as<uint32_t>(), d_out.as<double>(), st);
            ARSO_CUDA(cudaStreamSynchronize(st));  // host tables above are freed on return
        } else {
            const int n = (int)c->n;
            const uint32_t blocks = expect_hbm_blocks(n);
            const uint64_t CH = 512;
            Scratch psi(st, c->state_bytes()), phi(st, c->state_bytes()), part(st, CH * blocks * 12 * 8), d_ar(st, G);
            copy_h2d(d_ar.ptr, ar.data(), G, st);
            ARSO_CUDA(cudaMemcpyAsync(psi.ptr, ref_state_ptr(c), c->state_bytes(), cudaMemcpyDeviceToDevice, st));
            const float2 one = make_float2(1.f, 0.f);
            ARSO_CUDA(cudaMemsetAsync(phi.ptr, 0, c->state_bytes(), st));
            copy_h2d(phi.as<float2>() + target, &one, sizeof(float2), st);
            // positions in descending chunks [c0, c1), each walked from c1 - 1 down
            for (uint64_t c1 = G; c1 > 0;) {
                const uint64_t c0 = c1 > CH ? c1 - CH : 0;
                for (uint64_t pos = c1; pos-- > c0;) {
                    DGate d;
                    M16 m;
                    hbm_gate(c->gates[c->perm[pos]], true, d, m);
                    launch_dual_gate_expect(psi.as<float2>(), phi.as<float2>(), n, d, m,
                                            part.as<double>() + (pos - c0) * blocks * 12, st);
                }
                launch_dual_expect_reduce(part.as<double>(), (uint32_t)(c1 - c0), blocks, d_loc.as<uint32_t>() + c0,
                                          d_ar.as<uint8_t>() + c0, d_out.as<double>(), st);
                c1 = c0;
            }
        }
        copy_d2h(v6.data(), d_out.ptr, 6 * L * 8, st);
        ARSO_CUDA(cudaStreamSynchronize(st));
    }
    s.assign(3 * L, 0.0);
    for (uint64_t l = 0; l < L; ++l)
        for (int k = 0; k < 3; ++k) {
            const double re = v6[6 * l + 2 * k], im = v6[6 * l + 2 * k + 1];
            s[k * L + l] = re * re + im * im;  // X, Z, Y blocks
        }
    return true;
}

static void exhaustive_by_trajectories(arso_circuit *c, const DevCrit &dc, cudaStream_t st, std::vector<double> &s,
                                       std::vector<uint8_t> &f);
static void exhaustive_finish(arso_circuit *c, const DevCrit &dc, cudaStream_t st, const std::vector<double> &s,
                              const std::vector<uint8_t> &f, double *P, std::vector<double> *per_loc_mean,
                              std::vector<double> *per_loc_pass, double *P_pass);

static void exhaustive(arso_circuit *c, const DevCrit &dc, cudaStream_t st, double *P, std::vector<double> *per_loc_mean,
                       std::vector<double> *per_loc_pass, double *P_pass) {
    const uint64_t L = c->L;
    const uint64_t T = 3 * L;
    std::vector<double> s(T);
    std::vector<uint8_t> f(T);
    const bool fast = !(c->flags & ARSO_OPT_NO_FAST_EXHAUSTIVE);
    if ((fast && dc.d.kind == ARSO_CRIT_FIDELITY && single_error_fidelities(c, st, s)) ||
        (fast && dc.d.kind == ARSO_CRIT_OUTCOME && single_error_outcomes(c, dc.d.target, st, s))) {
        for (uint64_t i = 0; i < T; ++i) f[i] = s[i] >= dc.d.threshold;
    } else {
        exhaustive_by_trajectories(c, dc, st, s, f);
    }
    exhaustive_finish(c, dc, st, s, f, P, per_loc_mean, per_loc_pass, P_pass);
}

// Every single-error state simulated as a trajectory with one event.
static void exhaustive_by_trajectories(arso_circuit *c, const DevCrit &dc, cudaStream_t st, std::vector<double> &s,
                                       std::vector<uint8_t> &f) {
    const uint64_t L = c->L;
    const uint64_t T = 3 * L;
    std::vector<uint64_t> off(T + 1);
    std::vector<uint32_t> ev(T);
    const uint32_t codes[3] = {1, 2, 3};  // X, Z, Y blocks
    for (uint64_t i = 0; i < T; ++i) {
        off[i] = i;
        ev[i] = (uint32_t)(((i % std::max<uint64_t>(L, 1)) << 2) | codes[i / std::max<uint64_t>(L, 1)]);
    }
    off[T] = T;
    arso_error_list *raw = nullptr;
    list_from_host(c, T, off.data(), ev.data(), st, &raw);
    std::unique_ptr<arso_error_list> e(raw);
    Scratch sc(st, std::max<uint64_t>(T, 1) * 8), pf(st, std::max<uint64_t>(T, 1));
    run_all(c, e.get(), dc, st, sc.as<double>(), pf.as<uint8_t>());
    s.assign(T, 0.0);
    f.assign(T, 0);
    if (T) {
        copy_d2h(s.data(), sc.ptr, T * 8, st);
        copy_d2h(f.data(), pf.ptr, T, st);
    }
    ARSO_CUDA(cudaStreamSynchronize(st));
}

static void exhaustive_finish(arso_circuit *c, const DevCrit &dc, cudaStream_t st, const std::vector<double> &s,
                              const std::vector<uint8_t> &f, double *P, std::vector<double> *per_loc_mean,
                              std::vector<double> *per_loc_pass, double *P_pass) {
    const uint64_t L = c->L;
    const uint64_t T = 3 * L;
    ensure_cache(c, st);
    // reference value
    Scratch ref(st, 8);
    score_into(ref_state_ptr(c), ref_state_ptr(c), (int)c->n, c->precision, dc.d, ref.as<double>(), st);
    double r = 0;
    copy_d2h(&r, ref.ptr, 8, st);
    ARSO_CUDA(cudaStreamSynchronize(st));
    const double rp = r >= dc.d.threshold ? 1.0 : 0.0;
    double Pm[4] = {r, 0, 0, 0}, Pp[4] = {rp, 0, 0, 0};
    for (uint64_t i = 0; i < T; ++i) {
        Pm[1 + i / L] += s[i];
        Pp[1 + i / L] += f[i];
    }
    for (int k = 1; k < 4; ++k) {
        Pm[k] = L ? Pm[k] / (double)L : 0.0;
        Pp[k] = L ? Pp[k] / (double)L : 0.0;
    }
    const double *sel = dc.aggregate == ARSO_AGG_MEAN ? Pm : Pp;
    for (int k = 0; k < 4; ++k) P[k] = sel[k];
    if (P_pass)
        for (int k = 0; k < 4; ++k) P_pass[k] = Pp[k];
    if (per_loc_mean) *per_loc_mean = s;
    if (per_loc_pass) {
        per_loc_pass->resize(T);
        for (uint64_t i = 0; i < T; ++i) (*per_loc_pass)[i] = f[i];
    }
}

// ------------------------------------------------------ persistent batch ---
// Every complex64 circuit of an arso_run_batch call in one launch of mix_kernel
// (kernels.h, MixArgs). The host lists the units in dependency order:
// error-free reference scores first, then the resident items longest first, then
// the streaming units by their level in their working slot's chain of passes.
enum MixKind { MK_NONE = 0, MK_SMALL = 1, MK_RES = 2, MK_STR = 3 };
static MixKind mix_kind(const arso_circuit *c) {
    if (c->precision != ARSO_C64 || (c->flags & ARSO_OPT_NO_PERSISTENT)) return MK_NONE;
    if (c->engine == 0) return c->reg_blocked ? MK_RES : MK_SMALL;
    return c->reg_blocked && c->tile_qubits == 13 ? MK_STR : MK_NONE;
}

constexpr uint64_t MIX_SLOT_BUDGET = 16ull << 30;  // working slots of all streaming circuits of a call

// set by arso_debug_stall_next_batch: no dependency wait of the next persistent launch can be met
static std::atomic<bool> g_stall_next_batch{false};

static void run_mixed(const std::vector<size_t> &sel, arso_circuit *const *circuits,
                      const arso_error_list *const *errors, const std::vector<DevCrit> &dcs,
                      const std::vector<double *> &d_score, const std::vector<uint8_t *> &d_pass, cudaStream_t st) {
    const size_t C = sel.size();
    if (!C) return;
    std::vector<MixKind> kind(C);
    for (size_t q = 0; q < C; ++q) {
        arso_circuit *c = circuits[sel[q]];
        kind[q] = mix_kind(c);
        ensure_cache(c, st);
        if (kind[q] == MK_STR && dcs[sel[q]].d.kind == ARSO_CRIT_OUTCOME && suffix_wanted(c, dcs[sel[q]].d))
            ensure_bwd_cache(c, dcs[sel[q]].d.target, st);
    }
    // first (and, streaming, last) event positions of every trajectory: all copies, one synchronisation
    std::vector<std::vector<uint32_t>> first(C), last(C);
    for (size_t q = 0; q < C; ++q) {
        const arso_error_list *e = errors[sel[q]];
        if (!e->n_traj) continue;
        first[q].resize(e->n_traj);
        copy_d2h(first[q].data(), e->d_first.ptr, e->n_traj * 4, st);
        if (kind[q] == MK_STR) {
            last[q].resize(e->n_traj);
            copy_d2h(last[q].data(), e->d_last.ptr, e->n_traj * 4, st);
        }
    }
    ARSO_CUDA(cudaStreamSynchronize(st));

    std::vector<MixRef> refs;
    std::vector<MixSmall> smalls;
    std::vector<BatchCircuit> rcircs;
    std::vector<BatchItem> items;
    std::vector<uint64_t> ids;
    std::vector<MixStream> streams;
    std::vector<MixPass> spasses;
    std::vector<MixTraj> strajs;
    std::vector<uint32_t> scslot;
    struct Res { uint32_t item; uint64_t cost; bool small; };
    std::vector<Res> res_units;
    struct Str { uint32_t stream, k, j, level; };
    std::vector<Str> str_units;
    // counters (zeroed): ref chunks done, then per stream slot and trajectory counters
    uint64_t n_counters = 0, n_partials = 0, work_bytes = 0;
    std::vector<uint64_t> ref_part_off, ref_ctr_off, st_slot_off, st_traj_off, st_part_off, st_work_off, st_pass_off,
        st_traj_tab_off, st_cslot_off;
    double bytes = 0.0, flops = 0.0, smem = 0.0;

    // pass 1: streaming slot counts (the slot budget split by each circuit's work)
    std::vector<std::vector<uint64_t>> sid(C);
    std::vector<std::vector<int>> sstart(C), send(C);
    std::vector<double> swork(C, 0.0);
    double work_total = 0.0;
    for (size_t q = 0; q < C; ++q) {
        if (kind[q] != MK_STR) continue;
        arso_circuit *c = circuits[sel[q]];
        const uint32_t P = (uint32_t)c->passes.size();
        const bool suffix = suffix_wanted(c, dcs[sel[q]].d);
        for (uint64_t t = 0; t < first[q].size(); ++t) {
            if (first[q][t] == NO_EVENT) continue;
            uint32_t fp = c->pass_of_pos[first[q][t]];
            while (c->ckpt_pass[fp] == NO_EVENT) --fp;
            uint32_t lp = P - 1;
            if (suffix) {
                lp = c->pass_of_pos[last[q][t]];
                while (c->ckpt_pass[lp + 1] == NO_EVENT) ++lp;
            }
            sid[q].push_back(t);
            sstart[q].push_back((int)fp);
            send[q].push_back((int)lp);
            swork[q] += (double)(lp - fp + 1) * (double)c->state_bytes();
        }
        work_total += swork[q];
    }
    for (size_t q = 0; q < C; ++q) {
        arso_circuit *c = circuits[sel[q]];
        const arso_error_list *e = errors[sel[q]];
        const DevCrit &dc = dcs[sel[q]];
        const uint64_t N = 1ull << c->n;
        // the circuit's error-free score, filled into its error-free trajectories
        MixRef r{};
        r.n = (int)c->n;
        r.chunks = (uint32_t)((N + 8191) >> 13);
        r.psi_R = static_cast<const float2 *>(ref_state_ptr(c));
        r.crit = dc.d;
        r.first = e->d_first.as<uint32_t>();
        r.n_traj = e->n_traj;
        r.score = d_score[sel[q]];
        r.pass_flags = d_pass[sel[q]];
        ref_part_off.push_back(n_partials);
        n_partials += r.chunks;
        ref_ctr_off.push_back(n_counters);
        n_counters += 1;
        refs.push_back(r);
        bytes += (double)c->state_bytes();
        if (kind[q] == MK_SMALL || kind[q] == MK_RES) {
            const bool small = kind[q] == MK_SMALL;
            std::vector<std::pair<uint32_t, uint64_t>> todo;  // (checkpoint, trajectory)
            for (uint64_t t = 0; t < first[q].size(); ++t)
                if (first[q][t] != NO_EVENT)
                    todo.emplace_back((small ? first[q][t] : c->phase_of_pos[first[q][t]]) / (uint32_t)c->ckpt_every, t);
            std::sort(todo.begin(), todo.end());
            const uint32_t per = small ? std::min<uint32_t>(MIX_SMALL_MAX, 1u << (13 - c->n)) : 1u << (13 - c->n);
            const uint32_t desc = small ? (uint32_t)smalls.size() : (uint32_t)rcircs.size();
            const uint64_t G = c->gates.size();
            for (size_t k = 0; k < todo.size(); k += per) {
                BatchItem it{};
                it.circuit = desc;
                it.count = (uint32_t)std::min<size_t>(per, todo.size() - k);
                it.ck = todo[k].first;
                it.off = ids.size();
                for (size_t u = 0; u < it.count; ++u) ids.push_back(todo[k + u].second);
                const uint64_t g0 = small ? std::min<uint64_t>(G, (uint64_t)it.ck * c->ckpt_every)
                                          : c->ph_gb[std::min<uint64_t>(c->ph_R.size(), (uint64_t)it.ck * c->ckpt_every)];
                res_units.push_back({(uint32_t)items.size(), G - g0, small});
                items.push_back(it);
                bytes += (double)it.count * 2.0 * c->state_bytes();
                const double amps = (double)it.count * (double)N;
                flops += (c->flops_prefix[G] - c->flops_prefix[g0]) * amps;
                if (small) {
                    smem += (double)(G - g0) * 16.0 * amps;  // the gate engine reads and writes the state per gate
                } else {
                    const uint32_t nph = (uint32_t)c->ph_R.size(), ph0 = std::min<uint32_t>(nph, it.ck * (uint32_t)c->ckpt_every);
                    if (ph0 < nph) {
                        const uint32_t n = c->n;
                        const uint32_t load_packed = 0u | ((n - 4) << 5) | ((n - 3) << 10) | ((n - 2) << 15) | ((n - 1) << 20);
                        const uint32_t remaps = (c->ph_R[ph0] != load_packed) + c->chg_prefix[nph] - c->chg_prefix[ph0 + 1];
                        smem += (double)remaps * 16.0 * amps;
                    }
                }
            }
            if (small) {
                MixSmall m{};
                m.n = (int)c->n;
                m.G = (uint32_t)G;
                m.ckpt_every = (uint32_t)c->ckpt_every;
                m.n_ckpt = c->n_ckpt;
                m.gates = c->d_gates.as<DGate>();
                m.mats = c->d_mats.as<float2>();
                m.cache = c->d_cache.as<float2>();
                m.offsets = e->d_offsets.as<uint64_t>();
                m.keys = e->d_key.as<uint32_t>();
                m.crit = dc.d;
                m.score = d_score[sel[q]];
                m.pass_flags = d_pass[sel[q]];
                smalls.push_back(m);
            } else {
                BatchCircuit b{};
                b.n = (int)c->n;
                b.n_phases = (uint32_t)c->ph_R.size();
                b.n_ckpt = c->n_ckpt;
                b.ckpt_every = (uint32_t)c->ckpt_every;
                b.gates = c->d_gates.as<DGate>();
                b.mats = c->d_mats.as<float2>();
                b.ph_gb = c->d_ph_gb.as<uint32_t>();
                b.ph_R = c->d_ph_R.as<uint32_t>();
                b.phase_of_pos = c->d_phase_of_pos.as<uint32_t>();
                b.rops = c->d_rops.as<RegOp>();
                b.cache = c->d_cache.as<float2>();
                b.offsets = e->d_offsets.as<uint64_t>();
                b.keys = e->d_key.as<uint32_t>();
                b.crit = dc.d;
                b.score = d_score[sel[q]];
                b.pass_flags = d_pass[sel[q]];
                rcircs.push_back(b);
            }
            continue;
        }
        // streaming: trajectories sorted by (start, end), dealt round robin to slots; each
        // slot runs its trajectories one after another
        const uint32_t P = (uint32_t)c->passes.size();
        const size_t sb = c->state_bytes();
        const uint64_t T = sid[q].size();
        const uint32_t tiles = 1u << (c->n - c->tile_qubits);
        const bool overlap = dc.d.kind == ARSO_CRIT_OUTCOME && suffix_wanted(c, dc.d);
        uint64_t S = 1;
        if (T) {
            const double share = work_total > 0 ? swork[q] / work_total : 1.0;
            S = std::max<uint64_t>(1, std::min<uint64_t>(T, (uint64_t)(share * (double)MIX_SLOT_BUDGET / (double)sb)));
        }
        std::vector<size_t> order(T);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
            return sstart[q][x] != sstart[q][y] ? sstart[q][x] < sstart[q][y] : send[q][x] < send[q][y];
        });
        const uint32_t si = (uint32_t)streams.size();
        std::vector<uint32_t> slot_level(S, 0), slot_base(S, 0);
        const uint64_t traj0 = strajs.size();
        for (uint64_t k = 0; k < T; ++k) {
            const size_t o = order[k];
            const uint32_t slot = (uint32_t)(k % S);
            MixTraj mt{};
            mt.tr = sid[q][o];
            mt.slot = slot;
            mt.base = slot_base[slot];
            mt.start = sstart[q][o];
            mt.end = send[q][o];
            const uint32_t len = (uint32_t)(mt.end - mt.start + 1);
            ARSO_REQUIRE((uint64_t)slot_base[slot] + (uint64_t)len * tiles < (1ull << 32), "persistent batch: slot chain too long");
            for (uint32_t j = (uint32_t)mt.start; j <= (uint32_t)mt.end; ++j) {
                str_units.push_back({si, (uint32_t)k, j, slot_level[slot] + (j - (uint32_t)mt.start)});
                bytes += 2.0 * (double)sb;
                flops += c->passes[j].flops_per_amp * (double)N;
                smem += (double)(c->passes[j].remaps + ((int)j != mt.end ? c->passes[j].end_remap : 0u)) * 16.0 * (double)N;
            }
            slot_level[slot] += len;
            slot_base[slot] += len * tiles;
            strajs.push_back(mt);
        }
        MixStream ms{};
        ms.n = (int)c->n;
        ms.t = (int)c->tile_qubits;
        ms.c = (int)c->low_qubits;
        ms.tiles = tiles;
        ms.ph_gb = c->d_ph_gb.as<uint32_t>();
        ms.ph_R = c->d_ph_R.as<uint32_t>();
        ms.rops = c->d_rops.as<RegOp>();
        ms.mats = c->d_mats.as<float2>();
        ms.cache = c->d_cache.as<float2>();
        ms.ref_cache = overlap ? c->d_bwd.as<float2>() : c->d_cache.as<float2>();
        ms.offsets = e->d_offsets.as<uint64_t>();
        ms.keys = e->d_key.as<uint32_t>();
        ms.crit = dc.d;
        if (overlap) ms.crit.kind = ARSO_CRIT_FIDELITY;  // |<t|W a>| = |<W^dagger t|a>|
        ms.score = d_score[sel[q]];
        ms.pass_flags = d_pass[sel[q]];
        st_pass_off.push_back(spasses.size());
        for (uint32_t j = 0; j < P; ++j) {
            MixPass mp{};
            uint64_t tm = 0;
            for (uint32_t qq : c->passes[j].tile_qubits) tm |= 1ull << qq;
            mp.rest_mask = ((1ull << c->n) - 1) & ~tm;
            mp.offs = c->d_offs.as<uint32_t>() + c->offs_base[j];
            mp.gb = c->passes[j].gb;
            mp.pb = c->passes[j].pb;
            mp.pe = c->passes[j].pe;
            spasses.push_back(mp);
        }
        st_cslot_off.push_back(scslot.size());
        scslot.insert(scslot.end(), c->ckpt_pass.begin(), c->ckpt_pass.end());
        st_traj_tab_off.push_back(traj0);
        st_slot_off.push_back(n_counters);
        n_counters += S;
        st_traj_off.push_back(n_counters);
        n_counters += T;
        st_part_off.push_back(n_partials);
        n_partials += T * tiles;
        st_work_off.push_back(work_bytes);
        work_bytes += S * sb;
        streams.push_back(ms);
    }
    // the unit list: references, resident items longest first, streaming units by level
    std::stable_sort(res_units.begin(), res_units.end(), [](const Res &x, const Res &y) { return x.cost > y.cost; });
    std::stable_sort(str_units.begin(), str_units.end(), [](const Str &x, const Str &y) { return x.level < y.level; });
    std::vector<MixUnit> units;
    std::vector<uint64_t> unit_end;
    uint64_t total = 0;
    for (size_t q = 0; q < refs.size(); ++q) {
        units.push_back({MIX_REF, (uint32_t)q, 0, 0});
        unit_end.push_back(total += refs[q].chunks);
    }
    for (const Res &r : res_units) {
        units.push_back({r.small ? (uint32_t)MIX_SMALL : (uint32_t)MIX_RES, r.item, 0, 0});
        unit_end.push_back(total += 1);
    }
    ARSO_REQUIRE(units.size() + str_units.size() < (1ull << 32), "persistent batch: too many units");
    for (const Str &x : str_units) {
        units.push_back({MIX_STR, x.stream, x.k, x.j});
        unit_end.push_back(total += streams[x.stream].tiles);
    }
    if (!total) return;

    // device tables; descriptors point into the shared buffers
    Scratch d_units(st, units.size() * sizeof(MixUnit)), d_end(st, unit_end.size() * 8);
    Scratch d_refs(st, std::max<size_t>(refs.size(), 1) * sizeof(MixRef));
    Scratch d_smalls(st, std::max<size_t>(smalls.size(), 1) * sizeof(MixSmall));
    Scratch d_rcircs(st, std::max<size_t>(rcircs.size(), 1) * sizeof(BatchCircuit));
    Scratch d_items(st, std::max<size_t>(items.size(), 1) * sizeof(BatchItem));
    Scratch d_ids(st, std::max<size_t>(ids.size(), 1) * 8);
    Scratch d_streams(st, std::max<size_t>(streams.size(), 1) * sizeof(MixStream));
    Scratch d_passes(st, std::max<size_t>(spasses.size(), 1) * sizeof(MixPass));
    Scratch d_trajs(st, std::max<size_t>(strajs.size(), 1) * sizeof(MixTraj));
    Scratch d_cslot(st, std::max<size_t>(scslot.size(), 1) * 4);
    Scratch d_parts(st, std::max<uint64_t>(n_partials, 1) * sizeof(Partial));
    Scratch d_ctr(st, std::max<uint64_t>(n_counters, 1) * 4);
    Scratch d_work(st, work_bytes);
    Scratch d_qc(st, 16);  // queue counter (8 bytes) and error word
    for (size_t q = 0; q < refs.size(); ++q) {
        refs[q].partials = d_parts.as<Partial>() + ref_part_off[q];
        refs[q].done = d_ctr.as<uint32_t>() + ref_ctr_off[q];
    }
    for (size_t q = 0; q < streams.size(); ++q) {
        MixStream &ms = streams[q];
        ms.passes = d_passes.as<MixPass>() + st_pass_off[q];
        ms.cache_slot = d_cslot.as<uint32_t>() + st_cslot_off[q];
        ms.trajs = d_trajs.as<MixTraj>() + st_traj_tab_off[q];
        ms.slot_done = d_ctr.as<uint32_t>() + st_slot_off[q];
        ms.traj_done = d_ctr.as<uint32_t>() + st_traj_off[q];
        ms.partials = d_parts.as<Partial>() + st_part_off[q];
        ms.work = reinterpret_cast<float2 *>(d_work.as<char>() + st_work_off[q]);
    }
    auto up = [&](Scratch &d, const void *src, size_t b) {
        if (b) copy_h2d(d.ptr, src, b, st);
    };
    up(d_units, units.data(), units.size() * sizeof(MixUnit));
    up(d_end, unit_end.data(), unit_end.size() * 8);
    up(d_refs, refs.data(), refs.size() * sizeof(MixRef));
    up(d_smalls, smalls.data(), smalls.size() * sizeof(MixSmall));
    up(d_rcircs, rcircs.data(), rcircs.size() * sizeof(BatchCircuit));
    up(d_items, items.data(), items.size() * sizeof(BatchItem));
    up(d_ids, ids.data(), ids.size() * 8);
    up(d_streams, streams.data(), streams.size() * sizeof(MixStream));
    up(d_passes, spasses.data(), spasses.size() * sizeof(MixPass));
    up(d_trajs, strajs.data(), strajs.size() * sizeof(MixTraj));
    up(d_cslot, scslot.data(), scslot.size() * 4);
    ARSO_CUDA(cudaMemsetAsync(d_ctr.ptr, 0, std::max<uint64_t>(n_counters, 1) * 4, st));
    ARSO_CUDA(cudaMemsetAsync(d_qc.ptr, 0, 16, st));
    MixArgs a{};
    a.units = d_units.as<MixUnit>();
    a.unit_end = d_end.as<uint64_t>();
    a.n_units = (uint32_t)units.size();
    a.n_sub = total;
    a.refs = d_refs.as<MixRef>();
    a.smalls = d_smalls.as<MixSmall>();
    a.rcircs = d_rcircs.as<BatchCircuit>();
    a.items = d_items.as<BatchItem>();
    a.ids = d_ids.as<uint64_t>();
    a.streams = d_streams.as<MixStream>();
    a.counter = d_qc.as<unsigned long long>();
    a.err = reinterpret_cast<uint32_t *>(d_qc.as<char>() + 8);
    a.wait_limit = 1u << 22;
    if (g_stall_next_batch.exchange(false)) {  // arso_debug_stall_next_batch: no wait can be met
        a.stall_extra = 1u << 30;
        a.wait_limit = 1u << 12;
    }
    launch_mix(a, bytes, flops, smem, st);
    uint32_t err = 0;
    copy_d2h(&err, a.err, 4, st);
    ARSO_CUDA(cudaStreamSynchronize(st));  // also keeps the host tables alive until the launch is done
    if (err) throw Error(ARSO_ETIMEOUT, "persistent batch: a dependency wait gave up");
}

// Eq. (4) with E(N_e) = L p_e
static double eq4(const double *P, uint64_t L, double pe) {
    const double E = (double)L * pe;
    return (P[1] + P[2] + P[3]) * E + P[0] * (1.0 - 3.0 * E);
}

}  // namespace arso

using namespace arso;

// ================================================================ C ABI ====
extern "C" {

const char *arso_last_error(void) { return g_last_error.c_str(); }
const char *arso_version(void) { return "arso-gb300 0.1 (sm_103a)"; }

arso_status arso_compile_circuit(uint32_t n_qubits, const arso_gate *gates, size_t n_gates,
                                 const arso_compile_opts *opts, arso_circuit **out) {
    return guard([&] {
        ARSO_REQUIRE(out != nullptr, "out is NULL");
        *out = nullptr;
        std::unique_ptr<arso_circuit> c(new arso_circuit());
        build_circuit(c.get(), n_qubits, gates, n_gates, opts);
        upload_circuit(c.get());
        *out = c.release();
    });
}

void arso_circuit_free(arso_circuit *c) { delete c; }

arso_status arso_plan_phases(uint32_t n_qubits, const arso_gate *gates, size_t n_gates,
                             const arso_compile_opts *opts, uint32_t *n_phases, uint32_t *n_tensor) {
    return guard([&] {
        ARSO_REQUIRE(n_phases != nullptr, "n_phases is NULL");
        arso_circuit c;
        build_circuit(&c, n_qubits, gates, n_gates, opts);
        *n_phases = c.reg_blocked ? (uint32_t)c.ph_R.size() : 0u;
        if (n_tensor) {
            *n_tensor = 0;
            for (uint32_t t : c.ph_t) *n_tensor += t != NO_TENSOR;
        }
    });
}

arso_status arso_plan_tensor_phase(uint32_t n_qubits, const arso_gate *gates, size_t n_gates,
                                   const arso_compile_opts *opts, uint32_t phase, uint32_t *reg_bits,
                                   uint32_t *pos_begin, uint32_t *pos_end, uint32_t *pass, uint8_t *roles,
                                   uint32_t roles_capacity, uint16_t *image, uint32_t *has_image) {
    return guard([&] {
        ARSO_REQUIRE(reg_bits && pos_begin && pos_end && pass && has_image, "NULL argument");
        arso_circuit c;
        build_circuit(&c, n_qubits, gates, n_gates, opts);
        ARSO_REQUIRE(c.reg_blocked && phase < c.ph_R.size(), "phase out of range");
        *reg_bits = c.ph_R[phase];
        *pos_begin = c.ph_gb[phase];
        *pos_end = c.ph_gb[phase + 1];
        *pass = c.pass_of_pos.empty() ? 0u : c.pass_of_pos[c.ph_gb[phase]];
        if (roles) {
            ARSO_REQUIRE(*pos_end - *pos_begin <= roles_capacity, "roles_capacity too small");
            for (uint32_t p = *pos_begin; p < *pos_end; ++p) roles[p - *pos_begin] = c.role[p];
        }
        const uint32_t t = phase < c.ph_t.size() ? c.ph_t[phase] : NO_TENSOR;
        *has_image = t != NO_TENSOR;
        if (image && t != NO_TENSOR)
            std::copy(c.tmats.begin() + (size_t)t * TENSOR_IMAGE_HALVES,
                      c.tmats.begin() + (size_t)(t + 1) * TENSOR_IMAGE_HALVES, image);
    });
}

arso_status arso_plan_schedule(uint32_t n_qubits, const arso_gate *gates, size_t n_gates,
                               const arso_compile_opts *opts, uint32_t *n_passes, uint32_t capacity, uint32_t *perm,
                               uint32_t *pass_begin, uint64_t *tile_mask) {
    return guard([&] {
        ARSO_REQUIRE(n_passes != nullptr, "n_passes is NULL");
        arso_circuit c;
        build_circuit(&c, n_qubits, gates, n_gates, opts);
        const uint32_t P = (uint32_t)c.passes.size();
        *n_passes = P;
        if (!perm && !pass_begin && !tile_mask) return;
        ARSO_REQUIRE(P <= capacity, "capacity too small for the schedule");
        if (perm) std::copy(c.perm.begin(), c.perm.end(), perm);
        for (uint32_t p = 0; p < P; ++p) {
            if (pass_begin) pass_begin[p] = c.passes[p].gb;
            if (tile_mask) {
                uint64_t m = 0;
                for (uint32_t q : c.passes[p].tile_qubits) m |= 1ull << q;
                tile_mask[p] = m;
            }
        }
        if (pass_begin) pass_begin[P] = P ? c.passes[P - 1].ge : 0;
    });
}

arso_status arso_circuit_get_info(const arso_circuit *c, arso_circuit_info *out) {
    return guard([&] {
        ARSO_REQUIRE(c && out, "NULL argument");
        out->n_qubits = c->n;
        out->G = c->gates.size();
        out->k = c->k;
        out->m = c->m;
        out->L = c->L;
        out->engine = (uint32_t)c->engine;
        out->n_passes = (uint32_t)c->passes.size();
        out->tile_qubits = c->tile_qubits;
        out->precision = (uint32_t)c->precision;
        out->checkpoint_every = c->ckpt_every;
        out->n_phases = c->reg_blocked ? (uint32_t)c->ph_R.size() : 0u;
        out->tensor_phases = 0;
        for (uint32_t t : c->ph_t) out->tensor_phases += t != NO_TENSOR;
    });
}

arso_status arso_sample_errors(const arso_circuit *c, double p_x, double p_z, double p_y, uint64_t seed,
                               uint64_t traj_begin, uint64_t n_traj, void *stream, arso_error_list **out) {
    return guard([&] {
        ARSO_REQUIRE(c && out, "NULL argument");
        *out = nullptr;
        sample(c, p_x, p_z, p_y, seed, traj_begin, n_traj, (cudaStream_t)stream, out);
    });
}

arso_status arso_sample_errors_batch(size_t count, const arso_circuit *const *circuits, const double *p_x,
                                     const double *p_z, const double *p_y, const uint64_t *seeds,
                                     const uint64_t *traj_begin, const uint64_t *n_traj, void *stream,
                                     arso_error_list **out) {
    return guard([&] {
        ARSO_REQUIRE(count == 0 || (circuits && p_x && p_z && p_y && seeds && traj_begin && n_traj && out),
                     "NULL argument");
        for (size_t i = 0; i < count; ++i) out[i] = nullptr;
        sample_batch(count, circuits, p_x, p_z, p_y, seeds, traj_begin, n_traj, (cudaStream_t)stream, out);
    });
}

arso_status arso_error_list_from_host(const arso_circuit *c, uint64_t n_traj, const uint64_t *offsets,
                                      const uint32_t *events, void *stream, arso_error_list **out) {
    return guard([&] {
        ARSO_REQUIRE(c && out, "NULL argument");
        *out = nullptr;
        list_from_host(c, n_traj, offsets, events, (cudaStream_t)stream, out);
    });
}

arso_status arso_error_list_info(const arso_error_list *e, uint64_t *n_traj, uint64_t *n_events) {
    return guard([&] {
        ARSO_REQUIRE(e != nullptr, "NULL error list");
        if (n_traj) *n_traj = e->n_traj;
        if (n_events) *n_events = e->n_events;
    });
}

arso_status arso_error_list_copy(const arso_error_list *e, uint64_t *offsets, uint32_t *events, void *stream) {
    return guard([&] {
        ARSO_REQUIRE(e != nullptr, "NULL error list");
        cudaStream_t st = (cudaStream_t)stream;
        if (offsets)
            copy_d2h(offsets, e->d_offsets.ptr, (e->n_traj + 1) * 8, st);
        if (events && e->n_events)
            copy_d2h(events, e->d_loc.ptr, e->n_events * 4, st);
        ARSO_CUDA(cudaStreamSynchronize(st));
    });
}

void arso_error_list_free(arso_error_list *e) { delete e; }

arso_status arso_run_trajectories(const arso_circuit *cc, const arso_error_list *e, const arso_criterion *crit,
                                  void *stream, double *score_out, uint8_t *pass_out) {
    return guard([&] {
        ARSO_REQUIRE(cc && e && crit && score_out, "NULL argument");
        ARSO_REQUIRE(e->circ == cc, "error list belongs to another circuit");
        arso_circuit *c = const_cast<arso_circuit *>(cc);
        cudaStream_t st = (cudaStream_t)stream;
        DevCrit dc;
        make_crit(c, crit, dc, st);
        const bool sdev = is_device_ptr(score_out), pdev = pass_out && is_device_ptr(pass_out);
        Scratch sc(st, sdev ? 0 : std::max<uint64_t>(e->n_traj, 1) * 8);
        Scratch pf(st, (pass_out && !pdev) ? std::max<uint64_t>(e->n_traj, 1) : 0);
        double *d_score = sdev ? score_out : sc.as<double>();
        uint8_t *d_pass = pass_out ? (pdev ? pass_out : pf.as<uint8_t>()) : nullptr;
        run_all(c, e, dc, st, d_score, d_pass);
        if (!sdev && e->n_traj)
            copy_d2h(score_out, d_score, e->n_traj * 8, st);
        if (pass_out && !pdev && e->n_traj)
            copy_d2h(pass_out, d_pass, e->n_traj, st);
        ARSO_CUDA(cudaStreamSynchronize(st));
    });
}

arso_status arso_aggregate(const double *score, const uint8_t *pass_flags, uint64_t n, void *stream, double *out) {
    return guard([&] {
        ARSO_REQUIRE(score && out, "NULL argument");
        ARSO_REQUIRE(is_device_ptr(score) && (!pass_flags || is_device_ptr(pass_flags)), "inputs must be device memory");
        cudaStream_t st = (cudaStream_t)stream;
        Scratch sums(st, 24);
        launch_sum_scores(score, pass_flags, n, sums.as<double>(), st);
        double h[3];
        copy_d2h(h, sums.ptr, 24, st);
        ARSO_CUDA(cudaStreamSynchronize(st));
        const double N = (double)std::max<uint64_t>(n, 1);
        const double vs = n > 1 ? std::max(0.0, (h[1] - h[0] * h[0] / N) / (N - 1)) : 0.0;
        const double vp = n > 1 ? std::max(0.0, (h[2] - h[2] * h[2] / N) / (N - 1)) : 0.0;
        out[0] = h[0] / N;
        out[1] = h[2] / N;
        out[2] = std::sqrt(vs / N);
        out[3] = std::sqrt(vp / N);
        out[4] = (double)n;
    });
}

arso_status arso_debug_stall_next_batch(void) {
    g_stall_next_batch.store(true);
    return ARSO_OK;
}

arso_status arso_run_batch(size_t count, arso_circuit *const *circuits, const arso_error_list *const *errors,
                           const arso_criterion *crits, void *stream, double *const *score_out,
                           uint8_t *const *pass_out) {
    return guard([&] {
        ARSO_REQUIRE(count == 0 || (circuits && errors && crits && score_out), "NULL argument");
        cudaStream_t st = (cudaStream_t)stream;
        std::vector<DevCrit> dcs(count);
        std::vector<std::unique_ptr<Scratch>> tmp;
        std::vector<double *> d_score(count);
        std::vector<uint8_t *> d_pass(count);
        for (size_t i = 0; i < count; ++i) {
            arso_circuit *c = circuits[i];
            const arso_error_list *e = errors[i];
            ARSO_REQUIRE(c && e && score_out[i], "NULL circuit, error list or output");
            ARSO_REQUIRE(e->circ == c, "error list belongs to another circuit");
            make_crit(c, &crits[i], dcs[i], st);
            ensure_cache(c, st);
            const uint64_t T = std::max<uint64_t>(e->n_traj, 1);
            if (is_device_ptr(score_out[i])) {
                d_score[i] = score_out[i];
            } else {
                tmp.emplace_back(new Scratch(st, T * 8));
                d_score[i] = tmp.back()->as<double>();
            }
            uint8_t *po = pass_out ? pass_out[i] : nullptr;
            if (po && is_device_ptr(po)) {
                d_pass[i] = po;
            } else if (po) {
                tmp.emplace_back(new Scratch(st, T));
                d_pass[i] = tmp.back()->as<uint8_t>();
            } else {
                d_pass[i] = nullptr;
            }
        }
        // every complex64 circuit in one persistent launch; circuits that opt out run
        // the earlier route (register-blocked resident circuits in one batched resident
        // launch, the others on their own launches)
        std::vector<size_t> mixed, group;
        for (size_t i = 0; i < count; ++i) {
            if (mix_kind(circuits[i]) != MK_NONE) mixed.push_back(i);
            else if (circuits[i]->engine == 0 && circuits[i]->reg_blocked) group.push_back(i);
            else run_all(circuits[i], errors[i], dcs[i], st, d_score[i], d_pass[i]);
        }
        run_mixed(mixed, circuits, errors, dcs, d_score, d_pass, st);
        if (!group.empty()) {
            Scratch refs(st, group.size() * 8);
            std::vector<BatchCircuit> descs(group.size());
            std::vector<BatchItem> items;
            std::vector<uint64_t> ids;
            double bytes = 0;
            for (size_t gi = 0; gi < group.size(); ++gi) {
                const size_t i = group[gi];
                arso_circuit *c = circuits[i];
                const arso_error_list *e = errors[i];
                double *ref = refs.as<double>() + gi;
                score_into(ref_state_ptr(c), ref_state_ptr(c), (int)c->n, c->precision, dcs[i].d, ref, st);
                launch_fill_error_free(e->d_first.as<uint32_t>(), e->n_traj, ref, dcs[i].d.threshold, d_score[i],
                                       d_pass[i], st);
                BatchCircuit &b = descs[gi];
                b.n = (int)c->n;
                b.n_phases = (uint32_t)c->ph_R.size();
                b.n_ckpt = c->n_ckpt;
                b.ckpt_every = (uint32_t)c->ckpt_every;
                b.gates = c->d_gates.as<DGate>();
                b.mats = c->d_mats.as<float2>();
                b.ph_gb = c->d_ph_gb.as<uint32_t>();
                b.ph_R = c->d_ph_R.as<uint32_t>();
                b.phase_of_pos = c->d_phase_of_pos.as<uint32_t>();
                b.rops = c->d_rops.as<RegOp>();
                b.cache = c->d_cache.as<float2>();
                b.offsets = e->d_offsets.as<uint64_t>();
                b.keys = e->d_key.as<uint32_t>();
                b.crit = dcs[i].d;
                b.score = d_score[i];
                b.pass_flags = d_pass[i];
                if (!e->n_traj) continue;
                std::vector<uint32_t> first(e->n_traj);
                copy_d2h(first.data(), e->d_first.ptr, e->n_traj * 4, st);
                ARSO_CUDA(cudaStreamSynchronize(st));
                std::vector<std::pair<uint32_t, uint64_t>> todo;  // (checkpoint, trajectory)
                for (uint64_t t = 0; t < e->n_traj; ++t)
                    if (first[t] != NO_EVENT) todo.emplace_back(c->phase_of_pos[first[t]] / (uint32_t)c->ckpt_every, t);
                std::sort(todo.begin(), todo.end());
                const uint32_t per_cta = 1u << (13 - c->n);
                for (size_t k = 0; k < todo.size(); k += per_cta) {
                    BatchItem it{};
                    it.circuit = (uint32_t)gi;
                    it.count = (uint32_t)std::min<size_t>(per_cta, todo.size() - k);
                    it.ck = todo[k].first;
                    it.off = ids.size();
                    for (size_t q = 0; q < it.count; ++q) ids.push_back(todo[k + q].second);
                    items.push_back(it);
                    bytes += (double)it.count * 2.0 * c->state_bytes();
                }
            }
            // longest items first (remaining phases), so the queue drains evenly
            std::stable_sort(items.begin(), items.end(), [&](const BatchItem &x, const BatchItem &y) {
                const BatchCircuit &a = descs[x.circuit], &b = descs[y.circuit];
                return (uint64_t)(a.n_phases - x.ck * a.ckpt_every) > (uint64_t)(b.n_phases - y.ck * b.ckpt_every);
            });
            if (!items.empty()) {
                Scratch d_descs(st, descs.size() * sizeof(BatchCircuit)), d_items(st, items.size() * sizeof(BatchItem));
                Scratch d_ids(st, ids.size() * 8), d_counter(st, 4);
                copy_h2d(d_descs.ptr, descs.data(), descs.size() * sizeof(BatchCircuit), st);
                copy_h2d(d_items.ptr, items.data(), items.size() * sizeof(BatchItem), st);
                copy_h2d(d_ids.ptr, ids.data(), ids.size() * 8, st);
                ARSO_CUDA(cudaMemsetAsync(d_counter.ptr, 0, 4, st));
                launch_batch_resident(d_descs.as<BatchCircuit>(), d_items.as<BatchItem>(), (uint32_t)items.size(),
                                      d_counter.as<uint32_t>(), d_ids.as<uint64_t>(), bytes, st);
                ARSO_CUDA(cudaStreamSynchronize(st));
            }
        }
        for (size_t i = 0; i < count; ++i) {
            const uint64_t T = errors[i]->n_traj;
            if (!T) continue;
            if (d_score[i] != score_out[i]) copy_d2h(score_out[i], d_score[i], T * 8, st);
            if (pass_out && pass_out[i] && d_pass[i] != pass_out[i]) copy_d2h(pass_out[i], d_pass[i], T, st);
        }
        ARSO_CUDA(cudaStreamSynchronize(st));
    });
}

arso_status arso_autotune(uint32_t n_qubits, const arso_gate *gates, size_t n_gates, const arso_criterion *crit,
                          double p, uint64_t n_traj, uint64_t seed, const arso_compile_opts *base, void *stream,
                          arso_compile_opts *best, double *ms_out, uint32_t *n_candidates) {
    return guard([&] {
        ARSO_REQUIRE(crit && best, "NULL argument");
        ARSO_REQUIRE(p >= 0 && p <= 1 && n_traj > 0, "need p in [0, 1] and n_traj > 0");
        cudaStream_t st = (cudaStream_t)stream;
        arso_compile_opts b0{};
        if (base) b0 = *base;
        std::vector<arso_compile_opts> cands;
        const int rmax = b0.precision == ARSO_C128 ? RESIDENT_MAX_N_C128 : RESIDENT_MAX_N_C64;
        if ((int)n_qubits <= rmax) {
            cands.push_back(b0);
        } else {
            for (uint32_t t = 10; t <= 14 && t <= n_qubits; ++t)
                for (uint32_t lq = 3; lq <= 5; ++lq) {
                    arso_compile_opts o = b0;
                    o.tile_qubits = t;
                    o.low_qubits = lq;
                    cands.push_back(o);
                }
        }
        cudaEvent_t e0, e1;
        ARSO_CUDA(cudaEventCreate(&e0));
        ARSO_CUDA(cudaEventCreate(&e1));
        double best_ms = INFINITY;
        size_t best_i = 0;
        for (size_t i = 0; i < cands.size(); ++i) {
            arso_circuit *c = nullptr;
            arso_status s1 = arso_compile_circuit(n_qubits, gates, n_gates, &cands[i], &c);
            if (s1 != ARSO_OK) throw Error(s1, arso_last_error());
            std::unique_ptr<arso_circuit> hold(c);
            DevCrit dc;
            make_crit(c, crit, dc, st);
            Scratch sc(st, n_traj * 8);
            double ms = INFINITY;
            for (int rep = 0; rep < 4; ++rep) {  // the first run builds the prefix cache; best of the other 3
                arso_error_list *raw = nullptr;
                ARSO_CUDA(cudaEventRecord(e0, st));
                sample(c, p / 3, p / 3, p / 3, seed, 0, n_traj, st, &raw);
                std::unique_ptr<arso_error_list> e(raw);
                run_all(c, e.get(), dc, st, sc.as<double>(), nullptr);
                ARSO_CUDA(cudaEventRecord(e1, st));
                ARSO_CUDA(cudaEventSynchronize(e1));
                float f = 0;
                ARSO_CUDA(cudaEventElapsedTime(&f, e0, e1));
                if (rep > 0) ms = std::min(ms, (double)f);
            }
            if (ms_out && i < 16) ms_out[i] = ms;
            if (ms < best_ms) best_ms = ms, best_i = i;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *best = cands[best_i];
        if (n_candidates) *n_candidates = (uint32_t)cands.size();
    });
}

arso_status arso_trajectory_states(const arso_circuit *cc, const arso_error_list *e, uint64_t first, uint64_t count,
                                   void *stream, void *amps_out) {
    return guard([&] {
        ARSO_REQUIRE(cc && e && amps_out, "NULL argument");
        ARSO_REQUIRE(e->circ == cc, "error list belongs to another circuit");
        ARSO_REQUIRE(first + count <= e->n_traj, "trajectory range out of bounds");
        ARSO_REQUIRE(is_device_ptr(amps_out), "amps_out must be device memory");
        arso_circuit *c = const_cast<arso_circuit *>(cc);
        cudaStream_t st = (cudaStream_t)stream;
        ensure_cache(c, st);
        if (!count) return;
        if (c->engine == 0) {
            ResidentArgs a = resident_args(c);
            a.first_traj = first;
            a.count = count;
            a.offsets = e->d_offsets.as<uint64_t>();
            a.keys = e->d_key.as<uint32_t>();
            a.first = e->d_first.as<uint32_t>();
            a.states_out = amps_out;
            launch_resident_any(c, a, 1, 2.0 * (double)count * c->state_bytes(), st);
        } else {
            std::vector<uint32_t> fp(count);
            copy_d2h(fp.data(), e->d_first.as<uint32_t>() + first, count * 4, st);
            ARSO_CUDA(cudaStreamSynchronize(st));
            std::vector<uint64_t> ids(count);
            for (uint64_t i = 0; i < count; ++i) ids[i] = first + i;
            DCrit none{};
            run_streaming(c, e, ids, fp, fp, none, nullptr, nullptr, amps_out, st);
        }
        ARSO_CUDA(cudaStreamSynchronize(st));
    });
}

arso_status arso_reference_state(const arso_circuit *cc, void *stream, void *amps_out) {
    return guard([&] {
        ARSO_REQUIRE(cc && amps_out, "NULL argument");
        arso_circuit *c = const_cast<arso_circuit *>(cc);
        cudaStream_t st = (cudaStream_t)stream;
        ensure_cache(c, st);
        ARSO_CUDA(cudaMemcpyAsync(amps_out, ref_state_ptr(c), c->state_bytes(), cudaMemcpyDefault, st));
        ARSO_CUDA(cudaStreamSynchronize(st));
    });
}

arso_status arso_exhaustive(const arso_circuit *cc, const arso_criterion *crit, void *stream, double *P_out,
                            double *per_location) {
    return guard([&] {
        ARSO_REQUIRE(cc && crit && P_out, "NULL argument");
        arso_circuit *c = const_cast<arso_circuit *>(cc);
        cudaStream_t st = (cudaStream_t)stream;
        DevCrit dc;
        make_crit(c, crit, dc, st);
        std::vector<double> pm, pp;
        exhaustive(c, dc, st, P_out, per_location ? &pm : nullptr, per_location ? &pp : nullptr, nullptr);
        if (per_location) {
            const std::vector<double> &v = dc.aggregate == ARSO_AGG_MEAN ? pm : pp;
            std::copy(v.begin(), v.end(), per_location);
        }
    });
}

arso_status arso_success_prob(const arso_circuit *cc, const arso_criterion *crit, double p, uint32_t mode,
                              uint64_t n_traj, uint64_t seed, void *stream, arso_result *out) {
    return guard([&] {
        ARSO_REQUIRE(cc && crit && out, "NULL argument");
        ARSO_REQUIRE(p >= 0.0 && p <= 1.0, "p must be in [0, 1]");
        ARSO_REQUIRE(mode <= ARSO_MODE_EXHAUSTIVE, "bad mode");
        arso_circuit *c = const_cast<arso_circuit *>(cc);
        cudaStream_t st = (cudaStream_t)stream;
        DevCrit dc;
        make_crit(c, crit, dc, st);
        std::memset(out, 0, sizeof(*out));
        out->expected_errors = (double)c->L * p;
        const bool mc = mode == ARSO_MODE_MONTE_CARLO || (mode == ARSO_MODE_AUTO && out->expected_errors > 1.0);
        if (mc) {
            ARSO_REQUIRE(n_traj > 0, "n_traj must be > 0 for Monte Carlo");
            const McOut o = mc_run(c, dc, p, n_traj, seed, st);
            out->mode_used = ARSO_MODE_MONTE_CARLO;
            out->mean = o.mean;
            out->pass_frac = o.pass_frac;
            out->value = dc.aggregate == ARSO_AGG_MEAN ? o.mean : o.pass_frac;
            out->stderr_value = dc.aggregate == ARSO_AGG_MEAN ? o.sd_mean : o.sd_pass;
            out->n_traj = n_traj;
        } else {
            double P[4], Pp[4];
            DevCrit dm;
            make_crit(c, crit, dm, st);
            dm.aggregate = ARSO_AGG_MEAN;
            exhaustive(c, dm, st, P, nullptr, nullptr, Pp);
            out->mode_used = ARSO_MODE_EXHAUSTIVE;
            out->mean = eq4(P, c->L, p / 3);
            out->pass_frac = eq4(Pp, c->L, p / 3);
            const double *sel = dc.aggregate == ARSO_AGG_MEAN ? P : Pp;
            out->value = dc.aggregate == ARSO_AGG_MEAN ? out->mean : out->pass_frac;
            out->P_R = sel[0];
            out->P_X = sel[1];
            out->P_Z = sel[2];
            out->P_Y = sel[3];
            out->n_traj = 3 * c->L;
        }
    });
}

arso_status arso_tolerable_rate(const arso_circuit *cc, const arso_criterion *crit, double P_target,
                                const arso_search_opts *opts, void *stream, arso_rate_result *out) {
    return guard([&] {
        ARSO_REQUIRE(cc && crit && out, "NULL argument");
        arso_circuit *c = const_cast<arso_circuit *>(cc);
        cudaStream_t st = (cudaStream_t)stream;
        arso_search_opts o{};
        if (opts) o = *opts;
        const double p_lo = o.p_lo > 0 ? o.p_lo : 1e-6, p_hi = o.p_hi > 0 ? o.p_hi : 1e-1;
        const double rel = o.rel_tol > 0 ? o.rel_tol : 0.02;
        const uint64_t nt = o.n_traj ? o.n_traj : 1000;
        const uint32_t max_probes = o.max_probes ? o.max_probes : 64;
        ARSO_REQUIRE(p_lo < p_hi && p_hi <= 1.0, "need 0 < p_lo < p_hi <= 1");
        ARSO_REQUIRE(o.surrogate == nullptr, "surrogate search is provided by arso_tolerable_rate_surrogate");
        DevCrit dc;
        make_crit(c, crit, dc, st);
        std::memset(out, 0, sizeof(*out));
        out->P1 = NAN;
        if (o.mode != ARSO_MODE_MONTE_CARLO) {
            double P[4];
            exhaustive(c, dc, st, P, nullptr, nullptr, nullptr);
            const double P1 = (P[1] + P[2] + P[3]) / 3.0;
            out->P1 = P1;
            if (P_target >= P1) {
                // Eq. (5) with count L
                const double denom = (double)c->L * (P1 - P[0]);
                out->p = denom != 0.0 ? (P_target - P[0]) / denom : INFINITY;
                out->lo = out->hi = out->p;
                out->mode_used = 0;
                out->converged = 1;
                return;
            }
        }
        out->mode_used = 1;
        ProbeMemo memo;
        memo.enabled = !(o.flags & ARSO_SEARCH_NO_REUSE);
        auto f = [&](double p) {
            const McOut m = mc_run_memo(c, dc, p, nt, o.seed, st, &memo);
            ++out->probes;
            return dc.aggregate == ARSO_AGG_MEAN ? m.mean : m.pass_frac;
        };
        double lo = p_lo, hi = p_hi;
        double v_lo = f(lo), v_hi = f(hi);
        if (v_lo < P_target || v_hi >= P_target) {
            out->p = v_lo < P_target ? lo : hi;
            out->lo = out->hi = out->p;
            out->value_lo = v_lo;
            out->value_hi = v_hi;
            throw Error(ARSO_ENOTCONVERGED, "target success probability is not bracketed by [p_lo, p_hi]");
        }
        while (hi / lo > 1.0 + rel && out->probes < max_probes) {
            const double mid = std::sqrt(lo * hi);
            const double v = f(mid);
            if (v >= P_target) lo = mid, v_lo = v;
            else hi = mid, v_hi = v;
        }
        out->lo = lo;
        out->hi = hi;
        out->value_lo = v_lo;
        out->value_hi = v_hi;
        if (v_lo == v_hi) {
            out->p = std::sqrt(lo * hi);
        } else {
            const double fr = (v_lo - P_target) / (v_lo - v_hi);
            out->p = std::pow(10.0, std::log10(lo) + fr * (std::log10(hi) - std::log10(lo)));
        }
        out->converged = hi / lo <= 1.0 + rel;
        if (!out->converged) throw Error(ARSO_ENOTCONVERGED, "probe budget exhausted before rel_tol");
    });
}

arso_status arso_tolerable_rate_surrogate(const arso_circuit *cc, const arso_criterion *crit, double P_target,
                                          const arso_search_opts *opts, void *stream, arso_rate_result *out) {
    return guard([&] {
        ARSO_REQUIRE(cc && crit && out && opts && opts->surrogate, "NULL argument or no surrogate");
        ARSO_REQUIRE(crit->aggregate == ARSO_AGG_PASS, "the surrogate predicts pass probabilities: aggregate must be PASS");
        arso_circuit *c = const_cast<arso_circuit *>(cc);
        cudaStream_t st = (cudaStream_t)stream;
        const double p_lo = opts->p_lo > 0 ? opts->p_lo : 1e-6, p_hi = opts->p_hi > 0 ? opts->p_hi : 1e-1;
        const double margin = opts->surrogate_margin > 0 ? opts->surrogate_margin : 0.15;
        const uint64_t nt = opts->n_traj ? opts->n_traj : 1000;
        ARSO_REQUIRE(p_lo < p_hi && p_hi <= 1.0, "need 0 < p_lo < p_hi <= 1");
        DevCrit dc;
        make_crit(c, crit, dc, st);
        std::memset(out, 0, sizeof(*out));
        out->P1 = NAN;
        out->mode_used = 1;
        out->used_surrogate = 1;
        // 1. the surrogate's crossing on a fine grid of log10 p (one batched forward)
        const std::vector<float> f = circuit_features(c, crit);
        const int K = 1024;
        const double a = std::log10(p_lo), b = std::log10(p_hi);
        std::vector<float> rows((size_t)K * ARSO_SURROGATE_INPUTS);
        for (int i = 0; i < K; ++i) {
            std::copy(f.begin(), f.end(), rows.begin() + (size_t)i * ARSO_SURROGATE_INPUTS);
            rows[(size_t)i * ARSO_SURROGATE_INPUTS + ARSO_N_FEATURES] = (float)(a + (b - a) * i / (K - 1));
        }
        Scratch d_rows(st, rows.size() * 4), d_pred(st, K * 4);
        copy_h2d(d_rows.ptr, rows.data(), rows.size() * 4, st);
        const arso_status ps = arso_surrogate_predict(opts->surrogate, d_rows.as<float>(), K, d_pred.as<float>(), st);
        if (ps != ARSO_OK) throw Error(ps, arso_last_error());
        std::vector<float> pred(K);
        copy_d2h(pred.data(), d_pred.ptr, K * 4, st);
        ARSO_CUDA(cudaStreamSynchronize(st));
        int i0 = K - 1;
        for (int i = 0; i < K; ++i)
            if (pred[i] < P_target) { i0 = i; break; }
        double lp_s = a + (b - a) * std::max(0, i0) / (K - 1);
        if (i0 > 0 && pred[i0 - 1] != pred[i0]) {  // interpolate between the grid points around the crossing
            const double fr = (pred[i0 - 1] - P_target) / (pred[i0 - 1] - pred[i0]);
            lp_s = a + (b - a) * ((i0 - 1) + fr) / (K - 1);
        }
        // 2. verify the bracket with plain trajectories (common random numbers)
        ProbeMemo memo;
        memo.enabled = !(opts->flags & ARSO_SEARCH_NO_REUSE);
        auto probe = [&](double p) {
            const McOut m = mc_run_memo(c, dc, p, nt, opts->seed, st, &memo);
            ++out->probes;
            return m.pass_frac;
        };
        double lo = std::max(p_lo, std::pow(10.0, lp_s - margin)), hi = std::min(p_hi, std::pow(10.0, lp_s + margin));
        double v_lo = probe(lo), v_hi = probe(hi);
        // widen a side that fails, by steps of 2, 4, 8 margins (every probe reuses the
        // trajectories of the earlier ones whose error sets it shares)
        for (int widen = 0; widen < 3 && !(v_lo >= P_target && v_hi < P_target); ++widen) {
            const double step = std::pow(10.0, 2 * margin * (double)(1 << widen));
            if (v_lo < P_target && lo > p_lo) lo = std::max(p_lo, lo / step), v_lo = probe(lo);
            if (v_hi >= P_target && hi < p_hi) hi = std::min(p_hi, hi * step), v_hi = probe(hi);
        }
        out->verified = v_lo >= P_target && v_hi < P_target;
        // the surrogate missed by more than the widening reaches: the search range's ends
        if (!out->verified) {
            if (v_lo < P_target && lo > p_lo) lo = p_lo, v_lo = probe(lo);
            if (v_hi >= P_target && hi < p_hi) hi = p_hi, v_hi = probe(hi);
        }
        if (!(v_lo >= P_target && v_hi < P_target)) {
            out->p = v_lo < P_target ? lo : hi;
            out->lo = out->hi = out->p;
            out->value_lo = v_lo;
            out->value_hi = v_hi;
            throw Error(ARSO_ENOTCONVERGED, "target success probability is not bracketed by [p_lo, p_hi]");
        }
        // narrow a bracket wider than the nominal 10^(2 margin): bisection in log p while it
        // is more than four nominal widths, then plain probes at the log-linear interpolation
        // point kept inside the middle 60%, so the final interpolation spans at most a
        // nominal bracket
        const double nominal = 2 * margin * (1 + 1e-9);
        for (int r = 0; r < 24 && std::log10(hi / lo) > nominal; ++r) {
            const double w = std::log10(hi / lo);
            const double fr = w > 4 * nominal ? 0.5 : std::min(0.8, std::max(0.2, (v_lo - P_target) / (v_lo - v_hi)));
            const double pm = std::pow(10.0, std::log10(lo) + fr * w);
            const double vm = probe(pm);
            if (vm >= P_target) lo = pm, v_lo = vm;
            else hi = pm, v_hi = vm;
        }
        out->converged = std::log10(hi / lo) <= nominal;
        out->lo = lo;
        out->hi = hi;
        out->value_lo = v_lo;
        out->value_hi = v_hi;
        const double fr = (v_lo - P_target) / (v_lo - v_hi);
        out->p = std::pow(10.0, std::log10(lo) + fr * (std::log10(hi) - std::log10(lo)));
        if (!out->converged) throw Error(ARSO_ENOTCONVERGED, "probe budget exhausted before the nominal bracket");
    });
}

arso_status arso_apply_gate(uint32_t n, void *amps, const arso_gate *gate, void *stream) {
    return guard([&] {
        ARSO_REQUIRE(amps && gate, "NULL argument");
        ARSO_REQUIRE(n >= 2 && n <= 34, "n_qubits must be in [2, 34]");
        ARSO_REQUIRE(is_device_ptr(amps), "amps must be device memory");
        HostGate h{};
        h.kind = gate->kind;
        h.arity = gate->kind >= ARSO_GATE_CX ? 2 : 1;
        h.q0 = gate->q[0];
        h.q1 = h.arity == 2 ? gate->q[1] : gate->q[0];
        ARSO_REQUIRE(h.q0 < n && h.q1 < n && (h.arity == 1 || h.q0 != h.q1), "bad gate qubits");
        matrix_for(*gate, h);
        DGate d{};
        // the single-gate HBM kernel takes H and the omega phases as plain dense/diagonal gates
        d.cls = h.cls == GC_H ? (uint8_t)GC_DENSE1 : h.cls == GC_OMEGA ? (uint8_t)GC_DIAG1 : h.cls == GC_CZ ? (uint8_t)GC_DIAG2 : h.cls;
        d.arity = (uint8_t)h.arity;
        d.q0 = (uint8_t)h.q0;
        d.q1 = (uint8_t)h.q1;
        M16 m{};
        if (h.arity == 1 && d.cls == GC_DIAG1) {
            m.m[0] = make_float2((float)h.m[0].real(), (float)h.m[0].imag());
            m.m[1] = make_float2((float)h.m[3].real(), (float)h.m[3].imag());
        } else {
            for (int i = 0; i < (h.arity == 1 ? 4 : 16); ++i)
                m.m[i] = make_float2((float)h.m[i].real(), (float)h.m[i].imag());
        }
        if (h.cls == GC_NOP) return;
        launch_gate_pairs(static_cast<float2 *>(amps), (int)n, d, m, (cudaStream_t)stream);
        ARSO_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    });
}

arso_status arso_apply_pauli(uint32_t n, void *amps, uint32_t qubit, uint32_t code, void *stream) {
    return guard([&] {
        ARSO_REQUIRE(amps != nullptr, "NULL argument");
        ARSO_REQUIRE(n >= 1 && n <= 34 && qubit < n, "bad qubit");
        ARSO_REQUIRE(code >= 1 && code <= 3, "code must be 1 (X), 2 (Z) or 3 (Y)");
        ARSO_REQUIRE(is_device_ptr(amps), "amps must be device memory");
        launch_pauli(static_cast<float2 *>(amps), (int)n, qubit, code, (cudaStream_t)stream);
        ARSO_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    });
}

arso_status arso_score_state(uint32_t n, const void *amps, const void *ref, const arso_criterion *crit, void *stream,
                             double *score_out) {
    return guard([&] {
        ARSO_REQUIRE(amps && crit && score_out, "NULL argument");
        ARSO_REQUIRE(n >= 1 && n <= 34, "bad n");
        ARSO_REQUIRE(crit->kind != ARSO_CRIT_FIDELITY || ref != nullptr, "fidelity needs ref");
        cudaStream_t st = (cudaStream_t)stream;
        arso_circuit tmp;
        tmp.n = n;
        DevCrit dc;
        make_crit(&tmp, crit, dc, st);
        Scratch d(st, 8);
        score_into(amps, ref ? ref : amps, (int)n, ARSO_C64, dc.d, d.as<double>(), st);
        copy_d2h(score_out, d.ptr, 8, st);
        ARSO_CUDA(cudaStreamSynchronize(st));
    });
}

}  // extern "C"
