// Internal types shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/arso.h"

namespace arso {

// ---------------------------------------------------------------- errors ---
struct Error : std::runtime_error {
    arso_status status;
    Error(arso_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};
void set_last_error(const std::string &m);

#define ARSO_CUDA(call)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            throw ::arso::Error(e_ == cudaErrorMemoryAllocation ? ARSO_ENOMEM : ARSO_ECUDA,   \
                                std::string(#call) + ": " + cudaGetErrorString(e_));          \
    } while (0)
#define ARSO_REQUIRE(cond, msg)                                              \
    do {                                                                     \
        if (!(cond)) throw ::arso::Error(ARSO_EINVAL, msg);                  \
    } while (0)

// ------------------------------------------------------- device gate code --
// Gate classes: how a kernel applies the gate.
enum GateClass : uint8_t {
    GC_NOP = 0,     // identity
    GC_DENSE1 = 1,  // 2x2 dense
    GC_DIAG1 = 2,   // diag(d0, d1)
    GC_X = 3,       // bit flip
    GC_DENSE2 = 4,  // 4x4 dense
    GC_DIAG2 = 5,   // diag(d0..d3)
    GC_CX = 6,      // controlled bit flip (q0 control, q1 target)
    GC_SWAP = 7,
    GC_H = 8,       // Hadamard, 1/sqrt2 applied as a two-float constant (unbiased rounding)
    GC_OMEGA = 9,   // diag(1, e^{i k pi/4}), k in DGate::mat; exact for even k, two-float 1/sqrt2 for odd k
    GC_CZ = 10,     // diag(1, 1, 1, -1)
    GC_SU2 = 11,    // 2x2 dense of the form [[a, b], [-conj b, conj a]] (register kernels read a and b)
};

// Register-blocked execution (tiles of >= 2^10 amplitudes): every thread
// holds 2^REG_BITS amplitudes of the tile in registers; a "phase" fixes which
// REG_BITS tile-local bits index those registers. Gates that mix amplitudes
// need their qubits among the register bits of the phase that runs them;
// diagonal gates, X gates and Pauli errors act on any bit.
constexpr int REG_BITS = 5;
constexpr int RB_MIN_TILE = 10;                   // 32 threads x 32 amplitudes
// gates per phase at most: the register kernels stage a phase's gate records
// in shared memory (double-buffered: the next phase's copy overlaps this one)
constexpr int MAX_PHASE_OPS = 64;
inline uint32_t pack_rbits(const uint32_t *p) {   // 5 local bit positions, 5 bits each
    uint32_t r = 0;
    for (int b = 0; b < REG_BITS; ++b) r |= p[b] << (5 * b);
    return r;
}

// 1/sqrt(2) split into a float and its float remainder, so that c*x can be
// formed as fma(hi, x, lo*x) without the bias of a rounded constant; the bias
// would otherwise shrink the norm by ~2.4e-8 per H or T gate.
constexpr double RSQRT2_D = 0.70710678118654752440084436210485;
constexpr float RSQRT2_HI = (float)RSQRT2_D;
constexpr float RSQRT2_LO = (float)(RSQRT2_D - (double)RSQRT2_HI);

// One gate as the kernels see it. q0/q1 are tile-local bit positions for
// the pass that contains the gate (global positions for the resident engine).
struct DGate {
    uint8_t cls;
    uint8_t q0, q1;
    uint8_t arity;
    uint32_t mat;   // offset (in complex entries) into the matrix pool
};

// One gate as the register-blocked kernels see it: everything in one 32-byte
// record (two 16-byte loads, no dependent second load for the common gates).
//   w0  = cls | p0 << 8 | p1 << 12 | q0 << 16 | q1 << 24, with p0/p1 the
//         register positions of q0/q1 in the gate's phase (15: thread bit)
//   aux = matrix-pool offset (dense and two-qubit diagonal gates) or the
//         exponent k of GC_OMEGA
//   c0, c1 = inline constants: (a, b) of GC_SU2, (d0, d1) of GC_DIAG1
struct __align__(16) RegOp {
    uint32_t w0, aux;
    float2 c0, c1;
    uint32_t pad[2];
};

// Register-kernel op codes (RegOp::pad[0] bits 0-7): the gate class with its
// register positions resolved on the host, so the kernel dispatches once.
// Mask-dependent variants follow their base code: the kernel adds
// sa * (bit q0 of m ^ xa) + sb * (bit q1 of m ^ xb), with sa (bits 8-9),
// sb (bits 10-11), xa (bit 12), xb (bit 13) of pad[0].
enum RegOpCode : uint32_t {
    OP_SU2 = 0,      // + register position 0..4 (0: the packed lanes)
    OP_DENSE1 = 5,   // + position
    OP_H = 10,       // + 2 * position + mask bit of q0
    OP_CZ_RR = 20,   // + 4 * pair index of (lower, higher) position + 2 * want(lower) + want(higher)
    OP_CZ_RT = 60,   // + 2 * register position + want(register qubit); the other qubit is a thread bit
    OP_CZ_TT = 70,   // both qubits thread bits
    OP_X = 71,
    OP_OMEGA = 72,
    OP_DIAG1 = 73,
    OP_DIAG2 = 74,
    OP_CX = 75,      // + target position
    OP_DENSE2 = 80,
    OP_SWAP = 81,
    OP_NOP = 82,
};

// Tensor-core phases (streaming complex64 circuits compiled with
// ARSO_OPT_TENSOR_PHASES, tiles of 2^12..2^14 amplitudes). A phase whose gates on
// its register bits multiply to one 32 x 32 unitary U, the phase's other gates
// being diagonal, can run as a contraction on the tensor cores: the tile is a
// matrix of 2^(t-5) rows (threads) by 32 complex columns (register index), and
// U acts on every row. Each record of such a phase has a role (RegOp::pad[1]):
// a core gate (inside U), or a diagonal gate run in FP32 before or after U. A
// diagonal gate touching a register bit and another bit runs after U when a
// non-diagonal core gate of the phase acted on that register bit before it,
// otherwise before U; the planner admits no non-diagonal gate on that bit after
// it in the phase, so both orders equal the records' order.
enum TensorRole : uint32_t { TR_CORE = 0, TR_BEFORE = 1, TR_AFTER = 2 };
constexpr uint32_t NO_TENSOR = 0xFFFFFFFFu;
// a phase runs on the tensor cores when its unitary holds at least this many
// non-diagonal gates (below that the FP32 gate code is cheaper)
constexpr int TENSOR_MIN_DENSE = 2;
// fp16 operand images of one tensor phase: hi and lo terms of the real 64 x 64
// form of U, each 8 KiB in the tensor core's K-major shared-memory layout
constexpr uint32_t TENSOR_IMAGE_HALVES = 2 * 64 * 64;

// An event in engine order: (gate position << 3) | (slot << 2) | pauli code.
__host__ __device__ inline uint32_t ev_pos(uint32_t e) { return e >> 3; }
__host__ __device__ inline uint32_t ev_slot(uint32_t e) { return (e >> 2) & 1u; }
__host__ __device__ inline uint32_t ev_code(uint32_t e) { return e & 3u; }

constexpr uint32_t NO_EVENT = 0xFFFFFFFFu;

// Largest resident state (whole state in one CTA's shared memory).
constexpr int RESIDENT_MAX_N_C64 = 13;   // 64 KiB
constexpr int RESIDENT_MAX_N_C128 = 12;  // 64 KiB
constexpr int MAX_TILE_QUBITS = 14;      // 128 KiB complex64 tile

// ------------------------------------------------------------- host side --
struct HostGate {
    uint32_t kind;
    uint32_t q0, q1;
    int arity;
    uint8_t cls;
    uint32_t omega_k = 0;        // GC_OMEGA exponent
    std::complex<double> m[16];  // 2x2 (first 4) or 4x4, row-major
};

struct Pass {
    uint32_t gb, ge;                   // gate range in engine order
    std::vector<uint32_t> tile_qubits; // sorted global qubits, tile-local bit i -> tile_qubits[i]
    uint32_t pb = 0, pe = 0;           // register-blocked phases [pb, pe)
    double flops_per_amp = 0.0;        // algorithmic FP32 flops per amplitude of one sweep
    uint32_t remaps = 0;               // register-set changes inside the pass (from the load layout)
    uint32_t end_remap = 0;            // 1 if the last phase's set differs from the load layout
};

struct Criterion {
    uint32_t kind, aggregate;
    uint64_t target;
    double threshold;
    std::vector<uint64_t> set;
};

struct DeviceBuffer {
    void *ptr = nullptr;
    size_t bytes = 0;
    DeviceBuffer() = default;
    DeviceBuffer(const DeviceBuffer &) = delete;
    DeviceBuffer &operator=(const DeviceBuffer &) = delete;
    ~DeviceBuffer() { release(); }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    void ensure(size_t b) {
        if (b <= bytes) return;
        release();
        ARSO_CUDA(cudaMalloc(&ptr, b));
        bytes = b;
    }
    template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

}  // namespace arso

struct arso_circuit {
    uint32_t n = 0;
    int precision = ARSO_C64;
    int engine = 0;  // 0 resident, 1 streaming
    uint32_t tile_qubits = 0, low_qubits = 0, max_batch = 0, flags = 0;
    uint64_t cache_budget = 0;
    std::vector<arso::HostGate> gates;      // circuit order
    uint64_t k = 0, m = 0, L = 0;
    std::vector<uint32_t> perm;             // engine position -> circuit gate index
    std::vector<uint32_t> pos_of;           // circuit gate index -> engine position
    std::vector<uint32_t> loc_gate;         // location -> circuit gate index
    std::vector<arso::Pass> passes;         // streaming schedule (resident: one pass)
    std::vector<uint32_t> pass_of_pos;      // engine position -> pass index
    bool reg_blocked = false;               // phases planned (tile >= 2^10, complex64)
    std::vector<uint32_t> ph_gb;            // phase -> first engine position (plus a sentinel)
    std::vector<uint32_t> ph_R;             // phase -> packed register bits
    std::vector<uint8_t> rpos;              // engine position -> (reg pos of q0) | (reg pos of q1) << 4, 15 = none
    std::vector<uint32_t> phase_of_pos;     // engine position -> phase
    std::vector<double> flops_prefix;       // engine position k -> algorithmic FP32 flops per amplitude of
                                            // gates [0, k) (the tracing counts of arso.h)
    std::vector<uint32_t> chg_prefix;       // phase k -> phases 1 <= p < k whose register set differs from p-1's
    // tensor-core phases (ARSO_OPT_TENSOR_PHASES on a streaming complex64 circuit)
    bool tensor = false;
    std::vector<uint32_t> ph_t;             // phase -> index of its operand images, or NO_TENSOR
    std::vector<uint16_t> tmats;            // TENSOR_IMAGE_HALVES fp16 values per tensor phase
    std::vector<uint8_t> role;              // engine position -> TensorRole within its phase
    arso::DeviceBuffer d_tmats, d_ph_t;
    arso::DeviceBuffer d_terr;              // uint32: a tensor-phase wait gave up
    // device tables
    arso::DeviceBuffer d_gates;             // DGate[G] in engine order
    arso::DeviceBuffer d_mats;              // complex<float> or complex<double> pool
    arso::DeviceBuffer d_loc_key;           // location -> (pos << 1) | slot
    arso::DeviceBuffer d_pass_of_pos;       // uint32 per engine position
    arso::DeviceBuffer d_ph_gb, d_ph_R, d_rops, d_phase_of_pos;
    // prefix cache
    bool cache_ready = false;
    uint64_t ckpt_every = 1;                // resident: gates between checkpoints
    uint32_t n_ckpt = 0;                    // checkpoints (resident) or pass boundaries (streaming)
    std::vector<uint32_t> ckpt_pass;        // streaming: cached boundary index per pass
    arso::DeviceBuffer d_cache;             // n_ckpt states; the last one is psi_R
    // streaming complex64: backward states W^dagger |bwd_target> at the cached pass
    // boundaries (W = the error-free rest of the circuit), same entries as d_cache; the
    // outcome criterion's suffix reuse scores trajectories against them
    bool bwd_ready = false;
    uint64_t bwd_target = 0;
    arso::DeviceBuffer d_bwd;
    arso::DeviceBuffer d_offs;              // streaming: per pass, tile-high offsets
    std::vector<uint64_t> offs_base;        // per pass offset of its table in d_offs
    size_t state_bytes() const { return (size_t(1) << n) * (precision == ARSO_C128 ? 16 : 8); }
};

struct arso_error_list {
    const arso_circuit *circ = nullptr;
    uint64_t n_traj = 0, n_events = 0;
    arso::DeviceBuffer d_offsets;  // uint64[n_traj + 1]
    arso::DeviceBuffer d_loc;      // uint32 (loc << 2) | code, location order
    arso::DeviceBuffer d_key;      // uint32 engine-order keys
    arso::DeviceBuffer d_first;    // uint32 per trajectory: first engine position with an event, or NO_EVENT
    arso::DeviceBuffer d_last;     // uint32 per trajectory: last engine position with an event, or NO_EVENT
};

namespace arso {
// circuit.cpp
void matrix_for(const arso_gate &g, HostGate &h);  // h.arity must be set
std::vector<float> circuit_features(const arso_circuit *c, const arso_criterion *crit);
void build_circuit(arso_circuit *c, uint32_t n, const arso_gate *gates, size_t n_gates,
                   const arso_compile_opts *opts);
}  // namespace arso
