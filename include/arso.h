/*
 * arso.h - C ABI of the GB300 library for the Monte Carlo Pauli-error path of
 * ArsoNISQ: state-vector simulation of a quantum circuit with Pauli X/Z/Y
 * error gates appended after its gates, a per-trajectory success criterion,
 * the success probability at an error rate p, and the tolerable error rate
 * for a target success probability.
 *
 * Conventions (all entry points):
 *  - Every call returns an arso_status; nothing throws or aborts across the
 *    ABI. On a non-OK status arso_last_error() returns a thread-local message.
 *  - Inputs are caller-owned and copied (or fully consumed) before return.
 *  - Handles (arso_circuit, arso_error_list, arso_surrogate) are library-owned
 *    and freed with their *_free function; freeing NULL is a no-op.
 *  - Output arrays are caller-allocated. Where a pointer may be host or device
 *    memory the library detects which (cudaPointerGetAttributes).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls that
 *    return host values synchronise that stream before returning.
 *  - Qubit q is bit q of the amplitude index (little-endian). Amplitude arrays
 *    are interleaved (re, im): float pairs for ARSO_C64, double pairs for
 *    ARSO_C128.
 *  - Error locations: location l enumerates (gate g, qubit slot j) in circuit
 *    order, one location per qubit of each gate, so L = k + 2m for k one-qubit
 *    and m two-qubit gates (Sec. IV-B.1, Eq. (3)).
 *  - Pauli codes: 1 = X, 2 = Z, 3 = Y, acting as Eq. (2) prints them:
 *    X (a0, a1) -> (a1, a0); Z -> (a0, -a1); Y -> (-i a1, i a0).
 *  - The library allocates device memory for its own handles and scratch with
 *    the CUDA runtime; it never takes ownership of caller memory.
 */
#ifndef ARSO_H
#define ARSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ARSO_OK = 0,
    ARSO_EINVAL = 1,         /* bad argument: NULL handle, qubit out of range, p outside [0,1] ... */
    ARSO_ENOMEM = 2,         /* a device or host allocation failed */
    ARSO_ECUDA = 3,          /* a CUDA runtime call or kernel launch failed */
    ARSO_ETIMEOUT = 4,       /* a bounded device-side wait gave up */
    ARSO_EUNSUPPORTED = 5,   /* valid request outside what this build supports */
    ARSO_ENOTCONVERGED = 6   /* a search ended without meeting its tolerance */
} arso_status;

/* Gate kinds. One-qubit gates use q[0]; two-qubit gates use q[0], q[1]
 * (control first for CX and CP). Textbook matrices:
 *   H = [[1,1],[1,-1]]/sqrt2, X, Y = [[0,-i],[i,0]], Z, S = diag(1,i),
 *   SDG = diag(1,-i), T = diag(1,e^{i pi/4}), TDG = diag(1,e^{-i pi/4}),
 *   RX(t) = [[c,-is],[-is,c]], RY(t) = [[c,-s],[s,c]] (c = cos t/2, s = sin t/2),
 *   RZ(t) = diag(e^{-it/2}, e^{it/2}), P(l) = diag(1, e^{il}),
 *   CX, CZ = diag(1,1,1,-1), CP(l) = diag(1,1,1,e^{il}), SWAP.
 * U and U2 take an explicit unitary in `matrix`: row-major, (re, im) pairs,
 * 2x2 (8 doubles) or 4x4 (32 doubles), local index k = bit(q0) + 2*bit(q1). */
enum {
    ARSO_GATE_ID = 0, ARSO_GATE_H, ARSO_GATE_X, ARSO_GATE_Y, ARSO_GATE_Z,
    ARSO_GATE_S, ARSO_GATE_SDG, ARSO_GATE_T, ARSO_GATE_TDG,
    ARSO_GATE_RX, ARSO_GATE_RY, ARSO_GATE_RZ, ARSO_GATE_P, ARSO_GATE_U,
    ARSO_GATE_CX = 32, ARSO_GATE_CZ, ARSO_GATE_CP, ARSO_GATE_SWAP, ARSO_GATE_U2
};

typedef struct {
    uint32_t kind;          /* ARSO_GATE_* */
    uint32_t q[2];          /* qubits; q[1] ignored for one-qubit gates */
    double param;           /* angle for RX/RY/RZ/P/CP, ignored otherwise */
    const double *matrix;   /* U/U2 only: caller-owned, copied on entry */
} arso_gate;

enum { ARSO_C64 = 0, ARSO_C128 = 1 };

typedef struct {
    uint32_t precision;     /* ARSO_C64 (complex64 amplitudes, FP32 arithmetic) or ARSO_C128 */
    uint32_t tile_qubits;   /* streaming passes: qubits per tile; 0 = auto (13 for complex64, the
                               size arso_run_batch's persistent launch takes; arso_autotune
                               measures 10..14) */
    uint32_t low_qubits;    /* streaming passes: qubits 0..low-1 are in every tile; 0 = auto (4) */
    uint32_t max_batch;     /* streaming engine: trajectories resident at once; 0 = auto */
    uint64_t cache_bytes;   /* budget for cached error-free prefix states; 0 = auto */
    uint32_t flags;         /* ARSO_OPT_* */
} arso_compile_opts;
/* Fidelity scores are taken right after a trajectory's last error, against the
 * cached error-free state at that pass boundary: the error-free suffix W is
 * unitary and common to both states, so <W a|W b> = <a|b> (exact). Outcome
 * probabilities (streaming complex64 circuits) likewise, as |<phi|a>|^2 with the
 * backward state phi = W^dagger |target> cached at that boundary. This flag
 * turns that off (every trajectory then runs to the end; for comparisons). */
/* The streaming engine records each batch's pass launches into a CUDA graph
 * (keyed by the batch's pass range and slot count) and replays it for later
 * batches of the same shape; this flag launches every pass directly. */
/* Exhaustive single-error analysis (Sec. IV-B.1) takes every single-error
 * score from one sweep. Fidelity: the state with error P on qubit q after gate
 * g has fidelity <psi_g|P|psi_g>^2 with psi_R, because the rest of the circuit
 * is unitary and maps psi_g to psi_R, so one error-free sweep of Pauli
 * expectations suffices; it keeps the state in one CTA (resident circuits) or in
 * HBM (streaming complex64 circuits, one launch per gate that applies it and
 * measures its qubits).
 * Outcome probability: the score is |<phi_g|P|psi_g>|^2 with the backward state
 * phi_g = W^dagger |target> for the rest W of the circuit; one backward sweep
 * carries psi and phi from (psi_R, |target>) with the adjoint gates (one CTA,
 * or one HBM launch per gate for streaming complex64 circuits). This flag
 * simulates the 3L single-error trajectories instead (for comparisons). */
/* arso_run_batch runs circuits with ARSO_OPT_NO_PERSISTENT on their own
 * launches instead of the batch's persistent launch (for comparisons). */
/* ARSO_OPT_TENSOR_PHASES (streaming complex64 circuits, 12-14-qubit tiles): the
 * phase planner forms register phases whose gates on the five register bits
 * multiply to one 32 x 32 unitary U (the phase's other gates being diagonal),
 * and the pass kernel applies U to the tile on the tensor cores (a 2^(t-5) x 64
 * by 64 x 64 real contraction on FP16 operands: per entry an integer high part
 * and a low part, under a power-of-two scale per row, the high products summed
 * exactly and the rest in a second FP32 accumulator; about FP32 accuracy)
 * instead of gate by gate. A phase holding one of the trajectory's Pauli errors, or with
 * fewer than two non-diagonal gates, runs gate by gate. A wait for the tensor
 * cores is bounded; one that gives up makes the call return ARSO_ETIMEOUT. */
enum { ARSO_OPT_NO_SUFFIX_REUSE = 1, ARSO_OPT_NO_GRAPHS = 2, ARSO_OPT_NO_FAST_EXHAUSTIVE = 4,
       ARSO_OPT_NO_PERSISTENT = 8, ARSO_OPT_TENSOR_PHASES = 16 };

typedef struct arso_circuit arso_circuit;
typedef struct arso_error_list arso_error_list;

/* Compile a circuit (Sec. II: a list of gates acting on n qubits) for the GPU:
 * builds gate matrices, the error-location table, the fused pass schedule (each
 * pass's tile qubits chosen to place the most gates from the circuit's
 * frontier, Sec. II's gate order kept on every qubit) and
 * uploads them. n_qubits in [1, 30]; gates may be empty. `opts` may be NULL.
 * The error-free prefix-state cache is built lazily on first use.
 * Errors: ARSO_EINVAL (bad kind/qubit/matrix), ARSO_ENOMEM, ARSO_ECUDA. */
arso_status arso_compile_circuit(uint32_t n_qubits, const arso_gate *gates, size_t n_gates,
                                 const arso_compile_opts *opts, arso_circuit **out);
void arso_circuit_free(arso_circuit *c);

typedef struct {
    uint32_t n_qubits;
    uint64_t G;             /* gates (the paper's circuit size, Sec. II) */
    uint64_t k, m;          /* one- and two-qubit gates */
    uint64_t L;             /* error locations, k + 2m */
    uint32_t engine;        /* 0 = resident (whole state on chip), 1 = streaming passes */
    uint32_t n_passes;      /* streaming: fused passes; resident: 1 */
    uint32_t tile_qubits;
    uint32_t precision;
    uint64_t checkpoint_every; /* resident: gates between cached prefix states */
    uint32_t n_phases;      /* register phases (0 when the circuit has none) */
    uint32_t tensor_phases; /* phases that run on the tensor cores (ARSO_OPT_TENSOR_PHASES) */
} arso_circuit_info;
arso_status arso_circuit_get_info(const arso_circuit *c, arso_circuit_info *out);

/* Host-only view of the compile step (no GPU needed): the engine order and the
 * fused pass schedule that arso_compile_circuit would build. *n_passes is set
 * on every call; perm (n_gates entries: engine position -> gate index),
 * pass_begin (n_passes + 1 entries) and tile_mask (n_passes entries, bit q set
 * when qubit q is a tile qubit of the pass) are filled when non-NULL and
 * *n_passes <= capacity. Errors: as arso_compile_circuit, and ARSO_EINVAL when
 * capacity is too small for non-NULL arrays. */
arso_status arso_plan_schedule(uint32_t n_qubits, const arso_gate *gates, size_t n_gates,
                               const arso_compile_opts *opts, uint32_t *n_passes, uint32_t capacity,
                               uint32_t *perm, uint32_t *pass_begin, uint64_t *tile_mask);
/* Host-only: the number of register-bit phases the compile step plans (each
 * phase boundary inside a pass is one shared-memory transpose of the tile);
 * 0 when the circuit does not use the register-blocked kernels. *n_tensor (may
 * be NULL) receives how many of them run on the tensor cores. */
arso_status arso_plan_phases(uint32_t n_qubits, const arso_gate *gates, size_t n_gates,
                             const arso_compile_opts *opts, uint32_t *n_phases, uint32_t *n_tensor);
/* Host-only test support (no counterpart in the paper): the tensor-core operand of
 * register phase `phase` of the schedule arso_compile_circuit would build with
 * `opts` (flags with ARSO_OPT_TENSOR_PHASES). *reg_bits: the phase's five register
 * bits (tile-local bit positions of its pass, register bit b at bits 5b..5b+4);
 * [*pos_begin, *pos_end): its gates as engine positions (the order arso_plan_schedule
 * returns); *pass: its pass. roles (may be NULL; *pos_end - *pos_begin bytes, at most
 * roles_capacity): 0 inside the phase's unitary U, 1 a diagonal gate run before U,
 * 2 one run after it. image (may be NULL; 8192 values): the real 64 x 64 form B of U
 * (row n = 4p + 2c + lane for output register 2p + lane, c = 0 real part, 1 imaginary
 * part; column k likewise for the input register), scaled by 2^8 and split into the
 * integer hi = rint(2^8 B) and lo = fp16(2^8 B - hi), both as binary16 bits: hi at
 * index (n/8)*512 + (k/8)*64 + (n%8)*8 + k%8, lo 4096 further. *has_image = 0 when the
 * phase runs gate by gate (image untouched). Errors: ARSO_EINVAL (phase out of range,
 * roles_capacity too small), and as arso_compile_circuit. */
arso_status arso_plan_tensor_phase(uint32_t n_qubits, const arso_gate *gates, size_t n_gates,
                                   const arso_compile_opts *opts, uint32_t phase, uint32_t *reg_bits,
                                   uint32_t *pos_begin, uint32_t *pos_end, uint32_t *pass, uint8_t *roles,
                                   uint32_t roles_capacity, uint16_t *image, uint32_t *has_image);

/* Sample Pauli errors (Sec. IV-B.2): after every gate, each of its qubits
 * independently suffers X, Z or Y with probabilities p_x, p_z, p_y. Trajectory
 * t in [traj_begin, traj_begin + n_traj), location l draws
 * Philox4x32-10(counter = (l >> 1, t mod 2^32, t >> 32, 0x41525345),
 *               key = (seed mod 2^32, seed >> 32))
 * and uses words (w0, w1) for even l, (w2, w3) for odd l. Error iff
 * w_a < min(floor(p_tot 2^32), 2^32 - 1); type X if w_b < floor(p_x/p_tot 2^32),
 * else Z if w_b < floor((p_x+p_z)/p_tot 2^32), else Y. The draw is independent
 * of p, so error sets at two rates are nested. Result: per-trajectory event
 * lists in device memory (CSR), library-owned.
 * Errors: ARSO_EINVAL (p_* < 0 or p_tot > 1), ARSO_ENOMEM, ARSO_ECUDA. */
arso_status arso_sample_errors(const arso_circuit *c, double p_x, double p_z, double p_y,
                               uint64_t seed, uint64_t traj_begin, uint64_t n_traj,
                               void *stream, arso_error_list **out);
/* The error lists of many circuits in one call (Sec. IV-B.2 for a batch of
 * circuits): entry i is exactly arso_sample_errors(circuits[i], p_x[i], p_z[i],
 * p_y[i], seeds[i], traj_begin[i], n_traj[i]) (the same draws and events, bit
 * for bit), but each sampling kernel runs once for the whole batch. All
 * arrays have `count` entries (host memory); out[i] receives list i (freed by
 * arso_error_list_free). On error every out[i] is NULL.
 * Errors: ARSO_EINVAL, ARSO_ENOMEM, ARSO_ECUDA. */
arso_status arso_sample_errors_batch(size_t count, const arso_circuit *const *circuits, const double *p_x,
                                     const double *p_z, const double *p_y, const uint64_t *seeds,
                                     const uint64_t *traj_begin, const uint64_t *n_traj, void *stream,
                                     arso_error_list **out);

/* Build an error list from explicit host events (tests, exhaustive analysis).
 * offsets: n_traj + 1 entries, events[offsets[t] .. offsets[t+1]) belong to
 * trajectory t, each encoded (location << 2) | code, strictly increasing in
 * location within a trajectory. */
arso_status arso_error_list_from_host(const arso_circuit *c, uint64_t n_traj, const uint64_t *offsets,
                                      const uint32_t *events, void *stream, arso_error_list **out);
arso_status arso_error_list_info(const arso_error_list *e, uint64_t *n_traj, uint64_t *n_events);
/* Copy the CSR to host arrays (offsets: n_traj + 1; events: n_events, encoded
 * (location << 2) | code, location order). Synchronises `stream`. */
arso_status arso_error_list_copy(const arso_error_list *e, uint64_t *offsets, uint32_t *events, void *stream);
void arso_error_list_free(arso_error_list *e);

/* Success criteria (Sec. II): fidelity |<psi_R|psi>|^2 with the error-free
 * final state; probability of the correct outcome |psi_target|^2; binning,
 * the probability of an outcome in `set`; argmax, 1 if the most likely outcome
 * is `target` (lowest index wins ties). A trajectory passes iff score >=
 * threshold. aggregate selects what arso_success_prob reports as `value`:
 * the mean score (the paper's averaged P, Sec. IV-C) or the pass fraction. */
enum { ARSO_CRIT_FIDELITY = 0, ARSO_CRIT_OUTCOME = 1, ARSO_CRIT_BINNING = 2, ARSO_CRIT_ARGMAX = 3 };
enum { ARSO_AGG_MEAN = 0, ARSO_AGG_PASS = 1 };
typedef struct {
    uint32_t kind;
    uint32_t aggregate;
    uint64_t target;
    const uint64_t *set;    /* binning only: caller-owned, copied */
    size_t set_len;
    double threshold;
} arso_criterion;

/* Run every trajectory of `errors` (Sec. IV-B: the circuit with the sampled
 * error gates appended after their gates) and score it. score_out: n_traj
 * doubles; pass_out: n_traj bytes or NULL. Host or device pointers.
 * Trajectories with no error take the score of the error-free state; the
 * others restart from the cached error-free state before their first error.
 * Errors: ARSO_EINVAL, ARSO_ENOMEM, ARSO_ECUDA. */
arso_status arso_run_trajectories(const arso_circuit *c, const arso_error_list *errors,
                                  const arso_criterion *crit, void *stream,
                                  double *score_out, uint8_t *pass_out);

/* Aggregate per-trajectory results (Sec. IV-C, last paragraph: the success
 * probability is the average of the criterion over the simulated states).
 * score (n doubles) and pass_flags (n bytes, may be NULL) are device
 * pointers; out[5] (host) = {mean score, pass fraction, stderr of the mean
 * score, stderr of the pass fraction, n}. FP64 sums in a fixed order. */
arso_status arso_aggregate(const double *score, const uint8_t *pass_flags, uint64_t n, void *stream, double *out);

/* Run the trajectories of many circuits of uneven sizes and depths in one
 * call (Sec. IV-B, Monte Carlo runs, for a batch of circuits). Every complex64
 * circuit (resident, and streaming with 13-qubit tiles) runs in ONE persistent
 * launch: CTAs pull work from a device queue in a dependency order: the
 * error-free score of each circuit (which the error-free trajectories take),
 * blocks of trajectories of resident circuits (2^(13-n) side by side in one CTA,
 * at most 32 below 10 qubits), and one pass of one trajectory of a streaming
 * circuit per tile. Streaming trajectories run in working slots (16 GiB in all,
 * split over the circuits by their work); a tile waits, with a bounded poll, for
 * its slot's previous pass. Circuits compiled with ARSO_OPT_NO_PERSISTENT,
 * complex128 circuits and streaming circuits with other tile sizes run their own
 * launches (resident launch or captured pass sequence). score_out[i] (n_traj of
 * errors[i] doubles) and pass_out[i] (bytes, or NULL; pass_out itself may be
 * NULL) are device or host pointers as in arso_run_trajectories. Scores equal
 * those of arso_run_trajectories bit for bit, except that error-free
 * trajectories take psi_R's score summed in another order (within rounding).
 * Errors: ARSO_EINVAL, ARSO_ENOMEM, ARSO_ECUDA, ARSO_ETIMEOUT (a dependency wait
 * gave up; no score of the call is valid). */
arso_status arso_run_batch(size_t count, arso_circuit *const *circuits, const arso_error_list *const *errors,
                           const arso_criterion *crits, void *stream, double *const *score_out,
                           uint8_t *const *pass_out);
/* Test support for the failure path of arso_run_batch's persistent launch (no
 * counterpart in the paper). A tile's wait for its slot's previous pass polls a
 * bounded number of times; one that gives up sets an error word, every CTA
 * leaves at its next queue pull, and the call returns ARSO_ETIMEOUT. This makes
 * the next persistent launch add 2^30 to every wait's target, with a short poll
 * limit, so that its first streaming tile's wait runs out: nothing hangs or
 * faults, and the next call on the same context runs normally. Only a batch
 * with a streaming circuit in the persistent launch waits at all. One-shot,
 * process-wide. */
arso_status arso_debug_stall_next_batch(void);

/* Autotune the fused-pass schedule of a circuit by measurement: for each
 * candidate (tile_qubits in 10..14, low_qubits in 3..5) compile the circuit,
 * time n_traj trajectories at uniform rate p (CUDA events on `stream`; best
 * of three runs after one warm-up run that also builds the prefix cache) and return the
 * fastest options in *best (precision and the other fields copied from
 * `base`, which may be NULL). ms_out (optional, capacity 16) receives each
 * candidate's time in candidate order, tile-major; *n_candidates their number.
 * Circuits that fit the resident engine have a single candidate. */
arso_status arso_autotune(uint32_t n_qubits, const arso_gate *gates, size_t n_gates, const arso_criterion *crit,
                          double p, uint64_t n_traj, uint64_t seed, const arso_compile_opts *base, void *stream,
                          arso_compile_opts *best, double *ms_out, uint32_t *n_candidates);

/* Final state vectors of trajectories [first, first + count) of `errors`
 * (count * 2^n amplitudes, device pointer, layout per the circuit's
 * precision). For parity checks and inspection. */
arso_status arso_trajectory_states(const arso_circuit *c, const arso_error_list *errors,
                                   uint64_t first, uint64_t count, void *stream, void *amps_out);
/* The error-free final state psi_R (2^n amplitudes, device pointer). */
arso_status arso_reference_state(const arso_circuit *c, void *stream, void *amps_out);

/* Success probability at error rate p, uniform p_X = p_Z = p_Y = p/3 (Sec. IV-C,
 * Fig. 2). mode AUTO follows the paper: Monte Carlo when the expected error
 * count L*p exceeds one, otherwise the exhaustive single-error analysis and
 * Eq. (4). */
enum { ARSO_MODE_AUTO = 0, ARSO_MODE_MONTE_CARLO = 1, ARSO_MODE_EXHAUSTIVE = 2 };
typedef struct {
    double value;           /* mean or pass fraction, per criterion.aggregate */
    double mean, pass_frac; /* MC: both aggregates; exhaustive: Eq. (4) of each */
    double stderr_value;    /* MC: sd / sqrt(n_traj) of `value`; exhaustive: 0 */
    double expected_errors; /* E(N) = L * p */
    uint32_t mode_used;
    uint64_t n_traj;        /* trajectories simulated */
    double P_R, P_X, P_Z, P_Y; /* exhaustive: Eq. (4) inputs (per aggregate) */
} arso_result;
arso_status arso_success_prob(const arso_circuit *c, const arso_criterion *crit, double p, uint32_t mode,
                              uint64_t n_traj, uint64_t seed, void *stream, arso_result *out);

/* Exhaustive single-error analysis (Sec. IV-B.1, Eq. (3)): psi_R and every
 * single X, Z, Y error at every location, 3L states. per_location (optional,
 * host, 3*L doubles ordered X block, Z block, Y block) receives the criterion
 * value of each state; P_out[4] = {P_R, P_X, P_Z, P_Y} (per aggregate). */
arso_status arso_exhaustive(const arso_circuit *c, const arso_criterion *crit, void *stream,
                            double *P_out, double *per_location);

/* Tolerable error rate (Sec. IV-D, Fig. 3) for target success P_target:
 * exhaustive analysis first; if P_target >= sum_e P_e / 3, Eq. (5) with
 * count L; otherwise Monte Carlo probes at successive p, bisected in log10 p on
 * common random numbers until hi/lo <= 1 + rel_tol, answer interpolated
 * log-linearly inside the final bracket. A surrogate (arso_surrogate_*) may
 * narrow the initial bracket; the plain simulator then verifies it. */
typedef struct arso_surrogate arso_surrogate;
typedef struct {
    double p_lo, p_hi;      /* search bracket (default 1e-6, 1e-1 when 0) */
    double rel_tol;         /* default 0.02 */
    uint64_t n_traj;        /* trajectories per probe (default 1000) */
    uint64_t seed;
    uint32_t max_probes;    /* default 64 */
    uint32_t mode;          /* ARSO_MODE_AUTO (Fig. 3) or ARSO_MODE_MONTE_CARLO (skip Eq. (5)) */
    const arso_surrogate *surrogate; /* NULL = plain search */
    const float *features;  /* surrogate inputs for this circuit (32 floats), with `surrogate` */
    double surrogate_margin;/* verify bracket half-width in log10 p (default 0.15) */
    uint32_t flags;         /* ARSO_SEARCH_NO_REUSE: simulate every trajectory of every probe */
} arso_search_opts;
/* Probes of one search draw the same random numbers, so the error sets of a
 * trajectory are nested in p; a trajectory with as many events at p as at an
 * earlier probe has the same events and its score is reused (exact). The
 * reuse applies to the register-blocked resident engine and the streaming
 * engine. */
#define ARSO_SEARCH_NO_REUSE 1u
typedef struct {
    double p, lo, hi, value_lo, value_hi;
    uint32_t probes;        /* plain-simulator probes */
    uint32_t mode_used;     /* 0 = Eq. (5), 1 = Monte Carlo search */
    uint32_t used_surrogate, verified, converged;
    double P1;              /* success subject to one average error */
} arso_rate_result;
arso_status arso_tolerable_rate(const arso_circuit *c, const arso_criterion *crit, double P_target,
                                const arso_search_opts *opts, void *stream, arso_rate_result *out);

/* ---- learned surrogate of the success probability (not part of the paper) ----
 * A 33 -> 256 -> 256 -> 1 MLP (ReLU hidden layers, sigmoid output) that maps
 * a circuit's features and log10 p to the probability that one trajectory
 * passes its criterion. Weights are bfloat16 with FP32 master copies; all
 * products accumulate in FP32. Training minimises the mean binary
 * cross-entropy against pass flags produced by arso_run_trajectories, with
 * Adam, entirely on the GPU. Inputs are standardised with the per-column mean
 * and standard deviation of the training set (stored in the handle).
 * It narrows the bracket of arso_tolerable_rate_surrogate; the plain
 * simulator verifies the bracket and remains the fallback.
 * The GEMMs run on the tensor cores (tcgen05, BF16 operands): FP32 activations
 * and gradients enter as three bf16 terms each, so products keep FP32 accuracy.
 * Gradients are summed in a fixed order (bit-reproducible). Errors: ARSO_EINVAL
 * for NULL pointers or sizes out of range (train: 1 <= n < 2^32, 1 <= batch <=
 * 65536; grads: 1 <= n <= 2^20), ARSO_ETIMEOUT if a GEMM's bounded wait gave
 * up, ARSO_ECUDA for a CUDA error. Device rows are caller-owned and only read. */
#define ARSO_N_FEATURES 32
#define ARSO_SURROGATE_INPUTS 33
/* 32 features of a compiled circuit and criterion (host floats): n, G, L, k,
 * m, depth, two-qubit layers, log10 L, log10 G, two-qubit fraction, counts of
 * H X Y Z S SDG T TDG RX RY RZ P U CX CZ CP SWAP U2, criterion one-hot (4). */
arso_status arso_circuit_features(const arso_circuit *c, const arso_criterion *crit, float *out);
arso_status arso_surrogate_create(uint64_t seed, arso_surrogate **out);
void arso_surrogate_free(arso_surrogate *s);
/* Train on n device rows x (n x 33 floats, row-major) with device labels y
 * (n floats in {0, 1}): `epochs` passes in shuffled mini-batches of `batch`
 * rows, Adam with learning rate lr. *loss_out (host, may be NULL) receives the
 * mean loss of the last epoch. The first call fixes the standardisation. */
arso_status arso_surrogate_train(arso_surrogate *s, const float *x, const float *y, uint64_t n, uint32_t epochs,
                                 uint32_t batch, double lr, uint64_t seed, void *stream, double *loss_out);
/* Predicted pass probabilities of n device rows into out (n device floats). */
arso_status arso_surrogate_predict(const arso_surrogate *s, const float *x, uint64_t n, float *out, void *stream);
/* Parameters as FP32 (host arrays, layout W1[33x256] b1[256] W2[256x256]
 * b2[256] W3[256] b3[1], row-major; ARSO_SURROGATE_PARAMS floats). set also
 * refreshes the bfloat16 copies; get returns the FP32 masters. */
#define ARSO_SURROGATE_PARAMS (33 * 256 + 256 + 256 * 256 + 256 + 256 + 1)
arso_status arso_surrogate_get_params(const arso_surrogate *s, float *out);
arso_status arso_surrogate_set_params(arso_surrogate *s, const float *in);
/* Standardisation (host, 33 means and 33 standard deviations). */
arso_status arso_surrogate_set_norm(arso_surrogate *s, const float *mean, const float *stdev);
/* Loss and gradients (host, ARSO_SURROGATE_PARAMS floats, same layout) of the
 * mean binary cross-entropy on n device rows, with the current bfloat16
 * weights; no update. For checking the backward kernels. */
arso_status arso_surrogate_grads(const arso_surrogate *s, const float *x, const float *y, uint64_t n, void *stream,
                                 float *grads_out, double *loss_out);
/* Test support for the failure path of the tensor-core GEMMs (no counterpart in
 * the paper). Every wait of those kernels on an mbarrier is bounded; one that
 * gives up skips the remaining MMAs, waits (again bounded) for any of its TMA
 * copies still in flight, frees its tensor memory, sets an error word and
 * returns, and the API call that launched it returns ARSO_ETIMEOUT. This makes
 * the next GEMM launch whose B operand comes by TMA arm its TMA barrier for the
 * operand's bytes but issue no copy, with a short wait limit, so that its wait
 * runs out with nothing outstanding; nothing hangs or faults and the context
 * stays usable. One-shot, process-wide. */
arso_status arso_debug_stall_next_gemm(void);
/* Tolerable rate with the surrogate (Sec. IV-D, Monte Carlo branch): bisect
 * log10 p on the surrogate's prediction for the circuit's features, take the
 * bracket [p_s 10^-m, p_s 10^m] (m = opts->surrogate_margin), verify it with
 * opts->n_traj plain trajectories at each end (values straddle P_target),
 * widen a failing side by 10^(2m), 10^(4m), 10^(8m) in turn, and if it still
 * fails move that side to the search range's end (opts->p_lo / p_hi); then
 * narrow the bracket to width 10^(2m) with plain probes (bisection in log p
 * while wider than four such widths, then probes at the log-linear
 * interpolation point kept inside the middle 60%; at most 24), and answer by
 * log-linear interpolation inside it. All probes share one set of random
 * numbers and reuse each other's trajectories. out->verified = 1 when the
 * surrogate's (widened) bracket held, 0 when the range ends were needed.
 * Errors: ARSO_ENOTCONVERGED when even [p_lo, p_hi] does not bracket the
 * target. */
arso_status arso_tolerable_rate_surrogate(const arso_circuit *c, const arso_criterion *crit, double P_target,
                                          const arso_search_opts *opts, void *stream, arso_rate_result *out);

/* ---- single-step kernels (each also runs inside the fused trajectory path) ---- */

/* Apply one gate to a device state (2^n amplitudes, complex64) as a strided
 * pair/quad update over HBM (Sec. II: a gate manipulates the amplitudes). */
arso_status arso_apply_gate(uint32_t n_qubits, void *amps, const arso_gate *gate, void *stream);
/* Apply the Pauli error gate `code` on `qubit` (Eq. (2)) to a device state
 * (complex64): X/Y as an index permutation, Z/Y as a phase. */
arso_status arso_apply_pauli(uint32_t n_qubits, void *amps, uint32_t qubit, uint32_t code, void *stream);
/* Score one device state (complex64) against `crit`; ref (complex64, device)
 * is psi_R for fidelity and ignored otherwise. FP64 accumulation. *score_out
 * is a host double. */
arso_status arso_score_state(uint32_t n_qubits, const void *amps, const void *ref,
                             const arso_criterion *crit, void *stream, double *score_out);

/* Allocation-free variant of arso_score_state (the paper has no counterpart:
 * this serves callers that cannot call cudaMalloc, such as code running inside
 * another framework's memory arena or on a path where an allocation would
 * synchronise the device or fail under memory pressure). Same arguments and
 * result as arso_score_state; its scratch lives in fixed-size device arrays
 * compiled into the library, which every GPU that loads the library holds
 * until the process exits. Limits: binning criteria up to 20 qubits (an
 * outcome bitmap of 2^20 bits), other criteria up to 34 qubits; larger
 * requests return ARSO_EINVAL. Every call looks up the arrays' device
 * addresses in the context current on the calling thread (no allocation, and
 * no cached address that a device reset could leave stale); the first call in
 * a context loads the library's module there, so make it before any stream
 * capture. All calls in a context share the arrays (each call overwrites what
 * it reads), so calls that overlap on the GPU race. It calls no cudaMalloc or
 * cudaFree. */
arso_status arso_score_state_noalloc(uint32_t n_qubits, const void *amps, const void *ref,
                                     const arso_criterion *crit, void *stream, double *score_out);

/* ---- tracing: per-kernel device time and traffic (not part of the paper) ----
 * When enabled, the library records a CUDA event pair on the launching stream
 * around every kernel launch and accumulates, per kernel family, the number
 * of launches, their summed device time and the algorithmic bytes they move
 * (the reads and writes the algorithm requires, not cache-level traffic).
 * Streaming passes also count algorithmic flops: per amplitude and gate, 14
 * for a dense one-qubit gate (2x2 complex matrix-vector product), 30 for a
 * dense two-qubit gate, 6 for a diagonal gate, 4 for H, 2 for an odd power
 * of the T phase and 0 for permutations and sign flips (X, CX, SWAP, CZ, Z,
 * S), times the amplitudes each launch sweeps.
 * Launch and host<->device transfer counters run whether or not timing is
 * enabled. Process-wide, thread-safe; reading resolves pending events. */
enum {
    ARSO_K_PASS = 0,        /* streaming pass, state written back to HBM */
    ARSO_K_PASS_LAST = 1,   /* last streaming pass, fused criterion reduction */
    ARSO_K_RESIDENT = 2,    /* resident whole-state trajectory kernel */
    ARSO_K_SAMPLE = 3,      /* Philox error sampling (count + fill) */
    ARSO_K_REDUCE = 4,      /* criterion partials, finish, sums */
    ARSO_K_OTHER = 5,       /* bookkeeping kernels (scan, sort, fill, init) */
    ARSO_K_GEMM = 6,        /* surrogate MLP GEMMs on the tensor cores */
    ARSO_K_MIX = 7,         /* persistent launch of a batch of uneven circuits (arso_run_batch) */
    ARSO_K_COUNT = 8
};
typedef struct {
    uint64_t launches;
    double ms;              /* summed device time (timing enabled only) */
    double bytes;           /* summed algorithmic bytes (timing enabled only) */
    double flops;           /* summed algorithmic flops (timing enabled only): FP32 flops of the
                               register-blocked passes and persistent-batch work (per amplitude and
                               gate as above), and 2 M N K per M x N x K surrogate GEMM; 0 for other
                               kernels */
    double smem_bytes;      /* summed algorithmic shared-memory bytes (timing enabled only): per
                               register-set change of the register-blocked kernels, one write and one
                               read of the 2^n amplitudes (16 bytes each); per gate of the shared-memory
                               gate engine (below 10 qubits), one read and one write of the state */
} arso_kernel_stats;
arso_status arso_profile_enable(int on);
arso_status arso_profile_reset(void);
arso_status arso_profile_read(uint32_t kernel, arso_kernel_stats *out);
/* Total kernel launches and bytes copied host->device / device->host by the
 * library since the last reset. */
arso_status arso_profile_counters(uint64_t *launches, uint64_t *h2d_bytes, uint64_t *d2h_bytes);

const char *arso_last_error(void);
const char *arso_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ARSO_H */
