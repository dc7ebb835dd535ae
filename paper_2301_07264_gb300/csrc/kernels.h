// Kernel argument blocks and launcher declarations (host <-> device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace arso {

// Per-tile partial of a criterion. Fidelity: (a, b) = sum conj(R) psi.
// Outcome / binning: a = sum |psi|^2 over the selected outcomes. Argmax:
// (maxp, idx), the lowest index winning ties.
struct Partial {
    double a, b;
    double maxp;
    unsigned long long idx;
};

// Device view of a criterion.
struct DCrit {
    uint32_t kind;
    double threshold;
    unsigned long long target;
    const uint32_t *bitmap;  // binning set, 2^n bits (device)
};

struct ResidentArgs {
    int n;
    uint32_t G;
    const DGate *gates;
    const void *mats;
    const void *cache;           // n_ckpt states; entry c = after gates [0, c*every); last = psi_R
    uint64_t ckpt_every;
    uint32_t n_ckpt;
    // trajectories [first_traj, first_traj + count) of the error list, or, with
    // ids (register-blocked kernel only), the trajectories ids[0 .. count)
    uint64_t first_traj, count;
    const uint64_t *ids;
    const uint64_t *offsets;
    const uint32_t *keys;
    const uint32_t *first;       // per trajectory: engine position of the first event or NO_EVENT
    DCrit crit;
    const double *ref_score;     // device scalar: score of psi_R
    double *score;               // device, indexed by trajectory
    uint8_t *pass_flags;         // device or null
    void *states_out;            // non-null: store final states (count * 2^n) instead of scoring
    // register-blocked execution: checkpoints sit at phase boundaries
    uint32_t n_phases;
    const uint32_t *ph_gb, *ph_R;
    const RegOp *rops;
    const uint32_t *phase_of_pos;  // gate position -> phase
};

// mode: 0 = score trajectories, 1 = store final states, 2 = error-free run filling the cache
void launch_resident_rb(const ResidentArgs &a, int mode, double bytes, cudaStream_t st);

struct PassArgs {
    int n, t, c;                 // qubits, tile qubits, contiguous low qubits
    uint64_t rest_mask;          // global bits outside the tile
    const uint32_t *offs;        // 2^(t-c) offsets of the tile's high part
    uint32_t gb, ge;             // gate range (engine order)
    int pass;
    const DGate *gates;
    const void *mats;
    // ideal (error-free) mode: one slot from ideal_src to ideal_dst
    int ideal;
    const void *ideal_src;
    void *ideal_dst;
    // trajectory mode
    const void *cache;           // cached boundary states
    const void *ref_cache;       // states the end pass is scored against, at the same entries
                                 // (NULL: cache; backward states for the outcome criterion)
    const uint32_t *cache_slot;  // pass index -> cache entry (valid for cached boundaries)
    uint32_t ref_slot;           // cache entry of psi_R
    void *work;                  // slots * 2^n working states
    const int *start_pass;       // per slot
    const int *end_pass;         // per slot: the pass whose output is scored, against the cached
                                 // error-free state at the boundary after it (psi_R for the last pass)
    const uint64_t *slot_traj;   // per slot: trajectory index in the error list
    const uint64_t *offsets;
    const uint32_t *keys;
    DCrit crit;
    Partial *partials;           // last pass: slots * tiles
    int store_last;              // last pass stores the state instead of reducing
    // register-blocked execution
    uint32_t pb, pe;             // phases of this pass
    const uint32_t *ph_gb;       // phase -> first engine position (with sentinel)
    const uint32_t *ph_R;        // phase -> packed register bits
    const RegOp *rops;           // engine position -> register-kernel gate record
    // tensor-core phases (NULL: every phase runs gate by gate)
    const uint32_t *ph_t;        // phase -> operand-image index or NO_TENSOR
    const void *tmats;           // TENSOR_IMAGE_HALVES fp16 values per image
    uint32_t *terr;              // set when a wait for the tensor cores gave up
};

void launch_pass_rb(const PassArgs &a, bool last, uint32_t slots, double bytes, cudaStream_t st, double flops = 0.0,
                    double smem_bytes = 0.0);
void prepare_pass_rb();

// Batched resident execution: one persistent launch over (circuit, trajectory
// block) items of many register-blocked resident circuits (10 <= n <= 13).
struct BatchCircuit {
    int n;
    uint32_t n_phases, n_ckpt, ckpt_every;
    const DGate *gates;
    const float2 *mats;
    const uint32_t *ph_gb, *ph_R, *phase_of_pos;
    const RegOp *rops;
    const float2 *cache;
    const uint64_t *offsets;
    const uint32_t *keys;
    DCrit crit;
    double *score;
    uint8_t *pass_flags;
};
struct BatchItem {
    uint32_t circuit;   // index into the circuit descriptors
    uint32_t count;     // trajectories in this item (<= 2^(13 - n))
    uint32_t ck;        // checkpoint every trajectory of the item starts from
    uint32_t pad;
    uint64_t off;       // first entry in the trajectory-id array
};
void launch_batch_resident(const BatchCircuit *circs, const BatchItem *items, uint32_t n_items, uint32_t *counter,
                           const uint64_t *ids, double bytes, cudaStream_t st);

// Persistent launch over the work of many circuits of uneven size (one launch
// per arso_run_batch call). The work is a list of units; CTAs take sub-items
// from one counter in list order:
//  MIX_REF   error-free score of one circuit, one sub-item per 2^13-amplitude
//            chunk of psi_R; the last chunk fills the circuit's error-free
//            trajectories;
//  MIX_SMALL a batched item of a resident circuit below 2^10 amplitudes (shared-
//            memory gate engine, up to 32 trajectories side by side);
//  MIX_RES   a batched register-blocked resident item (BatchItem above);
//  MIX_STR   one pass of one trajectory of a streaming circuit, one sub-item per
//            tile; its dependencies (the trajectory's previous pass, or the slot's
//            previous trajectory) are per-slot counters of finished tiles, and the
//            list is ordered so that every unit's dependencies come before it.
enum : uint32_t { MIX_REF = 0, MIX_SMALL = 1, MIX_RES = 2, MIX_STR = 3 };
struct MixUnit {
    uint32_t kind;
    uint32_t idx;  // REF: reference descriptor; SMALL / RES: item; STR: stream descriptor
    uint32_t a, b; // STR: trajectory (index in the stream's table), pass
};
struct MixRef {
    int n;
    uint32_t chunks;         // ceil(2^n / 2^13)
    const float2 *psi_R;
    DCrit crit;
    const uint32_t *first;   // per trajectory: first event position or NO_EVENT
    uint64_t n_traj;
    Partial *partials;       // per chunk
    uint32_t *done;          // chunks finished (zeroed before the launch)
    double *score;
    uint8_t *pass_flags;
};
struct MixSmall {            // resident circuit of n <= 9 qubits, gate-indexed checkpoints
    int n;
    uint32_t G, ckpt_every, n_ckpt;
    const DGate *gates;
    const float2 *mats;
    const float2 *cache;
    const uint64_t *offsets;
    const uint32_t *keys;
    DCrit crit;
    double *score;
    uint8_t *pass_flags;
};
struct MixPass {
    uint64_t rest_mask;      // global bits outside the pass's tiles
    const uint32_t *offs;    // tile-high offsets of the pass
    uint32_t gb, pb, pe, pad;
};
struct MixTraj {
    uint64_t tr;             // trajectory index in the error list
    uint32_t slot;           // working slot
    uint32_t base;           // tiles the slot finished before this trajectory's first pass
    int start, end;          // first pass (from the cached boundary before it) and scored pass
};
struct MixStream {
    int n, t, c;
    uint32_t tiles;
    const MixPass *passes;
    const uint32_t *ph_gb, *ph_R;
    const RegOp *rops;
    const float2 *mats;
    const float2 *cache;       // cached error-free boundary states
    const float2 *ref_cache;   // states the scored pass is compared with, same entries
    const uint32_t *cache_slot;
    float2 *work;              // slots x 2^n
    uint32_t *slot_done;       // per slot: tiles finished (zeroed before the launch)
    const uint64_t *offsets;
    const uint32_t *keys;
    const MixTraj *trajs;
    Partial *partials;         // per trajectory x tiles
    uint32_t *traj_done;       // per trajectory: tiles of its scored pass finished (zeroed)
    DCrit crit;
    double *score;
    uint8_t *pass_flags;
};
struct MixArgs {
    const MixUnit *units;
    const uint64_t *unit_end;  // inclusive prefix sums of the sub-items per unit
    uint32_t n_units;
    uint64_t n_sub;
    const MixRef *refs;
    const MixSmall *smalls;
    const BatchCircuit *rcircs;
    const BatchItem *items;    // SMALL items index smalls, RES items index rcircs
    const uint64_t *ids;
    const MixStream *streams;
    unsigned long long *counter;
    uint32_t *err;             // bit 0: a dependency wait gave up
    uint32_t wait_limit;       // polls per wait
    uint32_t stall_extra;      // added to every wait's target: 0, except in the failure-path test
};
constexpr uint32_t MIX_SMALL_MAX = 32;  // trajectories per SMALL item
void launch_mix(const MixArgs &a, double bytes, double flops, double smem_bytes, cudaStream_t st);

void launch_resident(const ResidentArgs &a, bool ideal, int precision, double bytes, cudaStream_t st);
void launch_pass(const PassArgs &a, bool last, int precision, uint32_t slots, double bytes, cudaStream_t st);
void launch_finish_partials(const Partial *partials, uint32_t tiles, uint32_t slots, const uint64_t *slot_traj,
                            const DCrit &crit, double *score, uint8_t *pass_flags, cudaStream_t st);
void launch_fill_error_free(const uint32_t *first, uint64_t n_traj, const double *ref_score, double threshold,
                            double *score, uint8_t *pass_flags, cudaStream_t st);
struct M16 {
    float2 m[16];
};
void launch_gate_pairs(float2 *psi, int n, const DGate &g, const M16 &m, cudaStream_t st);
void launch_pauli(float2 *psi, int n, uint32_t q, uint32_t code, cudaStream_t st);
uint32_t launch_score_partials(const void *psi, const void *ref, int n, int precision, const DCrit &crit,
                               Partial *partials, uint32_t max_blocks, cudaStream_t st);
void launch_init_zero_state(void *psi, int n, int precision, cudaStream_t st);
// Pauli expectations (<X_q>, <Z_q>, <Y_q>) of the error-free state after each
// gate: resident circuits run one CTA per cached checkpoint segment
// (engine positions seg_pos[b] .. seg_pos[b + 1]; out[3 * location + k]), or a
// complex64 state in HBM (launch_gate_expect below).
void launch_expect_resident(const DGate *gates, const void *mats, int n, int precision, const void *ckpt,
                            const uint32_t *seg_pos, uint32_t n_seg, const uint32_t *first_loc, double *out,
                            cudaStream_t st);
uint32_t expect_hbm_blocks(int n);
// One gate fused with the expectations of its qubits on the updated state; block
// partials at partials + pos * expect_hbm_blocks(n) * 6 (the caller offsets), added
// in order by launch_gate_expect_reduce for `count` positions (block k: position k,
// locations loc[k] .. loc[k] + arity[k] - 1).
void launch_gate_expect(float2 *psi, int n, const DGate &g, const M16 &m, double *partials, cudaStream_t st);
void launch_gate_expect_reduce(const double *partials, uint32_t count, uint32_t blocks, const uint32_t *loc,
                               const uint8_t *arity, double *out3, cudaStream_t st);

// Backward single-error sweep for rank-1 criteria (outcome probability): psi and
// phi carried backward from (psi_R, |target>) with the adjoint gates; out6[6 * location
// + k] = (Re, Im) of <phi|X|psi>, <phi|Z|psi>, <phi|Y|psi> after the location's gate.
// Resident: one CTA, both states in shared memory, adj[pos] the adjoint gate at
// engine position pos (global qubits). HBM (complex64): one launch per gate with
// partials at partials + pos * expect_hbm_blocks(n) * 12 (the caller offsets), added
// in order by launch_dual_expect_reduce.
void launch_dual_expect_resident(const DGate *adj, const void *mats, uint32_t G, int n, int precision,
                                 const void *psi_R, uint64_t target, const uint32_t *first_loc, double *out6,
                                 cudaStream_t st);
void launch_dual_gate_expect(float2 *psi, float2 *phi, int n, const DGate &g, const M16 &m, double *partials,
                             cudaStream_t st);
void launch_dual_expect_reduce(const double *partials, uint32_t count, uint32_t blocks, const uint32_t *loc,
                               const uint8_t *arity, double *out6, cudaStream_t st);

// sampling (sample.cu)
struct SampleArgs {
    uint64_t seed, traj_begin, n_traj;
    uint32_t L;
    uint32_t thr, cut_x, cut_xz;  // cut_* saturate at 2^32 - 1 + carry handled via flags
    uint32_t cut_x_all, cut_xz_all; // 1 if the cut equals 2^32 (every draw below it)
};
void launch_sample_count(const SampleArgs &a, uint32_t *counts, cudaStream_t st);
// Batched sampling: one job per error list, trajectories numbered globally
// (job j owns [traj0, traj0 + a.n_traj)); counts are concatenated in that order.
struct SampleJob {
    SampleArgs a;
    uint64_t traj0;
    uint64_t *offsets;          // the list's offsets[n_traj + 1]
    const uint32_t *loc_key;    // the circuit's location -> engine key table
    uint32_t *ev_loc, *ev_key;  // the list's events (set after the counts are known)
    uint32_t *first, *last;
    uint32_t identity;          // the schedule keeps circuit order: keys need no sort
};
// count kernel and per-job scans (totals[j] = events of job j)
void launch_sample_batch_count(const SampleJob *jobs, uint32_t n_jobs, uint64_t n_total, uint32_t *counts,
                               uint64_t *totals, cudaStream_t st);
// event fill (when any job has events) and per-trajectory sort / first and last event
void launch_sample_batch_fill(const SampleJob *jobs, uint32_t n_jobs, uint64_t n_total, bool any_events,
                              cudaStream_t st);
void launch_exclusive_scan(const uint32_t *counts, uint64_t n, uint64_t *offsets, cudaStream_t st);
void launch_sample_fill(const SampleArgs &a, const uint64_t *offsets, const uint32_t *loc_key, uint32_t *ev_loc,
                        uint32_t *ev_key, cudaStream_t st);
void launch_keys_from_loc(const uint32_t *ev_loc, uint64_t n_events, const uint32_t *loc_key, uint32_t *ev_key,
                          cudaStream_t st);
void launch_sort_keys(const uint64_t *offsets, uint64_t n_traj, uint32_t *ev_key, cudaStream_t st);
void launch_first_event(const uint64_t *offsets, uint64_t n_traj, const uint32_t *ev_key, uint32_t *first,
                        uint32_t *last, cudaStream_t st);
void launch_sum_scores(const double *score, const uint8_t *pass_flags, uint64_t n, double *sums3, cudaStream_t st);

}  // namespace arso
