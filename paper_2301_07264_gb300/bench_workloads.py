"""Measurements of the workloads other than the default benchmark line
(used by bench.py --workload ...): the Grover-12 error-rate sweep, the
256-circuit uneven batch, and the surrogate-bracketed tolerable-rate search.
Every measured step runs through the C ABI; this module arranges calls."""
from __future__ import annotations

import math
import time

import numpy as np


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _kernel_stats(arso):
    names = (("pass", arso.K_PASS), ("pass_last", arso.K_PASS_LAST), ("resident", arso.K_RESIDENT),
             ("sample", arso.K_SAMPLE), ("reduce", arso.K_REDUCE), ("other", arso.K_OTHER), ("gemm", arso.K_GEMM),
             ("mix", arso.K_MIX))
    out = {}
    for name, k in names:
        st = arso.profile_read(k)
        out[name] = {"launches": st.launches, "ms": st.ms, "GB": st.bytes / 1e9, "TFLOP": st.flops / 1e12,
                     "smem_GB": st.smem_bytes / 1e9}
    return out


def grover12(args):
    """Grover (11 search qubits + 1 borrowed), argmax criterion, 16 rates
    logspace(1e-5, 1e-2); a step runs traj_per_step trajectories at every rate."""
    import torch
    from paper_2301_07264_gb300 import arso
    from workloads import circuits as W
    circ = W.grover12(0)
    cc = arso.compile_circuit(circ.n, circ.gates)
    crit = arso.make_criterion(circ.criterion)
    rates = np.logspace(-5, -2, 16)
    per = max(1, args.traj_per_step // 16)
    stream = torch.cuda.current_stream()
    res = np.zeros(16)

    scores = [torch.empty(per, dtype=torch.float64, device="cuda") for _ in rates]
    flag_l = [torch.empty(per, dtype=torch.uint8, device="cuda") for _ in rates]

    def step(k):
        # all 16 rates: one batched sampling call and one persistent launch (arso_run_batch)
        errs = arso.sample_errors_batch([cc] * len(rates), rates / 3, rates / 3, rates / 3, 0, k * per, per, stream)
        arso.run_batch([cc] * len(rates), errs, [crit] * len(rates), scores, flag_l, stream)
        for i in range(len(rates)):
            res[i] += arso.aggregate(scores[i], flag_l[i], stream)[1]

    for w in range(args.warmup):
        step(1000 + w)
    res[:] = 0
    arso.profile_reset()
    arso.profile_enable(True)
    e0, e1 = _events()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    arso.profile_enable(False)
    sec = e0.elapsed_time(e1) / 1e3
    total = per * 16 * args.steps
    info = cc.info()
    mx = arso.profile_read(arso.K_MIX)
    return {"metric": "error-injected trajectories/sec", "value": total / sec, "unit": "traj/s",
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "grover12_sweep", "n_qubits": 12, "G": info.G, "L": info.L,
                       "rates": "16 log-spaced in [1e-5, 1e-2]", "traj_per_rate_per_step": per,
                       "criterion": "argmax == marked",
                       "engine": "resident (whole state in one CTA), all rates in one persistent launch"},
            "results": {"pass_frac": (res / args.steps).round(4).tolist()},
            # on-chip roof inputs: the persistent launch's algorithmic FP32 flops and
            # shared-memory bytes over its device time (bench.py adds the peaks)
            "onchip": {"kernel": "mix_kernel (batched resident items)", "ms": mx.ms, "flops": mx.flops,
                       "smem_bytes": mx.smem_bytes, "launches": mx.launches},
            "kernels": _kernel_stats(arso)}


def qft4(args):
    """The 4-qubit QFT on |0101> (complex128, resident engine), Pauli errors at
    p = 1e-3 after every gate, 1,000 trajectories from seed 0 per step, fidelity
    with the ideal output state >= 0.5 (pass fraction)."""
    import torch
    from paper_2301_07264_gb300 import arso
    from workloads import circuits as W
    circ = W.qft4_0101()
    cc = arso.compile_circuit(circ.n, circ.gates, precision=arso.C128)
    p, T = 1e-3, 1000
    score = torch.empty(T, dtype=torch.float64, device="cuda")
    flags = torch.empty(T, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    res = []

    def step(k):
        errs = arso.sample_errors(cc, p / 3, p / 3, p / 3, 0, k * T, T, stream)
        arso.run_trajectories(cc, errs, circ.criterion, score, flags, stream)
        res.append(arso.aggregate(score, flags, stream))

    for w in range(args.warmup):
        step(1000 + w)
    res.clear()
    e0, e1 = _events()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    return {"metric": "error-injected trajectories/sec", "value": T * args.steps / sec, "unit": "traj/s",
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "qft4_0101_p1e-3", "n_qubits": 4, "G": circ.G, "L": circ.L,
                       "traj_per_step": T, "criterion": "fidelity >= 0.5 (pass fraction)", "precision": "complex128"},
            "results": {"first_step_pass_frac": res[0][1], "first_step_mean_fidelity": res[0][0]}}


def mix256(args):
    """256 circuits of 8..22 qubits (QFT, Grover, QAOA p=2, adders) at p = 5e-4,
    2000 trajectories each per step: one arso_sample_errors_batch call and one
    arso_run_batch call per step (the batch runs as one persistent launch)."""
    import torch
    from paper_2301_07264_gb300 import arso
    from workloads import circuits as W
    mix = W.mix_family(0)
    p, T = 5e-4, 2000
    ccs = [arso.compile_circuit(c.n, c.gates) for c in mix]
    crits = [c.criterion for c in mix]
    outs = [torch.empty(T, dtype=torch.float64, device="cuda") for _ in mix]
    stream = torch.cuda.current_stream()

    def step(k):
        errs = arso.sample_errors_batch(ccs, p / 3, p / 3, p / 3, 0, k * T, T, stream)
        arso.run_batch(ccs, errs, crits, outs, None, stream)

    for w in range(args.warmup):
        step(1000 + w)
    arso.profile_reset()
    arso.profile_enable(True)
    e0, e1 = _events()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    arso.profile_enable(False)
    sec = e0.elapsed_time(e1) / 1e3
    launches, _, _ = arso.profile_counters()
    fams = {f: sum(1 for c in mix if c.family == f) for f in ("qft", "grover", "qaoa", "adder")}
    return {"metric": "error-injected trajectories/sec", "value": len(mix) * T * args.steps / sec,
            "unit": "traj/s", "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "mix256_p5e-4", "circuits": len(mix), "families": fams,
                       "n_range": [min(c.n for c in mix), max(c.n for c in mix)],
                       "traj_per_circuit": T, "tile_qubits": 13},
            "gpu_launches_per_step": launches / args.steps,
            "mean_score": float(np.mean([float(o.mean()) for o in outs])),
            "kernels": _kernel_stats(arso)}


def _search_band(n):
    return "12-14 (trained sizes)" if n <= 14 else ("16-18 (trained sizes)" if n <= 18 else "20-24 (extrapolated)")


def search(args):
    """Tolerable rate (pass fraction >= 2/3 of fidelity >= 0.9) of unseen QAOA (p = 2)
    and brickwork circuits of 12-24 qubits: plain Monte Carlo bisection against the
    surrogate bracket with plain verification, both with 20,000 trajectories per
    probe on the same random numbers and the same range of p. The network is
    trained on simulator rows of 8-18-qubit circuits of the same families; results
    are reported per size band (12-14 and 16-18 trained, 20-24 extrapolated)."""
    import torch
    from paper_2301_07264_gb300 import arso, surrogate_data
    from workloads import circuits as W
    rng = np.random.default_rng(1)
    fam_train = []
    for k in range(180):
        n = int(rng.integers(4, 10)) * 2
        if k % 2:
            fam_train.append(W.qaoa_maxcut(n, 1000 + k))
        else:
            fam_train.append(W.brickwork(n, int(rng.integers(4, 24)), 1000 + k))
    for c in fam_train:
        c.criterion = W.Criterion("fidelity", threshold=0.9, aggregate="pass")
    t0 = time.perf_counter()
    x, y = surrogate_data.generate(fam_train, args.train_rows, seed=1, lp_lo=-5.0, lp_hi=-1.0, p_points=32)
    gen_s = time.perf_counter() - t0
    s = arso.surrogate_create(11)
    t0 = time.perf_counter()
    loss = arso.surrogate_train(s, x, y, epochs=args.search_epochs, batch=8192, lr=2e-3, seed=3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # the tensor-core GEMMs' share of one profiled training epoch (a fresh network, so the
    # timed run above is undisturbed): per-launch CUDA events on the library's stream
    probe = arso.surrogate_create(12)
    m = min(int(x.shape[0]), 262144)
    arso.profile_reset()
    arso.profile_enable(True)
    arso.surrogate_train(probe, x[:m], y[:m], epochs=1, batch=8192, lr=2e-3, seed=3)
    torch.cuda.synchronize()
    arso.profile_enable(False)
    ks = {name: arso.profile_read(k) for name, k in (("gemm", arso.K_GEMM), ("reduce", arso.K_REDUCE),
                                                    ("other", arso.K_OTHER))}
    total_ms = sum(v.ms for v in ks.values())
    gemm = ks["gemm"]
    train_info = {"rows": int(x.shape[0]), "epochs": args.search_epochs, "batch": 8192, "seconds": train_s,
                  "rows_per_s": 4 * int(x.shape[0]) / train_s,
                  "profiled_rows": m,
                  "gemm": {"kernel": "umma_gemm_kernel (tcgen05 kind::f16, TMEM accumulator)",
                           "launches": gemm.launches, "ms": gemm.ms, "share": gemm.ms / total_ms if total_ms else None,
                           "useful_tflops": gemm.flops / gemm.ms / 1e9 if gemm.ms else None},
                  "reduce_ms": ks["reduce"].ms, "other_ms": ks["other"].ms}
    # ablation: a network trained only on the three circuits of the other configurations
    # (QFT-4 on |0101>, Grover-12, brickwork-24), the literal reading of the training set
    s_abl, abl_info = None, None
    if args.search_ablation:
        lit = [W.qft4_0101(), W.grover12(0), W.brickwork24(0)]
        rows_per = [40_000, 40_000, 10_000]  # a 24-qubit row is a 24-qubit trajectory
        t0 = time.perf_counter()
        xs, ys = [], []
        for k, (c, nr) in enumerate(zip(lit, rows_per)):
            x_, y_ = surrogate_data.generate([c], nr, seed=40 + k, lp_lo=-5.0, lp_hi=-1.0, p_points=32)
            xs.append(x_)
            ys.append(y_)
        xa, ya = torch.cat(xs), torch.cat(ys)
        gen_a = time.perf_counter() - t0
        s_abl = arso.surrogate_create(13)
        loss_a = arso.surrogate_train(s_abl, xa, ya, epochs=80, batch=8192, lr=2e-3, seed=3)
        abl_info = {"train_circuits": ["qft4_0101", "grover12", "brickwork24"], "rows": int(xa.shape[0]),
                    "generate_seconds": gen_a, "train_loss": loss_a}
    # evaluation circuits, unseen: per band, alternating QAOA and brickwork
    rng = np.random.default_rng(2)
    nb = max(1, args.search_circuits)
    n_large = args.search_large if args.search_large > 0 else max(1, nb // 2)
    sizes = [(12, 14)] * nb + [(16, 18)] * nb + [(20, 22, 24)] * n_large
    evals = []
    for k, choice in enumerate(sizes):
        n = choice[k % len(choice)]
        c = W.qaoa_maxcut(n, 5000 + k) if k % 2 else W.brickwork(n, int(rng.integers(10, 41)), 5000 + k)
        evals.append(c)
    crit = W.Criterion("fidelity", threshold=0.9, aggregate="pass")
    p_lo, p_hi = 1e-5, 1e-2
    rows = []
    for c in evals:
        cc = arso.compile_circuit(c.n, c.gates)
        arso.success_prob(cc, crit, 1e-3, mode="mc", n_traj=256, seed=0)  # builds the prefix cache
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pl = arso.tolerable_rate(cc, crit, 2 / 3, n_traj=20000, seed=0, mode="mc", rel_tol=0.02, p_lo=p_lo,
                                 p_hi=p_hi)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        su = arso.tolerable_rate_surrogate(cc, crit, 2 / 3, s, n_traj=20000, seed=0, margin=args.search_margin,
                                           p_lo=p_lo, p_hi=p_hi)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        row = {"family": c.family, "n": c.n, "G": c.G, "L": c.L, "band": _search_band(c.n),
               "p_plain": pl.p, "probes_plain": pl.probes, "plain_s": t1 - t0,
               "p_surrogate": su.p, "probes_surrogate": su.probes, "surrogate_s": t2 - t1,
               "verified": su.verified, "rel_err": abs(su.p - pl.p) / pl.p}
        if s_abl is not None and c.n <= 18:
            t3 = time.perf_counter()
            ab = arso.tolerable_rate_surrogate(cc, crit, 2 / 3, s_abl, n_traj=20000, seed=0,
                                               margin=args.search_margin, p_lo=p_lo, p_hi=p_hi)
            torch.cuda.synchronize()
            row["ablation"] = {"p": ab.p, "probes": ab.probes, "seconds": time.perf_counter() - t3,
                               "verified": ab.verified, "rel_err": abs(ab.p - pl.p) / pl.p}
        rows.append(row)
    bands = {}
    for b in sorted({r["band"] for r in rows}):
        rs = [r for r in rows if r["band"] == b]
        pl_s, su_s = sum(r["plain_s"] for r in rs), sum(r["surrogate_s"] for r in rs)
        rel = [r["rel_err"] for r in rs]
        bands[b] = {"circuits": len(rs), "qubits": sorted({r["n"] for r in rs}),
                    "plain_searches_per_s": len(rs) / pl_s, "surrogate_searches_per_s": len(rs) / su_s,
                    "speedup": pl_s / su_s, "rel_err_max": max(rel), "rel_err_mean": float(np.mean(rel)),
                    "rel_err_p50_p90_p99": [float(np.percentile(rel, q)) for q in (50, 90, 99)],
                    "verified": sum(r["verified"] for r in rs),
                    "probes_plain_mean": float(np.mean([r["probes_plain"] for r in rs])),
                    "probes_surrogate_mean": float(np.mean([r["probes_surrogate"] for r in rs]))}
    if abl_info is not None:
        ra = [r for r in rows if "ablation" in r]
        abl_info.update({"circuits": len(ra), "qubits": "12-18",
                         "speedup": sum(r["plain_s"] for r in ra) / sum(r["ablation"]["seconds"] for r in ra),
                         "speedup_main_network_same_circuits":
                             sum(r["plain_s"] for r in ra) / sum(r["surrogate_s"] for r in ra),
                         "probes_mean": float(np.mean([r["ablation"]["probes"] for r in ra])),
                         "verified": sum(r["ablation"]["verified"] for r in ra),
                         "rel_err_max": max(r["ablation"]["rel_err"] for r in ra)})
    plain_s, sur_s = sum(r["plain_s"] for r in rows), sum(r["surrogate_s"] for r in rows)
    rel = [r["rel_err"] for r in rows]
    return {"metric": "tolerable-rate searches/sec", "value": len(evals) / sur_s, "unit": "searches/s",
            "higher_is_better": True, "dtype": "f32/bf16", "data": "synthetic",
            "config": {"workload": "surrogate_search", "eval_circuits": len(evals),
                       "eval_qubits": sorted({c.n for c in evals}), "train_qubits": "8-18",
                       "train_rows": int(x.shape[0]), "train_circuits": len(fam_train), "verify_traj": 20000,
                       "p_range": [p_lo, p_hi], "margin_log10": args.search_margin,
                       "target": "pass fraction >= 2/3 (fidelity >= 0.9)"},
            "plain_searches_per_s": len(evals) / plain_s, "speedup": plain_s / sur_s,
            "rel_err_max": max(rel), "rel_err_mean": float(np.mean(rel)),
            "rel_err_p50_p90_p99": [float(np.percentile(rel, q)) for q in (50, 90, 99)],
            "verified": sum(r["verified"] for r in rows), "bands": bands, "ablation_literal_training_set": abl_info,
            "train_loss": loss,
            "generate_seconds": gen_s, "train_seconds": train_s, "surrogate_train": train_info, "rows": rows}


def exhaustive(args):
    """Exhaustive single-error analysis (Sec. IV-B.1, all 3L single-error states):
    fidelity by the error-free sweep of Pauli expectations (brickwork-24, Grover-12),
    outcome probability by the backward sweep of psi and W^dagger |target> (a 20-qubit
    ripple-carry adder), each against simulating every single-error state as a
    trajectory."""
    import torch
    from paper_2301_07264_gb300 import arso
    from workloads import circuits as W
    rows = []
    adder = W.cuccaro_adder(9, 301, 177)  # 20 qubits, outcome probability of the sum
    for name, circ, kw in (("brickwork24", W.brickwork24(), {}), ("grover12", W.grover12(0), {}),
                           ("adder20_outcome", adder, {})):
        if circ.criterion.kind == "outcome":
            crit = W.Criterion("outcome", target=circ.criterion.target, threshold=0.5, aggregate="mean")
        else:
            crit = W.Criterion("fidelity", threshold=0.9, aggregate="mean")
        res = {}
        for route, flags in (("sweep", 0), ("trajectories", arso.OPT_NO_FAST_EXHAUSTIVE)):
            cc = arso.compile_circuit(circ.n, circ.gates, flags=flags, **kw)
            arso.reference_state(cc, torch.empty(1 << circ.n, dtype=torch.complex64, device="cuda"))  # cache
            torch.cuda.synchronize()
            arso.profile_reset()
            t0 = time.perf_counter()
            P, per = arso.exhaustive(cc, crit)
            torch.cuda.synchronize()
            # streaming fidelity sweep: one zero-state launch, then one launch per gate
            sweeps = arso.profile_read(arso.K_OTHER).launches - 1
            res[route] = (time.perf_counter() - t0, P, per, sweeps)
        (ts, Ps, pers, sweeps), (tt, Pt, pert, _) = res["sweep"], res["trajectories"]
        rows.append({"circuit": name, "n": circ.n, "G": circ.G, "L": circ.L, "states": 3 * circ.L,
                     "sweep_s": ts, "trajectories_s": tt, "speedup": tt / ts, "sweeps": sweeps,
                     "max_abs_diff": float(np.max(np.abs(pers - pert))), "P": Ps.tolist()})
    return {"metric": "single-error states scored/sec (exhaustive analysis)",
            "value": sum(r["states"] for r in rows) / sum(r["sweep_s"] for r in rows), "unit": "states/s",
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "exhaustive_single_error", "circuits": [r["circuit"] for r in rows]},
            "hbm_sweep": _hbm_sweep(rows), "rows": rows}


def _hbm_sweep(rows):
    """Streaming (HBM) sweep of brickwork-24: each launch applies one gate with the
    expectations of its qubits, reading and writing the 2^24-amplitude complex64 state
    once: 2 * 8 * 2^n bytes per launch."""
    r = next((r for r in rows if r["circuit"] == "brickwork24"), None)
    if r is None:
        return None
    gb = r["sweeps"] * 2 * 8 * (1 << r["n"]) / 1e9
    return {"kernel": "gate_expect_kernel", "gates": r["G"], "sweeps": r["sweeps"], "algorithmic_GB": gb,
            "achieved_GBps": gb / r["sweep_s"], "note": "whole sweep time, reductions included"}


def qv(args):
    """Quantum-volume circuits scored by their heavy-output probability (the
    paper's QV evaluation: binning on the heavy outputs, averaged over 200
    random circuits per data point): 200 circuits at each of 8, 12 and 16
    qubits, p = 1e-3, 500 trajectories per circuit, one arso_run_batch call per
    size and step. The heavy sets come from the library's error-free states."""
    import torch
    from paper_2301_07264_gb300 import arso
    from workloads import circuits as W
    sizes, per_size, T, p = (8, 12, 16), 200, 500, 1e-3
    groups = []
    for n in sizes:
        ccs, crits = [], []
        ref = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        for k in range(per_size):
            circ = W.quantum_volume(n, 10_000 * n + k)
            cc = arso.compile_circuit(n, circ.gates)
            arso.reference_state(cc, ref)
            probs = (ref.abs() ** 2).double().cpu().numpy()
            heavy = np.flatnonzero(probs > np.median(probs)).astype(np.uint64)
            ccs.append(cc)
            crits.append(W.Criterion("binning", basis_set=heavy.tolist(), threshold=2 / 3, aggregate="mean"))
        outs = [torch.empty(T, dtype=torch.float64, device="cuda") for _ in ccs]
        groups.append((n, ccs, crits, outs))
    stream = torch.cuda.current_stream()

    def step(k):
        for n, ccs, crits, outs in groups:
            errs = [arso.sample_errors(cc, p / 3, p / 3, p / 3, 0, k * T, T, stream) for cc in ccs]
            arso.run_batch(ccs, errs, crits, outs, None, stream)

    for w in range(args.warmup):
        step(1000 + w)
    hop = {n: [] for n in sizes}
    e0, e1 = _events()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    for n, ccs, crits, outs in groups:
        hop[n] = [float(o.mean().item()) for o in outs]
    total = len(sizes) * per_size * T * args.steps
    return {"metric": "error-injected trajectories/sec", "value": total / sec, "unit": "traj/s",
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "quantum_volume_heavy_output", "sizes": list(sizes), "circuits_per_size": per_size,
                       "traj_per_circuit": T, "p": p, "criterion": "binning on heavy outputs (mean)"},
            "results": {str(n): {"mean_heavy_output_probability": float(np.mean(hop[n])),
                                 "circuits_above_2/3": int(np.sum(np.asarray(hop[n]) > 2 / 3))} for n in sizes},
            "kernels": _kernel_stats(arso)}


def fit_inverse_gate_count(Gs, ps, G_extrapolate):
    """Least-squares fits of the tolerable rate linear in 1 / G (Sec. V-B):
    p* = b / G through the origin (used for the extrapolation to G_extrapolate
    gates) and p* = a + b / G with an intercept, each with its mean squared
    residual."""
    g_inv, pv = 1.0 / np.asarray(Gs, dtype=float), np.asarray(ps, dtype=float)
    b0 = float(g_inv @ pv / (g_inv @ g_inv))
    A = np.stack([np.ones(len(Gs)), g_inv], axis=1)
    coef, *_ = np.linalg.lstsq(A, pv, rcond=None)
    return {"b": b0, "mse": float(np.mean((b0 * g_inv - pv) ** 2)),
            "affine_a": float(coef[0]), "affine_b": float(coef[1]),
            "affine_mse": float(np.mean((A @ coef - pv) ** 2)),
            "G_56": int(G_extrapolate), "p_tol_56_extrapolated": b0 / G_extrapolate}


def families(args):
    """Tolerable error rate (target success 0.66, the paper's figure) of the
    paper's circuit families at several sizes, through the library's Fig. 3
    flow (exhaustive analysis, then Eq. (5) or Monte Carlo bisection), then
    per family least-squares fits of p* linear in 1 / G (through the origin,
    and with an intercept) and the extrapolation of the first to a 56-qubit
    instance of the family (the paper's quantum-advantage regime)."""
    import torch
    from paper_2301_07264_gb300 import arso
    from workloads import circuits as W
    P_target = 0.66
    fams = {
        "bv": (lambda n: W.bernstein_vazirani(n, (1 << (n - 1)) - 1 - (n % 3)), (6, 8, 10, 12, 14, 16)),
        "hlf": (lambda n: W.hidden_linear_function(n, 100 + n), (6, 8, 10, 12, 14, 16)),
        "ryrz": (lambda n: W.ryrz_ansatz(n, 1, 200 + n), (6, 8, 10, 12, 14, 16)),
        "qft": (lambda n: W.qft_basis(n, int(("10" * n)[:n], 2)), (6, 8, 10, 12, 14, 16)),
        "adder": (lambda n: W.cuccaro_adder((n - 2) // 2, 5 % (1 << ((n - 2) // 2)), 3), (6, 8, 10, 12, 14, 16)),
        "uccsd": (lambda n: W.uccsd_ansatz(n, n // 2, 300 + n), (4, 6, 8, 10)),
    }
    rows, fits = [], {}
    t0 = time.perf_counter()
    for name, (make, sizes) in fams.items():
        Gs, ps = [], []
        for n in sizes:
            circ = make(n)
            crit = W.Criterion(circ.criterion.kind, target=circ.criterion.target, threshold=circ.criterion.threshold,
                               aggregate="mean")
            cc = arso.compile_circuit(circ.n, circ.gates)
            r = arso.tolerable_rate(cc, crit, P_target, n_traj=4000, seed=0, rel_tol=0.05, p_lo=1e-7, p_hi=0.3)
            rows.append({"family": name, "n": n, "G": circ.G, "L": circ.L, "p_tol": r.p, "probes": r.probes,
                         "mode": "Eq. (5)" if r.mode_used == 0 else "Monte Carlo", "p_tol_times_G": r.p * circ.G})
            Gs.append(circ.G)
            ps.append(r.p)
        fits[name] = fit_inverse_gate_count(Gs, ps, make(56).G)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    return {"metric": "tolerable-rate searches/sec", "value": len(rows) / sec, "unit": "searches/s",
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "families_tolerable_rate", "target": P_target, "n_traj": 4000, "rel_tol": 0.05},
            "all_below_one_error": all(r["p_tol_times_G"] < 1.0 for r in rows),
            "fits": fits, "rows": rows}


def run(args):
    import torch
    torch.cuda.set_device(0)
    torch.cuda.set_stream(torch.cuda.Stream())
    return {"qft4": qft4, "grover12": grover12, "mix256": mix256, "search": search, "exhaustive": exhaustive, "qv": qv, "families": families}[args.workload](args)
