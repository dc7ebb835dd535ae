#!/usr/bin/env python
"""Benchmark: error-injected Monte Carlo trajectories per second.

Workload (default): random brickwork circuit, 24 qubits, depth 40 (per layer
Haar SU(2) on every qubit, then CZ on alternating neighbour pairs, open chain;
G = 1420 gates, L = 1880 error locations), uniform Pauli errors at
p in {1e-4, 1e-3}, fidelity with the error-free state >= 0.9, complex64
amplitudes (FP32 arithmetic, FP64 reductions), prefix-state reuse. The full
workload is 10,000 trajectories per p; one step is one batch of
--traj-per-step trajectories split evenly over the two rates and runs every
row of the path: Philox error sampling, prefix reuse, fused passes with
folded Pauli errors, fused fidelity reduction and aggregation.

Prints ONE JSON line (rank 0). Under torchrun every rank runs its own
trajectory range (weak scaling, no collective on the data path); the time is
the max over ranks after a barrier.

Other configurations (--workload): qft4 (4-qubit QFT on |0101>, complex128,
1,000 trajectories at p = 1e-3), grover12 (Grover, 11 search qubits + 1
borrowed, 16 rates, argmax), mix256 (256 uneven circuits of 8-22 qubits with
autotuned tiles), search (surrogate-bracketed vs plain tolerable-rate search),
exhaustive (single-error analysis by one sweep vs by trajectories), qv
(quantum-volume heavy-output probability), families (tolerable rate of the
paper's circuit families, 1/G fits and the 56-qubit extrapolation).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P_RATES = (1e-4, 1e-3)
TRAJ_PER_P = 10_000
METRIC = "error-injected trajectories/sec"
UNIT = "traj/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _bf16_peak():
    """Dense bf16 tensor peak for a kernel timed alone: the measured burst figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (cuBLAS bf16 burst)"
    except Exception:
        return 1900.0, "fallback"


def _kernel_sha():
    h = hashlib.sha256()
    for f in ("pass_rb.cu", "sim_common.cuh", "kernels.h", "internal.h"):
        with open(os.path.join(ROOT, "paper_2301_07264_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_ratio():
    """DRAM bytes per algorithmic byte of the pass launches, from the ncu capture
    recorded in profiles/pass_kernel_traffic.json, if that capture was taken on the
    current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "pass_kernel_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_sha") != _kernel_sha():
            return None
        return float(d["dram_bytes_per_algorithmic_byte"])
    except Exception:
        return None


def write_traffic(dram_csv, trace_json, out_path=None):
    """profiles/pass_kernel_traffic.json from an ncu capture of every pass launch of
    one run (dram__bytes_read.sum and dram__bytes_write.sum, --csv) and that run's
    --trace-all line (the library's algorithmic bytes of the same launches)."""
    import csv
    lines = [l for l in open(dram_csv) if l.startswith('"')]
    rows = list(csv.reader(lines))
    h = rows[0]
    mi, vi, ui, idi = h.index("Metric Name"), h.index("Metric Value"), h.index("Metric Unit"), h.index("ID")
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    rd = wr = 0.0
    ids = set()
    for r in rows[1:]:
        if r[mi] == "dram__bytes_read.sum":
            rd += float(r[vi].replace(",", "")) * scale[r[ui]]
            ids.add(r[idi])
        if r[mi] == "dram__bytes_write.sum":
            wr += float(r[vi].replace(",", "")) * scale[r[ui]]
    d = [json.loads(l) for l in open(trace_json) if l.startswith("{")][-1]
    t = d["trace_all"]
    n_ncu, n_alg = len(ids), t["pass_launches"]
    out = {
        "kernel": "pass_rb_kernel",
        "source_sha": _kernel_sha(),
        "source_files": ["paper_2301_07264_gb300/csrc/" + f for f in ("pass_rb.cu", "sim_common.cuh", "kernels.h",
                                                                      "internal.h")],
        "workload": d["config"]["workload"], "tile_qubits": d["config"].get("tile_qubits"),
        "commands": ["python bench.py --qubits 20 --steps 2 --warmup 3 --no-cpu-baseline --trace-all > trace20.json",
                     "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                     "--clock-control none -k regex:pass_rb_kernel --csv --log-file dram20.csv python bench.py "
                     "--qubits 20 --steps 2 --warmup 3 --no-cpu-baseline --trace-all",
                     "python bench.py --write-traffic dram20.csv trace20.json"],
        "dram_read_bytes": rd, "dram_write_bytes": wr, "launches_captured": n_ncu,
        "algorithmic_bytes": t["pass_algorithmic_bytes"], "launches_traced": n_alg,
        "dram_bytes_per_algorithmic_byte": round(((rd + wr) / n_ncu) / (t["pass_algorithmic_bytes"] / n_alg), 4),
        "ratio_over_totals": round((rd + wr) / t["pass_algorithmic_bytes"], 4),
        "note": "DRAM bytes of every pass launch of a whole 20-qubit run against the library's algorithmic bytes "
                "(one read and one write of every swept state) of the same run, per launch (ncu may capture a "
                "few launches fewer than the library traced). The bench multiplies the ratio by the 24-qubit "
                "launch's algorithmic bytes.",
    }
    with open(out_path or os.path.join(ROOT, "profiles", "pass_kernel_traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))
    return out


class ClockSampler:
    FIELDS = ("clocks.sm", "clocks.max.sm", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.samples.append(parts)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------- CPU oracle ---
# The FP64 oracle (test infrastructure) timed on this host's cores as the CPU
# baseline: never tuned for it, run as it stands, parallel only across
# trajectories (one worker process per core, each simulating its own errored
# trajectory with oracle.statevector.simulate, gate chunk by gate chunk).

def host_info():
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    import platform
    return f"{platform.machine()} {model or platform.processor() or 'unknown CPU'}, {os.cpu_count()} logical CPUs"


def _usable_cores(state_bytes):
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    try:  # about five state-sized temporaries per worker during a gate
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        cores = min(cores, max(1, int(avail * 0.5 // (6 * state_bytes))))
    except Exception:
        pass
    return max(1, min(cores, 64))


def _oracle_worker(conn, workload, traj):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import sampling, statevector
    from workloads import circuits as C
    circ = C.brickwork24(0) if workload == "brickwork24" else C.grover12(0)
    p = 1e-3
    events = sampling.sample_trajectory(0, traj, circ.L, p / 3, p / 3, p / 3)
    table = statevector.location_table(circ)
    first_loc = [0]
    for gate in circ.gates:
        first_loc.append(first_loc[-1] + len(gate.qubits))
    psi = statevector.zero_state(circ.n)
    g = 0
    conn.send(("ready", circ.G, circ.L, circ.n))
    while True:
        want = conn.recv()
        if want is None:
            break
        t0 = time.perf_counter()
        done = 0
        while done < want:
            g1 = min(circ.G, g + want - done)
            # the oracle's own simulate() over the next chunk, with this trajectory's errors in it
            ev = [(l - first_loc[g], c) for (l, c) in events if g <= table[l][0] < g1]
            psi = statevector.simulate(C.Circuit(circ.n, circ.gates[g:g1]), ev, psi0=psi)
            done += g1 - g
            g = g1
            if g == circ.G:  # trajectory finished: start the next one from |0...0>
                psi = statevector.zero_state(circ.n)
                g = 0
        conn.send((time.perf_counter() - t0, done))


class OracleFarm:
    """`procs` worker processes (spawn start method), each holding one errored
    trajectory of the workload in the FP64 oracle."""

    def __init__(self, workload, procs):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for i in range(procs):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(b, workload, 1000 * i + 1), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        infos = [self._recv(i, 600) for i in range(procs)]
        _, self.G, self.L, self.n = infos[0]

    def _recv(self, i, timeout):
        """Reply of worker i; raises if it died or stayed silent for `timeout` s."""
        c, pr = self.conns[i], self.procs[i]
        t0 = time.perf_counter()
        while not c.poll(1.0):
            if not pr.is_alive():
                raise RuntimeError(f"oracle worker {i} exited with code {pr.exitcode}")
            if time.perf_counter() - t0 > timeout:
                raise RuntimeError(f"oracle worker {i} gave no answer within {timeout} s")
        return c.recv()

    def step(self, gates_per_worker):
        """Every worker simulates the next `gates_per_worker` gates; returns
        (wall seconds, total gates)."""
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(int(gates_per_worker))
        done = sum(self._recv(i, 3600)[1] for i in range(len(self.conns)))
        return time.perf_counter() - t0, done

    def close(self):
        for c in self.conns:
            try:
                c.send(None)
            except Exception:
                pass
        for pr in self.procs:
            pr.join(timeout=30)
            if pr.is_alive():
                pr.terminate()


def errored_fraction(L, rates=P_RATES):
    return sum(1.0 - (1.0 - p) ** L for p in rates) / len(rates)


def oracle_gates_per_traj(G, L, rates, traj_per_rate):
    """Oracle gate applications per trajectory of the workload: an errored
    trajectory simulates all G gates, an error-free one reuses the reference
    state (computed once for the workload: G gates over all its trajectories)."""
    return G * (errored_fraction(L, rates) + 1.0 / (traj_per_rate * len(rates)))


def cpu_baseline(workload, seconds, rates, traj_per_rate, state_bytes):
    """The oracle on 1 core and on all usable cores, about `seconds` each."""
    out = {}
    for label, procs in (("single_core", 1), ("all_cores", _usable_cores(state_bytes))):
        farm = None
        try:
            farm = OracleFarm(workload, procs)
            dt, g = farm.step(1)  # warm-up, then calibration on about a tenth of the budget
            dt, g = farm.step(max(1, int(0.1 * seconds / max(dt, 1e-9))))
            per = max(1, int(seconds * g / procs / max(dt, 1e-9)))
            dt, g = farm.step(per)
        finally:
            if farm:
                farm.close()
        gates_per_traj = oracle_gates_per_traj(farm.G, farm.L, rates, traj_per_rate)
        out[label] = {"value": g / dt / gates_per_traj, "unit": UNIT, "cores": procs, "kind": "oracle",
                      "sample": f"FP64 numpy oracle simulate() over {g} gates of {procs} errored {workload} "
                                f"trajectories in {dt:.1f} s ({procs} worker processes, one trajectory each); "
                                f"traj/s = gates/s / {gates_per_traj:.1f} oracle gates per trajectory (errored "
                                f"fraction {errored_fraction(farm.L, rates):.3f} x G {farm.G}, plus the "
                                f"reference state once per workload)"}
    line = dict(out["all_cores"])
    line["single_core"] = out["single_core"]
    line["host"] = host_info()
    return line


def grover_cpu_baseline(seconds):
    from workloads import circuits as C
    circ = C.grover12(0)
    rates = [10 ** (-5 + 3 * i / 15) for i in range(16)]
    return cpu_baseline("grover12", seconds, rates, 100_000, 16 << circ.n)


def qft4_cpu_baseline():
    """The FP64 oracle on the whole QFT-4 workload step (1,000 trajectories at
    p = 1e-3 through montecarlo.run_trajectories), one core: it finishes in
    seconds, so no sampling is needed."""
    from oracle import montecarlo
    from workloads import circuits as C
    circ = C.qft4_0101()
    p, T = 1e-3, 1000
    t0 = time.perf_counter()
    montecarlo.run_trajectories(circ, 0, 0, T, p / 3, p / 3, p / 3)
    dt = time.perf_counter() - t0
    return {"value": T / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_info(),
            "sample": f"FP64 numpy oracle montecarlo.run_trajectories over all {T} trajectories of one step "
                      f"({dt:.2f} s, one core)"}


def run_reference(args):
    """--impl reference: the FP64 CPU oracle timed on this host's cores, on all
    usable cores in parallel over trajectories. Each step is a bounded sample of
    the workload (every worker simulates the next gates of its own errored
    trajectory); value = trajectory-equivalents per second."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from workloads import circuits as C
    circ = C.brickwork24(0)
    procs = _usable_cores(16 << circ.n)
    budget = float(os.environ.get("ARSO_REFERENCE_SECONDS", "150"))
    per_step = max(0.5, budget / max(args.steps + args.warmup, 1))
    gates_per_traj = oracle_gates_per_traj(circ.G, circ.L, P_RATES, TRAJ_PER_P)
    farm = None
    try:
        farm = OracleFarm("brickwork24", procs)
        dt, g = farm.step(1)
        dt, g = farm.step(max(1, int(0.2 * per_step / max(dt, 1e-9))))
        per = max(1, int(per_step * g / procs / max(dt, 1e-9)))
        for _ in range(max(args.warmup - 1, 0)):
            farm.step(per)
        times, gates = [], 0
        for _ in range(args.steps):
            dt, g = farm.step(per)
            times.append(dt)
            gates += g
    finally:
        if farm:
            farm.close()
    total = sum(times)
    traj_per_s = gates / total / gates_per_traj
    sample = (f"FP64 numpy oracle simulate() over {gates} gates of {procs} errored 24-qubit brickwork trajectories "
              f"({per} gates per worker per step, {procs} worker processes); traj/s = gates/s / "
              f"{gates_per_traj:.1f} oracle gates per trajectory (errored fraction "
              f"{errored_fraction(circ.L):.3f} x G {circ.G}, plus the reference state once per workload)")
    line = {
        "impl": "reference", "metric": METRIC, "value": traj_per_s, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(circ, args),
        "cpu_baseline": {"value": traj_per_s, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample,
                         "host": host_info()},
        "e2e": {"value": traj_per_s, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(circ, args, tile=None, passes=None):
    return {"workload": f"brickwork{circ.n}_depth40_p1e-4_1e-3", "n_qubits": circ.n, "depth": 40, "G": circ.G,
            "L": circ.L, "p": list(P_RATES), "trajectories_per_p": TRAJ_PER_P,
            "traj_per_step": args.traj_per_step, "criterion": "fidelity >= 0.9 (pass fraction)",
            "prefix_reuse": True, "suffix_reuse": not getattr(args, "no_suffix", False),
            "tile_qubits": tile, "passes": passes,
            "l2": "inputs larger than L2: every trajectory state is 128 MiB (> 126 MiB L2)"}


# ------------------------------------------------------------------ ours ---

def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    from paper_2301_07264_gb300 import arso
    from workloads import circuits as C

    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()  # a real stream: the pass sequences are captured and replayed as CUDA graphs
    torch.cuda.set_stream(stream)
    circ = C.brickwork(args.qubits, 40, 0)  # 24 qubits: the benchmark circuit (brickwork24)
    crit = arso.make_criterion(circ.criterion)
    if args.trace_all:  # algorithmic bytes of every launch, prefix-cache build and warm-up included
        arso.profile_reset()
        arso.profile_enable(True)
    # 12-qubit tiles: the measured best schedule for this circuit (four 128-thread CTAs per SM
    # cover the tile loads' latency better than two 256-thread ones); 0 keeps the library default
    tile = args.tile if args.tile >= 0 else 12
    cc = arso.compile_circuit(circ.n, circ.gates, tile_qubits=tile, low_qubits=args.low,
                              cache_bytes=int(args.cache_gb * (1 << 30)) if args.cache_gb else 0,
                              flags=(arso.OPT_NO_SUFFIX_REUSE if args.no_suffix else 0) |
                                    (arso.OPT_TENSOR_PHASES if args.tensor else 0))
    info = cc.info()
    half = args.traj_per_step // len(P_RATES)
    score = {p: torch.empty(half, dtype=torch.float64, device="cuda") for p in P_RATES}
    flags = {p: torch.empty(half, dtype=torch.uint8, device="cuda") for p in P_RATES}

    def begin_of(step_idx):
        return (rank * 1_000_000_000) + (step_idx * half) % TRAJ_PER_P

    def step(step_idx, host_out=None):
        res = []
        for p in P_RATES:
            errs = arso.sample_errors(cc, p / 3, p / 3, p / 3, 0, begin_of(step_idx), half, stream)
            if host_out is None:
                arso.run_trajectories(cc, errs, crit, score[p], flags[p], stream)
                res.append(arso.aggregate(score[p], flags[p], stream))
            else:
                s_h, f_h = host_out[p]
                arso.run_trajectories(cc, errs, crit, s_h, f_h, stream)
                res.append((float(np.mean(s_h)), float(np.mean(f_h))))
        return res

    # warm-up (also builds the prefix cache); warm-up batches lie outside the timed ranges
    for w in range(args.warmup):
        step(TRAJ_PER_P // half + w)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    before = None
    if args.trace_all:
        ps0 = arso.profile_read(arso.K_PASS)
        pl0 = arso.profile_read(arso.K_PASS_LAST)
        before = {"pass_launches": ps0.launches + pl0.launches, "pass_algorithmic_bytes": ps0.bytes + pl0.bytes}
    clocks = ClockSampler(dev)
    clocks.start()
    arso.profile_reset()
    arso.profile_enable(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    aggs = []
    for k in range(args.steps):
        aggs.append(step(k))
    ev1.record(stream)
    torch.cuda.synchronize()
    arso.profile_enable(False)
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches, _, _ = arso.profile_counters()
    kstats = {name: arso.profile_read(k) for name, k in
              (("pass", arso.K_PASS), ("pass_last", arso.K_PASS_LAST), ("resident", arso.K_RESIDENT),
               ("sample", arso.K_SAMPLE), ("reduce", arso.K_REDUCE), ("other", arso.K_OTHER))}
    clk = clocks.stop()
    if dist:
        t = torch.tensor([elapsed], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())

    # end to end through the public API with host (pinned) result buffers
    host_out = {p: (torch.empty(half, dtype=torch.float64, pin_memory=True).numpy(),
                    torch.empty(half, dtype=torch.uint8, pin_memory=True).numpy()) for p in P_RATES}
    e2e_steps = max(1, min(args.steps, 5))
    if before is not None:  # the timed steps' pass launches join the whole-run count
        before["pass_launches"] += kstats["pass"].launches + kstats["pass_last"].launches
        before["pass_algorithmic_bytes"] += kstats["pass"].bytes + kstats["pass_last"].bytes
    arso.profile_reset()
    arso.profile_enable(args.trace_all)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        step(k, host_out)
    torch.cuda.synchronize()
    e2e_time = time.perf_counter() - t0
    _, h2d, d2h = arso.profile_counters()
    if before is not None:  # and the end-to-end steps'
        arso.profile_enable(False)
        for k in (arso.K_PASS, arso.K_PASS_LAST):
            st_ = arso.profile_read(k)
            before["pass_launches"] += st_.launches
            before["pass_algorithmic_bytes"] += st_.bytes
    if dist:
        t = torch.tensor([e2e_time], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_time = float(t.item())

    if rank != 0:
        dist.destroy_process_group() if dist else None
        return 0

    total = args.traj_per_step * args.steps * ws
    value = total / elapsed
    peak, peak_kind = _peaks()
    ps = kstats["pass"]
    achieved = (ps.bytes / (ps.ms / 1e3)) / 1e9 if ps.ms > 0 else 0.0
    tflops = (ps.flops / (ps.ms / 1e3)) / 1e12 if ps.ms > 0 else 0.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = float(clk.get("sm_max_mhz") or 2070.0)
    fp32_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    tr = _traffic_ratio()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(circ, args, info.tile_qubits, info.n_passes),
        # The fused pass sweeps each state once per ~31 gates, so it is bound by
        # FP32 arithmetic, not by HBM: its roof is the FP32 rate of the SMs.
        "roofline": {"bound": "alu", "kernel": "pass_rb_kernel (fused register-blocked tile pass)",
                     "achieved": tflops, "peak": fp32_peak,
                     "peak_kind": f"nominal FP32 FMA rate: {sms} SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz "
                                  "(max SM clock seen)",
                     "unit": "TFLOP/s", "frac": tflops / fp32_peak if fp32_peak else None,
                     "traffic": (tr * ps.bytes / max(ps.launches, 1)) if tr is not None else None,
                     "algorithmic_flops_per_launch": ps.flops / max(ps.launches, 1),
                     "algorithmic_bytes_per_launch": ps.bytes / max(ps.launches, 1),
                     "avg_launch_ms": ps.ms / max(ps.launches, 1), "launches": ps.launches},
        "roofline_hbm": {"achieved": achieved, "peak": peak, "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                         "unit": "GB/s", "frac": achieved / peak},
        "kernels": {k: {"launches": v.launches, "ms": v.ms, "GB": v.bytes / 1e9, "TFLOP": v.flops / 1e12}
                    for k, v in kstats.items()},
        "e2e": {"value": args.traj_per_step * e2e_steps * ws / e2e_time, "unit": UNIT,
                "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps},
        "gpu_launches": launches,
        "clocks": clk,
        "results": {"pass_frac_p1e-4": float(np.mean([a[0][1] for a in aggs])),
                    "pass_frac_p1e-3": float(np.mean([a[1][1] for a in aggs]))},
    }
    if before is not None:
        # every pass launch of the run (cache build, warm-up, timed and end-to-end steps),
        # for comparison with a DRAM capture of the same launches
        line["trace_all"] = before
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline("brickwork24", args.cpu_seconds, P_RATES, TRAJ_PER_P, 16 << circ.n)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def onchip_roofline(oc, clk):
    """The resident (whole state on chip) kernel against its on-chip roofs: the FP32
    FMA rate (SMs x 128 lanes x 2 flop x clock) and the shared-memory bandwidth (SMs x
    128 bytes per clock: 32 banks of 4 bytes), at the highest SM clock seen."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = float(clk.get("sm_max_mhz") or 2070.0)
    sec = oc["ms"] / 1e3
    tf = oc["flops"] / sec / 1e12 if sec > 0 else 0.0
    gbs = oc["smem_bytes"] / sec / 1e9 if sec > 0 else 0.0
    fp32_peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    smem_peak = sms * 128 * mhz * 1e6 / 1e9
    f_alu, f_smem = tf / fp32_peak, gbs / smem_peak
    alu = {"bound": "alu" if f_alu >= f_smem else "smem", "kernel": oc["kernel"], "achieved": tf, "peak": fp32_peak,
           "peak_kind": f"nominal FP32 FMA rate: {sms} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz", "unit": "TFLOP/s",
           "frac": f_alu, "traffic": None, "launches": oc["launches"], "device_ms": oc["ms"]}
    smem = {"achieved": gbs, "peak": smem_peak, "unit": "GB/s", "frac": f_smem,
            "peak_kind": f"shared memory: {sms} SMs x 128 B/clock x {mhz:.0f} MHz",
            "note": "algorithmic bytes: one write and one read of the state per register-set change"}
    return alu, smem


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--traj-per-step", type=int, default=None,
                    help="default 1000 (brickwork24), 4096 (grover12: 256 per rate, several waves of the "
                         "persistent launch)")
    ap.add_argument("--tile", type=int, default=-1,
                    help="tile qubits of the brickwork circuit (-1: 12, the measured best; 0: library default)")
    ap.add_argument("--write-traffic", nargs=2, metavar=("DRAM_CSV", "TRACE_JSON"),
                    help="write profiles/pass_kernel_traffic.json from an ncu DRAM capture and a --trace-all line")
    ap.add_argument("--low", type=int, default=0, help="contiguous low qubits of every tile (0 = library default)")
    ap.add_argument("--qubits", type=int, default=24,
                    help="brickwork qubits (24 = the benchmark circuit; smaller sizes are profiling cases)")
    ap.add_argument("--trace-all", action="store_true",
                    help="also report the algorithmic bytes of every pass launch of the run (cache build and "
                         "warm-up included), to set against a DRAM capture of the same launches")
    ap.add_argument("--cache-gb", type=float, default=0.0, help="prefix-cache budget (0 = library default)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="seconds of oracle work per CPU-baseline setting (1 core, all cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tensor", action="store_true",
                    help="fused-unitary register phases on the tensor cores (ARSO_OPT_TENSOR_PHASES)")
    ap.add_argument("--no-suffix", action="store_true",
                    help="run every trajectory to the end instead of scoring after its last error")
    ap.add_argument("--workload", default="brickwork24", choices=["brickwork24", "qft4", "grover12", "mix256", "search", "exhaustive", "qv", "families"],
                    help="brickwork24 is the benchmark line; the others measure the other configurations")
    ap.add_argument("--search-circuits", type=int, default=8,
                    help="search workload: evaluation circuits per size band (half as many at 20-24 qubits)")
    ap.add_argument("--search-epochs", type=int, default=16, help="search workload: surrogate training epochs")
    ap.add_argument("--search-large", type=int, default=0,
                    help="search workload: evaluation circuits of 20-24 qubits (0: half of --search-circuits)")
    ap.add_argument("--search-ablation", action="store_true",
                    help="search workload: also train a network on the three circuits of the other "
                         "configurations only and search the 12-18-qubit circuits with it")
    ap.add_argument("--search-margin", type=float, default=0.08,
                    help="search workload: half-width of the surrogate's bracket in log10 p")
    ap.add_argument("--train-rows", type=int, default=2_000_000)
    args = ap.parse_args()
    if args.write_traffic:
        return write_traffic(*args.write_traffic)
    if args.traj_per_step is None:
        args.traj_per_step = 4096 if args.workload == "grover12" else 1000
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "brickwork24":
        from paper_2301_07264_gb300 import bench_workloads
        clocks = ClockSampler(0)
        clocks.start()
        line = bench_workloads.run(args)
        clk = clocks.stop()
        if line is not None:
            line["clocks"] = clk
            if args.workload == "grover12":
                line["roofline"], line["roofline_smem"] = onchip_roofline(line.pop("onchip"), clk)
            if args.workload == "grover12" and not args.no_cpu_baseline:
                line["cpu_baseline"] = grover_cpu_baseline(args.cpu_seconds)
            if args.workload == "qft4" and not args.no_cpu_baseline:
                line["cpu_baseline"] = qft4_cpu_baseline()
            if args.workload == "exhaustive" and line.get("hbm_sweep"):
                peak, src = _peaks()
                h = line["hbm_sweep"]
                h["peak_GBps"], h["peak_source"] = peak, src
                h["frac"] = h["achieved_GBps"] / peak
            if args.workload == "search":
                g = line["surrogate_train"]["gemm"]
                peak, src = _bf16_peak()
                g["peak_tflops"], g["peak_source"] = peak, src
                g["frac"] = g["useful_tflops"] / peak if g["useful_tflops"] else None
            print(json.dumps(line), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
