"""Benchmark: two-site MPO updates per second at chi = 256 on the 28-qubit unswapping
workload (n=28 all-to-all qubit pairs, 200 Haar SU(4) gates per half, hidden permutation,
perturbation exp(i 0.02 H) on the mirrored half, chi_max = 256, SVD cutoff 1e-10, tau = 1e6).

Workload.  On this workload the MPO saturates: from the middle of the contraction on, every
interior bond sits at chi = 256 and the contraction is a long sequence of 1024 x 1024 bond
factorisations.  One bench step is one pass of the whole hot path in that regime:
  restore the saturated MPO (bonds [4, 16, 64, 256 x 21, 64, 16, 4]; seeded right-isometric
  site tensors, each the identity plus an O(0.02) part, so the output stays peaked) with the
  circuit's layer cursors at 12 / 12,
  one outer iteration of Algorithm 1: route + absorb the next layer pair (plan, merge, gate,
  factorise, truncate, split, size check), then one unswap stage (parallel variant, six
  parity batches), rewiring by layout;
  then project onto |0...0>, extract the peak (exact best-first search) and draw 1000 samples.
value = two-site updates evaluated per second: absorption updates (each a full factorisation)
plus unswap trials (each decided either by the library's lower-bound certificate or by a full
factorisation), summed over ranks (replicas: each rank runs its own seeded instance); the
line also gives the full updates and the trials apart, the batches of independent chi = 256
updates of the microbenchmark (M0: 1, 8, 32 per launch, FP64 and mixed merges), the
algorithmic-work roofline of the whole step, and the measured FP64 / FP32 peaks it uses.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       python bench.py --profile-case --chi 256 --batch 4 [--precision 0|1]   (one M0 launch)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_21908_gb300 import workloads as W  # noqa: E402

METRIC = "two-site MPO updates/s at χ=256; time-to-peak; served p50/p99 latency"
UNIT = "updates/s"
N_QUBITS, CHI_MAX, EPS, TAU = 28, 256, 1e-10, 1e6
CURSOR = 12
N_SAMPLES = 1000
M0_BATCHES = (1, 8, 32)


def workload_name():
    return ("unswap28 saturated regime: n=28 all-to-all, 200 Haar SU(4) gates/half, hidden permutation, "
            "perturbation 0.02, chi_max=256, eps=1e-10, tau=1e6; MPO bonds [4,16,64,256x21,64,16,4]; "
            "step = one Algorithm-1 iteration (layer pair + unswap stage) + project + peak + 1000 samples")


def saturated_state(seed: int):
    """The seeded peaked MPO with every interior bond at chi_max (the saturated regime)."""
    return W.peaked_saturated_state(N_QUBITS, CHI_MAX, seed)


class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def aggregate_over_ranks(dev_ms: float, units: int, dist, device) -> tuple[float, int]:
    """Whole-job figures over the ranks: the slowest rank's device time (MAX) and the units
    all ranks processed (SUM).  Replicas share nothing else: no collective touches the data
    path.  `device` is where the reduction tensors live (cuda for NCCL, cpu for gloo)."""
    if dist is None:
        return dev_ms, units
    import torch
    t = torch.tensor([dev_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(u.item()))


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(seed: int, budget_s: float, min_updates: int = 2):
    """The FP64 oracle as it stands, timed on the host cores on a bounded sample of the
    same step: the first updates of the step's layer pair on the same saturated state."""
    from oracle import mpo

    circ = W.workload_unswap28(seed)
    cfg = mpo.Config(eps=EPS, chi_max=CHI_MAX, tau=TAU)
    ctr = mpo.Contraction(circ, cfg)
    B, lam = saturated_state(seed)
    ctr.state.B = [b.copy() for b in B]
    ctr.state.lam = [l.copy() for l in lam]
    ctr.left_cursor = ctr.right_cursor = CURSOR

    class Spent(Exception):
        pass

    done = [0]
    t_end = [0.0]
    update = ctr.state.apply

    def bounded_update(j, u16, c):
        # the oracle's own two-site update; stop between updates once the budget is spent
        if done[0] >= min_updates and time.perf_counter() - t0 > budget_s:
            raise Spent
        r = update(j, u16, c)
        done[0] += 1
        t_end[0] = time.perf_counter()
        return r

    ctr.state.apply = bounded_update
    t0 = time.perf_counter()
    try:
        for gidx in ctr.left_layers[CURSOR]:
            ctr._route_and_apply(mpo.SIDE_LEFT, gidx)
    except Spent:
        pass
    return done[0], t_end[0] - t0


def oracle_sample_threads(seed: int, budget_s: float, threads: int):
    """oracle_sample in a child process whose BLAS uses `threads` threads (the thread count is
    fixed by the environment before numpy loads).  Returns (updates, seconds)."""
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
            f"u, dt = bench.oracle_sample({seed}, {budget_s}); print(u, dt)")
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[var] = str(threads)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=budget_s * 20 + 600)
    if r.returncode != 0:
        raise RuntimeError(f"oracle child failed: {r.stderr[-2000:]}")
    u, dt = r.stdout.strip().split()[-2:]
    return int(u), float(dt)


def m0_inputs(batch: int, chi: int, seed: int = 0):
    """The microbenchmark's operands: `batch` independent two-site updates on disjoint bonds of
    an MPO whose interior bonds are all at chi, with random right-isometric site tensors (QR of
    complex Gaussians), geometric spectra exp(-k/64) and Haar 16 x 16 operators."""
    n = 2 * batch + 10
    chis = W.saturated_bond_dims(n, chi)
    rng = W.rng_for(21, 1000 * seed + batch)
    B = [W.random_right_isometry(rng, chis[j], chis[j + 1]) for j in range(n)]
    lam = [W.geometric_spectrum(chis[b + 1], 64.0) for b in range(n - 1)]
    ops = np.array([W.haar_unitary(rng, 16) for _ in range(batch)])
    bonds = [4 + 2 * k for k in range(batch)]
    return n, B, lam, ops, bonds


def measure_m0(binding, batch: int, precision: int, chi: int = CHI_MAX, reps: int = 3, trials: bool = False,
               device: int = 0):
    """Batches of independent chi x chi updates through pc_apply_updates (one combined launch
    set per batch), CUDA events on the library's stream, L2 flushed before each repetition.
    With trials: one unswap stage on the same state (every trial has chi_old = chi_max)."""
    import torch
    n, B, lam, ops, bonds = m0_inputs(batch, chi)
    ctx = binding.Context(eps=EPS, chi_max=chi, tau=1e12, precision=precision, device=device)
    c = ctx.load_gates(n, np.zeros((0, 2), np.int32), np.zeros((0, 4, 4), complex))
    stream = torch.cuda.ExternalStream(c.stream_handle())
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    times = []
    c.reset_timers(True)
    for rep in range(reps + 1):
        c.set_state(B, lam)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.apply_updates(bonds, ops)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep > 0:
            times.append(e0.elapsed_time(e1))
    st = c.stats()
    out = {"batch": batch, "precision": ["fp64", "tf32x3 merges"][precision], "chi": chi,
           "ms_per_launch_set": statistics.median(times), "updates_per_s": batch / (statistics.median(times) / 1e3),
           "fp64_sweeps_max": st["max_sweeps"], "fp32_sweeps_max": st["max_sweeps_fp32"],
           "deflated": st["n_deflated"], "fallbacks": st["fallbacks"]}
    if trials:
        c.set_state(B, lam)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        before = c.stats()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.unswap()
        e1.record(stream)
        torch.cuda.synchronize()
        st2 = c.stats()
        nt = st2["n_trials"] - before["n_trials"]
        out["trials"] = {"trials": nt, "certified": st2["n_trials_certified"] - before["n_trials_certified"],
                         "ms": e0.elapsed_time(e1), "trials_per_s": nt / (e0.elapsed_time(e1) / 1e3),
                         "note": "one parallel unswap stage on the same state: SWAP trials on every bond, "
                                 "interior bond matrices 1024 x 1024 (ends smaller)"}
    c.close()
    ctx.close()
    return out


MIX_KW = dict(eps=1e-10, chi_max=64, tau=3000)
MIX_COUNT = 8


def _contract_peak(c):
    """Contract and search the peak; a truncated MPO whose M|0> vanished reports its status."""
    st = c.contract()
    try:
        c.extract_peak()
        ok = True
    except Exception:
        ok = False
    return st, ok


def measure_batching(binding, circs, kw, label):
    """The same independent circuits contracted one after another (each on its own workspace)
    and as one batch (pc_batch_contract: every factorisation of every circuit in shared
    launches).  Wall time of each, launches, tasks per launch, and whether the batch gave each
    circuit its alone result (bond dimensions and unswap log)."""
    ctx = binding.Context(**kw)
    t0 = time.perf_counter()
    waves = 0
    alone = []
    for circ in circs:
        c = ctx.load_circuit(circ)
        st, _ = _contract_peak(c)
        waves += st["n_waves"]
        alone.append((list(c.bond_dims()), c.unswap_log().tolist()))
        c.close()
    t_seq = time.perf_counter() - t0
    hs = [ctx.load_circuit(circ) for circ in circs]
    batch = binding.Batch(ctx, max_tasks=256)
    t0 = time.perf_counter()
    batch.contract(hs)
    for h in hs:
        try:
            h.extract_peak()
        except Exception:
            pass
    t_bat = time.perf_counter() - t0
    cnt = batch.counters()
    same = all(list(h.bond_dims()) == a[0] and h.unswap_log().tolist() == a[1] for h, a in zip(hs, alone))
    for h in hs:
        h.close()
    batch.close()
    ctx.close()
    return {"workload": label, "circuits": len(circs), "sequential_s": t_seq, "batched_s": t_bat,
            "speedup": t_seq / t_bat, "sequential_waves": waves, "batched_launches": cnt["launches"],
            "tasks_per_launch": cnt["tasks"] / max(cnt["launches"], 1), "max_tasks_per_launch": cnt["max_tasks"],
            "batched_equals_alone": same}


def measure_hqap_time_to_peak(binding, device: int = 0):
    """Time to peak of the HQAP-like workload (RZZ gates, one-qubit layers, swap insertions,
    angle noise 0.1) at 12 qubits, 60 RZZ gates per half, 3 swap insertions, with App. A.4's
    cutoff 2e-3, strict acceptance and adaptive sides; chi_max = 64, tau = 3000 (reduced so the
    run completes in seconds).  Load, contract, exact peak: wall time through the C ABI."""
    import torch
    circ = W.hqap_like_mirror(12, 60, 3, 0.1, seed=0)
    ctx = binding.Context(eps=2e-3, chi_max=64, tau=3000, side_mode=binding.SIDE_ADAPTIVE, device=device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c = ctx.load_circuit(circ)
    st = c.contract()
    bits, p, _ = c.extract_peak()
    t = time.perf_counter() - t0
    out = {"workload": "HQAP-like: n=12, 60 RZZ gates/half + one-qubit layers, 3 swap insertions, angle noise 0.1, "
                       "eps=2e-3, chi_max=64, tau=3000, adaptive sides", "time_to_peak_s": t,
           "peak_is_planted": bool(np.array_equal(bits, circ.planted)), "p_peak": p,
           "updates": st["n_updates"], "trials": st["n_trials"], "accepted": st["n_accepted"]}
    c.close()
    ctx.close()
    return out


def measure_serving(binding, precision: int, rate: float, count: int = 12):
    """A Poisson stream of `count` requests (the circuit mix above, cutoff 1e-5 so both
    precisions reach the same bond dimensions) through pc_server: p50/p99 time-to-peak and
    circuits/hour."""
    circs = W.circuit_mix(count, seed=1)
    arrivals = W.poisson_arrivals(count, rate, seed=precision)
    srv = binding.Server(max_resident=8, memory_budget=16 << 30, max_tasks=256)
    t0 = time.perf_counter()
    tickets = []
    for circ, ta in zip(circs, arrivals):
        delay = ta - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(circ, n_samples=100, seed=5, eps=1e-5, chi_max=64, tau=3000,
                                  precision=precision))
    ok = 0
    for t in tickets:
        res, _, _ = srv.wait(t, timeout_s=600)
        ok += res["status"] == 0
    st = srv.stats()
    srv.close()
    return {"precision": ["fp64", "tf32x3 merges"][precision], "requests": count, "rate_per_s": rate,
            "completed": ok, "p50_s": st["p50_s"], "p99_s": st["p99_s"], "mean_s": st["mean_s"],
            "circuits_per_hour": st["circuits_per_hour"], "max_resident": st["max_resident_seen"],
            "launches": st["launches"], "tasks_per_launch": st["tasks"] / max(st["launches"], 1)}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return
    cores = cpu_cores()
    per_step = []
    units = 0
    for _ in range(args.warmup):
        oracle_sample(0, 2.0, 1)
    for _ in range(args.steps):
        u, dt = oracle_sample(0, 15.0)
        units += u
        per_step.append(dt)
    total = sum(per_step)
    value = units / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64c",
            "data": "synthetic", "config": {"workload": workload_name(), "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "per step: the first two-site updates of the step's layer pair "
                                       "(about 15 s of host work, at least two updates) on the saturated "
                                       "28-qubit state"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    world, rank, local = dist_setup()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2604_21908_gb300 import binding

    fp64_peak, fp32_peak = binding.measure_alu_peaks(local)
    # the FP64 Jacobi launch width, tuned on this device for the step's launch shapes
    tune_path = os.path.join(tempfile.gettempdir(), f"pc_jacobi_tuning_{os.getpid()}.txt")
    tune_shapes = [(1024, 1), (1024, 4), (1024, 8), (256, 8), (64, 8)]
    tune_ms = binding.autotune(tune_shapes, path=tune_path, device=local)
    seed = rank
    circ = W.workload_unswap28(seed)
    extra = {"precondition_sweeps": args.pre_sweeps} if args.pre_sweeps > 0 else {}
    ctx = binding.Context(eps=EPS, chi_max=CHI_MAX, tau=TAU, device=local, **extra)
    c = ctx.load_circuit(circ)
    B, lam = saturated_state(seed)
    c.set_state(B, lam)
    c.set_cursors(CURSOR, CURSOR)
    c.snapshot()
    stream = torch.cuda.ExternalStream(c.stream_handle())
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        c.restore()
        st = c.contract_iterations(1)
        bits, p, _ = c.extract_peak()
        c.sample(N_SAMPLES, 1234 + seed)
        return st, p

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    c.reset_timers(True)
    units = full = trials = certified = 0
    alg_flops = 0.0
    dev_ms = 0.0
    stats = None
    for _ in range(args.steps):
        flush.fill_(1.0)                       # L2 flush between timed steps
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        stats, p = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        dev_ms += ev0.elapsed_time(ev1)
        units += stats["n_updates"] + stats["n_trials"]
        full += stats["n_full"]
        trials += stats["n_trials"]
        certified += stats["n_trials_certified"]
        alg_flops += stats["alg_flops"]
    launches, kms, kflops = c.timers()
    clk = clocks.stop()
    c.reset_timers(False)
    t_max, units_all = aggregate_over_ranks(dev_ms, units, dist, "cuda")
    value = units_all / (t_max / 1e3)

    # end to end through the public API with host buffers: load the gate list, upload the
    # state, run the step, read back peak and samples (one step, rank-local)
    sites_bytes = sum(b.size for b in B) * 16 + sum(l.size for l in lam) * 8
    gate_bytes = circ.pairs.nbytes + circ.mats.size * 16 + circ.oneq_qubits.nbytes + circ.oneq_mats.size * 16
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c2 = ctx.load_circuit(circ)
    c2.set_state(B, lam)
    c2.set_cursors(CURSOR, CURSOR)
    st2 = c2.contract_iterations(1)
    bits2, p2, _ = c2.extract_peak()
    samples2 = c2.sample(N_SAMPLES, 1234 + seed)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_units = st2["n_updates"] + st2["n_trials"]
    c2.close()

    if rank == 0:
        names = ["merge_gate", "factorisation", "truncate", "split", "other", "trial_certificate"]
        share = {name: {"launches": int(launches[k]), "ms": float(kms[k]), "tflops": float(kflops[k] / 1e12)}
                 for k, name in enumerate(names)}
        timed = {k: kms[k] for k in (0, 1, 2, 3, 5)}
        dom = max(timed, key=timed.get)
        dom_launch = int(launches[dom])
        dom_ms = kms[dom] / max(dom_launch, 1)
        dom_flops = kflops[dom] / max(dom_launch, 1)
        achieved = dom_flops / (dom_ms * 1e-3) / 1e12 if dom_ms > 0 else 0.0
        step_ms = t_max / args.steps
        t_roof_ms = alg_flops / args.steps / (fp64_peak * 1e12) * 1e3
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            u, dt = oracle_sample_threads(seed, 20.0, cpu_cores())
            u1, dt1 = oracle_sample_threads(seed, 20.0, 1)
            cpu = {"value": u / dt, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                   "sample": f"{u} two-site updates (the first of the step's layer pair, chi=256 interior) "
                             f"on the saturated 28-qubit state, {dt:.1f} s, BLAS threads = cores",
                   "one_thread": {"value": u1 / dt1, "cores": 1, "sample": f"{u1} updates, {dt1:.1f} s"}}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64c", "data": "synthetic",
            "config": {"workload": workload_name(), "n_qubits": N_QUBITS, "chi_max": CHI_MAX, "eps": EPS,
                       "tau": TAU, "samples": N_SAMPLES, "units_per_step": units // max(args.steps, 1),
                       "parallelism": f"replicas{world}", "l2": "flushed between steps (256 MiB write); "
                       "working set > L2"},
            "units": {"absorption_updates_per_step": stats["n_updates"], "unswap_trials_per_step": stats["n_trials"],
                      "trials_certified_per_step": stats["n_trials_certified"],
                      "full_factorisations_per_step": stats["n_full"], "deflated_per_step": stats["n_deflated"],
                      "full_updates_per_s": full / (t_max / 1e3), "trials_per_s": trials / (t_max / 1e3)},
            "jacobi_sweeps": {"fp64_max": stats["max_sweeps"], "fp32_max": stats["max_sweeps_fp32"],
                              "fallbacks": stats["fallbacks"]},
            "peak_probability_of_step": p,
            "autotune": {"what": "FP64 Jacobi warps per row pair, two sweeps of random matrices per shape "
                                 "(row length, matrices per launch); the fastest width is installed",
                         "shapes": tune_shapes, "ms_width_1_2_4": tune_ms.tolist(),
                         "chosen": [int([1, 2, 4][int(np.argmin(r))]) for r in tune_ms]},
            "measured_peaks": {"fp64_tflops": fp64_peak, "fp32_tflops": fp32_peak,
                               "how": "FMA-chain kernel over every SM inside this run (pc_measure_alu_peaks), "
                                      "best of three after a warm-up, CUDA events"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp64_peak, "traffic": None,
                         "kernel": f"class '{names[dom]}' (the largest timed share of the step)",
                         "flops_per_launch": dom_flops, "ms_per_launch": dom_ms,
                         "peak_source": "of measured: FP64 FMA-chain peak of this device in this run",
                         "traffic_note": "null: the kernels changed since the last DRAM capture",
                         "step": {"what": "whole step against the FP64 pipe: T_roof = algorithmic flops / "
                                          "FP64 peak (updates 4(4L^2v+22v^3), trials values-only "
                                          "4(4Lv^2-4v^3/3), merges and gates), frac = T_roof / T_measured; "
                                          "the bytes term (16.8 MB per chi=256 update) is < 1e-4 of T_roof",
                                  "alg_flops_per_step": alg_flops / args.steps, "t_roof_ms": t_roof_ms,
                                  "t_measured_ms": step_ms, "frac": t_roof_ms / step_ms}},
            "kernel_share": share,
            "gpu_launches": int(sum(launches)),
            "e2e": {"value": e2e_units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(sites_bytes + gate_bytes),
                    "d2h_bytes_per_step": int(N_SAMPLES * N_QUBITS + N_QUBITS + 8)},
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        if world == 1 and not args.no_m0:
            m0 = [measure_m0(binding, b, 0, trials=(b == 8), device=local) for b in M0_BATCHES]
            m0.append(measure_m0(binding, 8, 1, device=local))
            line["m0"] = {"workload": "independent chi=256 updates (1024 x 1024 bond matrices), random right "
                                      "isometries, geometric spectra exp(-k/64), Haar 16x16 operators, eps=1e-10, "
                                      "chi_max=256", "runs": m0}
        if world == 1 and not args.no_serving:
            line["time_to_peak"] = measure_hqap_time_to_peak(binding, local)
            small = W.circuit_mix(MIX_COUNT, seed=0)
            line["batching"] = measure_batching(
                binding, small, MIX_KW, f"{MIX_COUNT} hidden-permutation mirrors, n in [8,12], 12-24 Haar gates/half, "
                                        "perturbation in [0,0.04], chi_max=64, eps=1e-10, tau=3000")
            wide = W.circuit_mix(6, seed=2, n_range=(20, 32), gates_range=(4, 8), pert_range=(0.0, 0.04))
            line["batching_cfg4_shape"] = measure_batching(
                binding, wide, dict(eps=1e-10, chi_max=64, tau=1e4),
                "the 64-circuit batching configuration's qubit range at reduced scale: 6 hidden-permutation "
                "mirrors, n in [20,32], 4-8 Haar gates/half, perturbation in [0,0.04], chi_max=64, eps=1e-10, tau=1e4")
            cap = MIX_COUNT / line["batching"]["batched_s"]        # circuits/s the batch sustains
            line["serving"] = {"workload": "Poisson arrivals at 0.5x and 2x the batched capacity of the small mix; "
                                           "12 requests each, 100 samples each, eps=1e-5, chi_max=64",
                               "fp64": [measure_serving(binding, 0, f * cap) for f in (0.5, 2.0)],
                               "mixed": [measure_serving(binding, 1, f * cap) for f in (0.5, 2.0)]}
        print(json.dumps(line), flush=True)
    c.close()
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_profile_case(args):
    """One M0 configuration for a profiler: `--batch` independent chi=`--chi` updates,
    `--repeat` times, printed as JSON (kernel classes, sweeps, updates/s)."""
    import torch
    from paper_2604_21908_gb300 import binding
    torch.cuda.set_device(0)
    out = measure_m0(binding, args.batch, args.precision, chi=args.chi, reps=args.repeat, trials=args.trials)
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-serving", action="store_true", help="skip the batching and serving measurements")
    ap.add_argument("--pre-sweeps", type=int, default=0, help="FP32 preconditioning sweep cap (0: library default)")
    ap.add_argument("--no-m0", action="store_true", help="skip the batches of independent updates")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip timing the oracle on the host cores")
    ap.add_argument("--profile-case", action="store_true", help="run one M0 configuration and exit")
    ap.add_argument("--chi", type=int, default=256)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--trials", action="store_true", help="profile case: also one unswap stage")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
