"""Benchmark of the MC-MD hot path on one GB300 (or N replicas on N GPUs).

Workload: the 1152-lipid bilayer (24x24 per leaflet, 3 lipid types 40/40/20,
~20k water beads, 33.6k beads), FP32 pair arithmetic over a Verlet pair list,
FP64 exchange energies.  One step = one MC-MD round: 100 MD steps at dt = 20 fs
with one lipid-exchange trial after every MD step (the run of 10k steps with
one trial per step is 100 such steps).  Headline: pair interactions per second
(in-cutoff unordered pairs x MD steps / time); swap trials per second beside.

`--impl reference` times the FP64 CPU oracle on the host cores instead (the
reference arm: a deliberately plain program, not a target).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MD_PER_STEP = 100
PAIR_FLOPS = 30          # algorithmic FP32 flops of one pair interaction (FMA = 2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the replica and swap-throughput lines")
    ap.add_argument("--separate-launches", action="store_true",
                    help="one kernel launch per phase instead of the persistent kernel (same arithmetic; for profilers)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist, device):
    """The job's time is the slowest rank's: max of x over all ranks (x itself
    on one rank); device is where the collective's tensor lives ("cuda" for
    NCCL, "cpu" for gloo)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload():
    from paper_2005_08348_gb300 import synth
    return synth.mcmd_large()


def config(m, extra=None):
    c = {"workload": "mcmd-bilayer-1152-lipids-3-types", "lipids": int(m.n_lipids), "beads": int(m.n_beads),
         "box_nm": [round(float(x), 3) for x in m.box], "md_steps_per_step": MD_PER_STEP,
         "swap_trials_per_step": MD_PER_STEP, "dt_ps": 0.02, "temperature_K": 310.0,
         "l2": "flushed between steps (256 MB write, untimed)"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------- oracle
def host_cores():
    """Host cores this process may use (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:  # noqa: BLE001 - not every host has affinity masks
        return os.cpu_count() or 1


def oracle_rate(m, budget_s=12.0, min_evals=2, threads=False):
    """FP64 oracle: force evaluations + exchange trials on the same system
    until the time budget is spent, on one host thread or (threads=True, the
    OpenMP build) on all host cores."""
    import oracle
    o = oracle.Oracle(m, threads=threads)
    st = o.state()
    t0 = time.perf_counter()
    pairs = 0
    evals = 0
    trials = 0
    while evals < min_evals or time.perf_counter() - t0 < budget_s:
        terms, _ = o.energy(st["pos_u"], ltype=st["ltype"])
        pairs += terms["pairs"]
        evals += 1
        o.md_steps(st, 1, swap_every=1)
        evals += 1
        pairs += terms["pairs"]
        trials += 1
    dt = time.perf_counter() - t0
    return dict(pairs_per_s=pairs / dt, trials_per_s=trials / dt, evals=evals, seconds=dt)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    m = workload()
    import oracle
    cores = host_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    threads = oracle.lib_omp() is not None
    o = oracle.Oracle(m, threads=threads)
    st = o.state()
    pairs = o.energy(st["pos_u"], forces=False)[0]["pairs"]
    for _ in range(args.warmup):
        o.md_steps(st, 1, swap_every=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.md_steps(st, 1, swap_every=1)
    dt = time.perf_counter() - t0
    value = pairs * args.steps / dt
    used = cores if threads else 1
    sample = (f"{args.steps} oracle MD steps with one exchange trial each on the 1152-lipid system, "
              + (f"energies on {used} host cores (OpenMP build)" if threads else "one host thread"))
    print(json.dumps({
        "impl": "reference", "metric": "pair-interactions/s", "value": value, "unit": "pair-interactions/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config(m, {"reference_step": "1 MD step + 1 exchange trial (bounded sample)"}),
        "cpu_baseline": {"value": value, "unit": "pair-interactions/s", "cores": used, "kind": "oracle",
                         "sample": sample, "host_cores": cores},
        "e2e": {"value": value, "unit": "pair-interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "swap_trials_per_s": args.steps / dt,
    }))


# ---------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, path, index):
        self.path, self.index, self.p = path, index, None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p))
    return {}


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2005_08348_gb300 import mdas

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    m = workload()
    m.system_id = rank
    sysm = mdas.System(m, precision="fp32", stream=stream.cuda_stream)
    if args.separate_launches:
        sysm.set_persistent(False)
    n_pairs0 = sysm.energy()["pairs"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        sysm.md_steps(MD_PER_STEP, swap_every=1)
    sysm.set_kernel_timing(True)
    sysm.pair_kernel_time(reset=True)
    c0 = sysm.counters()
    # the nvidia-smi clock log of the timed region (BENCH_LOG_DIR, else the temp directory)
    clocks = Clocks(os.path.join(os.environ.get("BENCH_LOG_DIR") or tempfile.gettempdir(),
                                 f"bench_clocks_r{rank}.csv"), local)
    if not args.no_clocks:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        sysm.md_steps(MD_PER_STEP, swap_every=1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = None if args.no_clocks else clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    pair_ms, pair_launches = sysm.pair_kernel_time(reset=True)
    sysm.set_kernel_timing(False)
    c1 = sysm.counters()
    n_pairs1 = sysm.energy()["pairs"]
    pairs_per_eval = 0.5 * (n_pairs0 + n_pairs1)
    md = c1["md_steps"] - c0["md_steps"]
    trials = c1["trials"] - c0["trials"]
    tmax = max_over_ranks(total_ms, dist, "cuda") / 1e3
    value = pairs_per_eval * md * ws / tmax
    trials_per_s = trials * ws / tmax

    # end to end through the C ABI with pinned host buffers: upload the state
    # (mdas_set_state_packed: positions, velocities, lipid types), run a
    # round, read the state back (mdas_get_state_packed), every step
    n = m.n_beads
    hbuf = (torch.empty((n, 4), dtype=torch.int32).pin_memory(), torch.empty((n, 4), dtype=torch.float32).pin_memory(),
            torch.empty(m.n_lipids, dtype=torch.int32).pin_memory())
    sysm.get_state_packed(*hbuf)
    for _ in range(2):
        sysm.set_state_packed(*hbuf)
        sysm.md_steps(MD_PER_STEP, swap_every=1)
        sysm.get_state_packed(*hbuf)
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sysm.set_state_packed(*hbuf)
        sysm.md_steps(MD_PER_STEP, swap_every=1)
        sysm.get_state_packed(*hbuf)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, "cuda")   # the slowest rank's
    h2d = d2h = sum(t.numel() * t.element_size() for t in hbuf)   # every array, each way, every step
    e2e_value = pairs_per_eval * MD_PER_STEP * ws / e2e_s

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s at the maximum SM clock
    # the MD kernel's time per MD step (the persistent kernel: the step, its
    # share of list rebuilds and the exchange trial)
    pair_avg_s = pair_ms / max(1, pair_launches) / 1e3
    achieved = pairs_per_eval * PAIR_FLOPS / pair_avg_s / 1e12 if pair_launches else None
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")
    if os.path.exists(tfile) and not args.separate_launches:
        # DRAM bytes of one step-kernel launch from an ncu capture of this
        # workload; void once the kernel source has changed since the capture
        import hashlib
        tj = json.load(open(tfile))
        h = hashlib.sha256()
        for name in tj.get("sources", []):
            src = os.path.join(ROOT, "paper_2005_08348_gb300", "csrc", name)
            h.update(open(src, "rb").read() if os.path.exists(src) else b"missing")
        if tj.get("sources") and tj.get("beads") == n and tj.get("sources_sha256") == h.hexdigest():
            traffic = tj.get("bytes_per_launch")
    out = {
        "metric": "pair-interactions/s", "value": value, "unit": "pair-interactions/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded bilayer, no trained parameters)",
        "config": config(m, {"parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                             "pairs_per_force_eval": pairs_per_eval,
                             "launches": "separate kernels" if args.separate_launches else "persistent kernel"}),
        "swap_trials_per_s": trials_per_s, "md_steps_per_s": md * ws / tmax,
        "gpu_launches": int(c1["kernel_launches"] - c0["kernel_launches"]),
        "e2e": {"value": e2e_value, "unit": "pair-interactions/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "roofline": {"kernel": "k_nl_step<float> + list build + trial kernels (separate launches)"
                     if args.separate_launches else
                     "k_md_run<float> (persistent: MD steps, list rebuilds, exchange trials)",
                     "bound": "alu", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": (achieved / fp32_peak) if achieved else None,
                     "traffic": traffic, "us_per_md_step": pair_avg_s * 1e6, "md_steps_timed": pair_launches,
                     "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (MEASURED_PEAKS sm_max_mhz)",
                     "flops_per_pair": PAIR_FLOPS},
        "clocks": clk,
        "wall_s_timed": wall,
    }
    # the informational lines and the CPU baseline belong to the one-GPU run
    # (a multi-GPU run would hold every GPU while rank 0 alone works on them)
    if not args.no_extra and ws == 1:
        out["batched_replicas"] = _extra(replica_benchmark, stream)
        out["swap_trials_4608_lipids"] = _extra(swap_benchmark, stream)
        out["mdas_4608_lipids"] = _extra(mdas_benchmark, stream)
        out["mutations_4608_lipids"] = _extra(mutation_benchmark, stream)
        out["head_rdf_4608_lipids"] = _extra(rdf_benchmark, stream)
        out["npt_1152_lipids"] = _extra(npt_benchmark, stream)
        out["fp64_mcmd_128_lipids"] = _extra(fp64_benchmark, stream)
        out["served"] = _extra(serving_benchmark, stream)
    if not args.no_cpu_baseline and ws == 1:
        import oracle
        cores = host_cores()
        os.environ.setdefault("OMP_NUM_THREADS", str(cores))
        one = oracle_rate(m, budget_s=8.0)
        omp = oracle_rate(m, budget_s=8.0, threads=True) if oracle.lib_omp() is not None else None
        ob, used = (omp, cores) if omp else (one, 1)
        out["cpu_baseline"] = {"value": ob["pairs_per_s"], "unit": "pair-interactions/s", "cores": used,
                               "kind": "oracle", "sample": f"{ob['evals']} FP64 force evaluations "
                               f"(half of them inside oracle MD steps with one exchange trial) on the same "
                               f"1152-lipid system, {ob['seconds']:.1f} s, "
                               + (f"{used} host cores (OpenMP build of the oracle)" if omp else "one host thread"),
                               "swap_trials_per_s": ob["trials_per_s"], "host_cores": cores,
                               "single_thread": {"value": one["pairs_per_s"], "cores": 1,
                                                 "swap_trials_per_s": one["trials_per_s"],
                                                 "sample": f"{one['evals']} force evaluations, {one['seconds']:.1f} s"}}
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def _elapsed(stream, fn):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3


def replica_benchmark(stream, n_rep=64, rounds=3):
    """64 independent bilayers of 128-2048 lipids, each advanced by 100 MD
    steps + 100 exchange trials per round: all replicas in one launch per
    phase (mdas_batch_run) against one replica at a time, both with the
    pair-list skin the autotuner picks for the batch; the batch also takes the
    tuner's layout and step shape, each replica run alone its own faster
    shape (four lanes while its step items fit one wave of the GPU's groups,
    else two) and the faster exchange-trial path."""
    from paper_2005_08348_gb300 import mdas, synth
    ms = synth.replica_set(n_rep)
    skin, part, wave, lanes, tune = mdas.tune_batch(ms, skins=(0.3, 0.35), waves=(0,), lanes=(2, 4),
                                                    md_steps=MD_PER_STEP, swap_trials=MD_PER_STEP, rounds=1,
                                                    stream=stream.cuda_stream)
    sys_b = [mdas.System(m, stream=stream.cuda_stream, list_skin=skin) for m in ms]
    sys_s = [mdas.System(m, stream=stream.cuda_stream, list_skin=skin) for m in ms]
    for s in sys_b:
        s.set_partitioned(part)
        s.set_batch_wave(wave)
        s.set_list_lanes(lanes)
    # a lone replica's faster step shape: four lanes while its four-lane step
    # items and its trial and close groups fit one wave of the persistent
    # kernel's groups (152 SMs x 8), else two (measured crossover)
    groups = 152 * 8
    solo_lanes = [4 if (m.n_beads + 31) // 32 + 17 <= groups else 2 for m in ms]
    for s, ln in zip(sys_s, solo_lanes):
        s.set_list_lanes(ln)
    pairs = sum(s.energy()["pairs"] for s in sys_b)
    mdas.batch_run(sys_b, MD_PER_STEP, MD_PER_STEP)
    for s in sys_s:
        s.md_steps(MD_PER_STEP)
        s.swap_trials(MD_PER_STEP, log=False)

    def batched():
        for _ in range(rounds):
            mdas.batch_run(sys_b, MD_PER_STEP, MD_PER_STEP)

    def solo():
        for _ in range(rounds):
            for s in sys_s:
                s.md_steps(MD_PER_STEP)
                s.swap_trials(MD_PER_STEP, log=False)

    # one replica at a time with whichever exchange-trial path is faster for
    # it (each has its own best shape: four lanes, and here the trial path)
    tb = _elapsed(stream, batched)
    ts_path = {}
    for path in ("sequential", "speculative"):
        for s in sys_s:
            s.set_trial_path(path)
        ts_path[path] = _elapsed(stream, solo)
    solo_path = min(ts_path, key=ts_path.get)
    ts = ts_path[solo_path]
    md = rounds * MD_PER_STEP
    res = {"workload": f"{n_rep} replicas, {sum(m.n_lipids for m in ms)} lipids, {sum(m.n_beads for m in ms)} beads",
           "batched_pair_interactions_per_s": pairs * md / tb, "one_at_a_time_pair_interactions_per_s": pairs * md / ts,
           "batched_swap_trials_per_s": n_rep * md / tb, "one_at_a_time_swap_trials_per_s": n_rep * md / ts,
           "speedup": ts / tb, "rounds": rounds, "list_skin_nm": skin,
           "layout": "partitioned (systems advance independently)" if part else "lockstep (kernel-wide barriers)",
           "wave_beads": wave or "all", "list_lanes_per_bead": lanes,
           "one_at_a_time_list_lanes_per_bead": {"4": solo_lanes.count(4), "2": solo_lanes.count(2)},
           "trial_path": "sequential", "one_at_a_time_trial_path": solo_path,
           "one_at_a_time_ms_per_round_by_trial_path": {k: round(1e3 * v / rounds, 2) for k, v in ts_path.items()},
           "autotune_us_per_md_step": {f"skin {k[0]:g} {'partitioned' if k[1] else 'lockstep'} wave {k[2] or 'all'} "
                                       f"lanes {k[3]}": round(v, 2) for k, v in tune.items()}}
    for s in sys_b + sys_s:
        s.close()
    return res


def mdas_benchmark(stream, n_moves=6):
    """MDAS moves on the 4608-lipid bilayer (~140k beads): 8 pairs (16
    lipids) exchanged along 10 lambda steps of 5 MD steps each, FP32 pair
    arithmetic, FP64 work; the linear path (Eq. 2) and the soft-core path
    (Eq. 4, delta = 0.05 nm^2)."""
    from paper_2005_08348_gb300 import mdas, synth
    m = synth.mdas_patch()
    res = {"workload": f"{m.n_lipids} lipids, {m.n_beads} beads; 8 pairs, 10 lambda steps x 5 MD steps",
           "force_evaluations_per_move": 10 * 5 + 10, "moves": n_moves}
    for name, delta in (("", 0.0), ("soft_core_", 0.05)):
        s = mdas.System(m, stream=stream.cuda_stream)
        if delta > 0:
            s.set_soft_core(delta)
        s.alchemical_move(8, 10, 5)
        acc = []

        def moves():
            for _ in range(n_moves):
                acc.append(s.alchemical_move(8, 10, 5)["accepted"])

        t = _elapsed(stream, moves)
        res[name + "moves_per_s"] = n_moves / t
        res[name + "ms_per_move"] = 1e3 * t / n_moves
        res[name + "accepted"] = int(sum(acc))
        s.close()
    return res


def mutation_benchmark(stream, n_batch=1024):
    """Semi-grand single-lipid mutations (Sec. 2) on the 4608-lipid bilayer:
    batches of 1024 trials with per-type chemical potentials."""
    from paper_2005_08348_gb300 import mdas, synth
    m = synth.mdas_patch()
    s = mdas.System(m, stream=stream.cuda_stream)
    mu = [0.0, 0.5, -0.3]
    s.mutation_trials(n_batch, mu=mu, log=False)
    stats = {}

    def batch():
        st, _ = s.mutation_trials(n_batch, mu=mu, log=False)
        stats.update(st)

    t = _elapsed(stream, batch)
    s.close()
    return {"workload": f"{m.n_lipids} lipids, {m.n_beads} beads; {n_batch} trials per call, mu = {mu} kJ/mol",
            "trials_per_s": n_batch / t, "accepted": int(stats.get("accepted", 0))}


def _extra(fn, stream):
    """An informational entry; a failure is reported in the line, not raised."""
    try:
        return fn(stream)
    except Exception as e:  # noqa: BLE001 - the headline line must still print
        return {"error": f"{type(e).__name__}: {e}"[:300]}


def rdf_benchmark(stream, n_calls=50):
    """The mixing observable (in-plane head-bead pair counts of one lipid
    type per leaflet) on the 4608-lipid bilayer after some MD: one
    mdas_head_rdf call (kernels, a 1 KB copy back), against the oracle's
    O(N^2) count of the same pairs on one host core."""
    import oracle
    from paper_2005_08348_gb300 import mdas, synth
    m = synth.mdas_patch()
    s = mdas.System(m, stream=stream.cuda_stream)
    s.md_steps(50, swap_every=0)
    s.head_rdf(0, 1, 3.0, 60)
    t = _elapsed(stream, lambda: [s.head_rdf(0, 1, 3.0, 60) for _ in range(n_calls)]) / n_calls
    st = s.get_state()
    o = oracle.Oracle(m)
    t0 = time.perf_counter()
    co, nho = o.head_rdf(st["pos_u"], st["ltype"], 0, 1, 3.0, 60)
    t_or = time.perf_counter() - t0
    c, nh = s.head_rdf(0, 1, 3.0, 60)
    s.close()
    return {"workload": f"{m.n_lipids} lipids, type 0 heads, 60 bins to 3 nm", "us_per_call": t * 1e6,
            "oracle_ms_per_call": t_or * 1e3, "heads": [int(x) for x in nh], "pairs_counted": int(c.sum()),
            "equal_to_oracle": bool((c == co).all() and (nh == nho).all())}


def npt_benchmark(stream, n_steps=1000):
    """The bench bilayer (1152 lipids) at constant pressure (semi-isotropic
    Parrinello-Rahman, 1 bar, 12 ps, a box update every 10 steps) against
    the same MD at constant volume, one exchange trial after every step.
    The synthetic bilayer is not equilibrated (it relaxes from about +1700
    bar to below zero within picoseconds), so at the paper's 12 ps its box
    would shrink by several percent during the timed steps and the two runs
    would sum different numbers of pairs.  The cost of the coupling (virial
    sums, box updates, segment ends) is the same for any coupling constant:
    tau_p = 10^4 ps keeps the box at its start, and the box update still
    runs every 10 steps."""
    from paper_2005_08348_gb300 import mdas, synth
    m = synth.mcmd_large()
    tau_p = 1e4
    out = {"workload": f"{m.n_lipids} lipids, {m.n_beads} beads; {n_steps} MD steps + trials",
           "pcouple": {"p_ref_bar": 1.0, "tau_p_ps": tau_p, "compressibility_per_bar": 3e-4, "nstpcouple": 10}}
    for name, pc in (("nvt", None), ("npt", dict(p_ref=1.0, tau_p=tau_p, compressibility=3e-4, nstpcouple=10))):
        s = mdas.System(m, stream=stream.cuda_stream, pcouple=pc)
        s.md_steps(100, swap_every=1)
        t = _elapsed(stream, lambda: s.md_steps(n_steps, swap_every=1))
        out[f"{name}_md_steps_per_s"] = n_steps / t
        if pc:
            box, _, p = s.box()
            out["box_nm_after"] = [round(float(x), 5) for x in box]
            out["pressure_bar_last_update"] = [round(float(x), 2) for x in p]
        s.close()
    out["npt_over_nvt_time"] = out["nvt_md_steps_per_s"] / out["npt_md_steps_per_s"]
    return out


def fp64_benchmark(stream, rounds=10):
    """Plain MC-MD in FP64 on the 128-lipid bilayer: rounds of 200 MD steps
    with one exchange trial every 10 steps (the FP64 workload the oracle runs
    in lockstep in the parity tests), and the same rounds in FP32."""
    from paper_2005_08348_gb300 import mdas, synth
    m = synth.mcmd_small()
    out = {"workload": f"{m.n_lipids} lipids, {m.n_beads} beads; 200 MD steps + 20 trials per round"}
    for prec in ("fp64", "fp32"):
        s = mdas.System(m, precision=prec, stream=stream.cuda_stream)
        s.md_steps(200, swap_every=10)
        pairs = s.energy()["pairs"]
        t = _elapsed(stream, lambda: [s.md_steps(200, swap_every=10) for _ in range(rounds)])
        out[f"{prec}_md_steps_per_s"] = 200 * rounds / t
        out[f"{prec}_pair_interactions_per_s"] = pairs * 200 * rounds / t
        out[f"{prec}_swap_trials_per_s"] = 20 * rounds / t
        s.close()
    return out


def swap_benchmark(stream, n_batch=1024, n_plain=300):
    """Exchange trials on the 4608-lipid bilayer (~140k beads): one trial per
    call (the plain path) against calls of 1024 trials, each on both trial
    paths (one after another from the pair lists, the default; speculative
    rounds); the ratio is the default batched path over the faster plain
    one."""
    from paper_2005_08348_gb300 import mdas, synth
    m = synth.mdas_patch()
    s = mdas.System(m, stream=stream.cuda_stream)
    out = {"workload": f"{m.n_lipids} lipids, {m.n_beads} beads", "batch": n_batch}
    for path in ("speculative", "sequential"):
        s.set_trial_path(path)
        s.swap_trials(16, log=False)
        t_plain = _elapsed(stream, lambda: [s.swap_trials(1, log=False) for _ in range(n_plain)])
        s.swap_trials(n_batch, log=False)
        t_batch = _elapsed(stream, lambda: s.swap_trials(n_batch, log=False))
        out[f"plain_trials_per_s_{path}"] = n_plain / t_plain
        out[f"batched_trials_per_s_{path}"] = n_batch / t_batch
    s.close()
    out["plain_trials_per_s"] = max(out["plain_trials_per_s_speculative"], out["plain_trials_per_s_sequential"])
    out["batched_trials_per_s"] = out["batched_trials_per_s_sequential"]
    out["ratio"] = out["batched_trials_per_s"] / out["plain_trials_per_s"]
    return out


def serving_benchmark(stream, n_jobs=500, n_patches=48, seed=1005):
    """Served sampling on device-resident patches: 48 seeded patches whose
    sizes are log-uniform over 128-16384 lipids (2-3 types) are added to the
    server once; each job draws its patch uniformly (so patch sizes are
    log-uniform per job) and its kind from the mix 60% 256 swap trials / 30%
    100 MD steps / 10% one MDAS move (8 pairs = 16 lipids, 10 lambda steps of
    5 MD steps); a patch's jobs run in order on its state.  Poisson arrivals
    at 0.25x, 0.5x and 0.9x of the saturation throughput measured first (all
    jobs submitted at once).  Beside it, the plain path: the same jobs on the
    same device-resident systems, one job at a time through the one-system
    calls (no batching)."""
    import numpy as np
    from paper_2005_08348_gb300 import mdas, synth
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(128), np.log(16384), n_patches)).astype(int) // 2 * 2
    pool = [synth.patch(int(n), int(rng.integers(2, 4)), seed=seed * 100 + k, system_id=k)
            for k, n in enumerate(sizes)]

    def draw_jobs(r):
        out = []
        for _ in range(n_jobs):
            x = r.uniform()
            kind, n = (mdas.JOB_SWAPS, 256) if x < 0.6 else ((mdas.JOB_MD, 100) if x < 0.9 else (mdas.JOB_MDAS, 0))
            out.append((int(r.integers(0, n_patches)), kind, n))
        return out

    sv = mdas.Server(64 << 30, max_active=64, md_quantum=25, stream=stream.cuda_stream)
    pids = [sv.add_patch(p) for p in pool]

    def serve(jobs, arrivals):
        t0 = sv.clock()
        k = 0
        done = []
        while len(done) < len(jobs):
            now = sv.clock() - t0
            while k < len(jobs) and arrivals[k] <= now:
                q, kind, n = jobs[k]
                sv.submit_to(pids[q], kind, n=n, n_pairs=8, n_lambda=10, md_per_lambda=5)
                k += 1
            a, qd = sv.run(1)
            done += sv.results()
            if a == 0 and qd == 0 and k < len(jobs):
                time.sleep(max(0.0, min(0.002, arrivals[k] - (sv.clock() - t0))))
        span = max(r["t_done"] for r in done) - t0
        lat = np.array([r["t_done"] - r["t_submit"] for r in done])
        return span, lat

    plain_sys = [mdas.System(p, stream=stream.cuda_stream) for p in pool]

    def plain(jobs):
        t0 = time.perf_counter()
        for q, kind, n in jobs:
            s = plain_sys[q]
            if kind == mdas.JOB_MD:
                s.md_steps(n)
            elif kind == mdas.JOB_SWAPS:
                s.swap_trials(n, log=False)
            else:
                s.alchemical_move(8, 10, 5)
        return time.perf_counter() - t0

    jobs = draw_jobs(np.random.default_rng(seed + 1))
    serve(jobs[:32], [0.0] * 32)                        # warm-up
    plain(jobs[:32])
    t_plain = plain(jobs)
    span, lat = serve(jobs, [0.0] * n_jobs)
    sat = n_jobs / span
    lipids = np.array([pool[q].n_lipids for q, _, _ in jobs])
    res = {"workload": f"{n_jobs} jobs per rate on {n_patches} device-resident patches of "
                       f"{int(sizes.min())}-{int(sizes.max())} lipids (log-uniform sizes), patch drawn per job",
           "job_lipids_median": int(np.median(lipids)), "job_lipids_max": int(lipids.max()),
           "saturation_jobs_per_s": sat, "plain_one_at_a_time_jobs_per_s": n_jobs / t_plain,
           "served_over_plain": sat * t_plain / n_jobs, "rates": []}
    for frac in (0.25, 0.5, 0.9):
        r = np.random.default_rng(seed + int(frac * 100))
        arr = np.cumsum(r.exponential(1.0 / (frac * sat), n_jobs))
        span, lat = serve(jobs, list(arr))
        res["rates"].append({"load": frac, "arrival_jobs_per_s": frac * sat, "throughput_jobs_per_s": n_jobs / span,
                             "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                             "max_ms": float(lat.max() * 1e3)})
    for s in plain_sys:
        s.close()
    sv.close()
    return res


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
