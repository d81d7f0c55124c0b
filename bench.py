#!/usr/bin/env python3
"""Benchmark of the ER-Euler / invert-Krylov transient on one GB300.

Workload: linear 3D RC power-grid mesh 100 x 100 x 100 (1M nodes), 6-neighbour conductances
0.1-10 S, ground caps 1 fF - 1 pF, 100 top-layer pads, 10k pulse loads; G factored once;
adaptive step (Alg. 2) with the Krylov dimension from the Eq.-16 residual test (eps 1e-7)
and tol 1e-6 over 2 ns.  A timed "step" is one accepted ER step (setup solves, the phi_1 and
phi_2 Krylov spaces, the update, the controller).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload batch      (batched Monte Carlo inverter chains, plain vs learned)
  python bench.py --workload solve --size 70   (the supernodal solves alone, for profiling)
  python bench.py --workload mesh2d --steps 1000  (the 32x32 mesh at fixed h and m alone)

Prints one JSON line (rank 0).  The value is accepted ER steps per second of the whole job;
N > 1 runs independent replicas (a single circuit does not shard: every G^-1 couples all
nodes), one per GPU.  --impl reference times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ER-Euler steps/s & Krylov vectors/s at rel err 1e-6; plain vs batched+learned"
UNIT = "steps/s"
FP64_FMA_PER_CLK_PER_SM = 2        # GB300: FP64 issue rate per SM (1/64 of FP32)
# DRAM bytes / algorithmic bytes of one solve pair, from an ncu capture of the same kernels on
# the 70^3 mesh; the full-size traffic is this ratio times the full-size algorithmic bytes
# (traffic grows with the factor).  Set to None whenever k_trsv_fwd / k_trsv_bwd change until
# a new capture is taken.
SOLVE_TRAFFIC_RATIO = 2.156 / 2.023
SOLVE_TRAFFIC_SOURCE = ("ncu dram bytes of the 70^3 pair (k_trsv_fwd<2,3,0> + k_trsv_bwd<2,3,0>, "
                        "ordering 1: 2.156 GB vs 2.023 GB algorithmic) scaled to the 100^3 pair "
                        "by its algorithmic bytes")
CLOCKS_DIR = os.environ.get("ERS_CLOCKS_DIR") or os.path.join(ROOT, ".bench")   # nvidia-smi samples
L2_BYTES = 129 * 2 ** 20              # GB300 L2; smaller factors get an L2 flush before each step
FLUSH_BYTES = 256 * 2 ** 20
SAMPLE_SIZE = 24                   # oracle sample: 24^3 mesh of the same generator
SAMPLE_STEPS = 40


def ordering_kw(a):
    """--ordering for ers.make_opts: nothing when the library default is meant."""
    return {} if a.ordering is None else {"ordering": a.ordering}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--size", type=int, default=100, help="mesh edge (workload: 100)")
    p.add_argument("--tol", type=float, default=1e-6)
    p.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle leg")
    p.add_argument("--no-extras", action="store_true",
                   help="main line only (no accuracy run, config [0] / [2] / batch sub-lines)")
    p.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--workload", default="mesh",
                   choices=["mesh", "chain", "batch", "solve", "mesh2d"])
    p.add_argument("--ordering", type=int, default=None,
                   help="ers_opts.ordering (0 or 1; default: the library's)")
    p.add_argument("--nrhs", type=int, default=2, help="solve: right-hand sides per pass")
    p.add_argument("--stages", type=int, default=2000, help="chain: inverter stages")
    p.add_argument("--batch-n", type=int, default=64, help="batch: instances")
    p.add_argument("--stage-lo", type=int, default=4)
    p.add_argument("--stage-hi", type=int, default=40)
    p.add_argument("--tree", type=int, default=20, help="batch: RC tree nodes per stage")
    p.add_argument("--t-end", type=float, default=0.3e-9)
    p.add_argument("--train-n", type=int, default=16)
    p.add_argument("--ctrl-parts", type=int, default=1,
                   help="batch: learned proposals used (1 step size, 2 Krylov dimension, 3 both)")
    p.add_argument("--ctrl-margin", type=float, default=0.3,
                   help="batch: log2 margin subtracted from proposed step ratios")
    p.add_argument("--seq-sample", type=int, default=4,
                   help="batch: instances timed one context at a time")
    return p.parse_args()


def workload(size, kind="mesh", stages=2000):
    from synth import circuits as S
    if kind == "chain":
        return S.inverter_chain(stages=stages, tree_nodes=100, seed=2, t_end=5e-9)
    loads = 10000 if size == 100 else max(1, (size ** 3) // 100)
    return S.rc_mesh_3d(size, size, size, seed=1, n_loads=loads)


def workload_t_end(kind):
    return 5e-9 if kind == "chain" else 2e-9


def workload_name(size, kind="mesh", stages=2000):
    if kind == "chain":
        return (f"invchain_{stages}x100: nonlinear inverter chain, {stages} stages x 100-node "
                f"RC trees ({stages * 100 + 1} nodes), square-law MOSFETs, LU refactor of G_k "
                f"every step, adaptive h (tol 1e-6, eps 1e-7), first steps from DC over 5 ns")
    return (f"rc3d_{size}x{size}x{size}: linear 3D RC power-grid mesh ({size ** 3} nodes), "
            f"pulse loads, G factored once, adaptive h (tol 1e-6, eps 1e-7) over 2 ns")


# --------------------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------------------
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clocks_start(gpu_index, path):
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={CLOCK_Q}",
                                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=f,
                                stderr=subprocess.DEVNULL), f
    except OSError:
        return None, None


def clocks_stop(proc, f, path):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    f.close()
    sm, smax, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax = max(smax, float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
            "samples": len(sm)}


# --------------------------------------------------------------------------------------
# oracle (CPU) sample: runs in a fresh single-threaded interpreter
# --------------------------------------------------------------------------------------
def oracle_sample(steps=SAMPLE_STEPS, size=SAMPLE_SIZE, kind="mesh", stages=2000):
    import numpy as np
    from oracle import ers_oracle as O
    circ = workload(size, kind, stages)
    x0 = O.dc_solution(circ, x0=circ.nodeset) if kind == "chain" else np.zeros(circ.n)
    t0 = time.perf_counter()
    x, t, st = O.er_run(circ, t_end=workload_t_end(kind), tol=1e-6, max_steps=steps, x0=x0)
    dt = time.perf_counter() - t0
    return {"steps": st.steps, "seconds": dt, "krylov": st.krylov, "t_reached": t, "n": circ.n}


def run_oracle_sample(steps=SAMPLE_STEPS, size=SAMPLE_SIZE, kind="mesh", stages=2000):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--steps", str(steps),
           "--size", str(size), "--workload", kind, "--stages", str(stages)]
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])
    value = r["steps"] / r["seconds"]
    what = (f"the {size}^3 mesh ({r['n']} nodes, same generator and seed) from x = 0"
            if kind == "mesh" else
            f"the {stages}-stage chain ({r['n']} nodes, same generator and seed) from DC")
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "n_sample": r["n"],
            "sample": (f"first {r['steps']} adaptive ER steps of {what}, the oracle's own "
                       f"sparse LU + numpy, 1 thread, {r['seconds']:.1f} s; steps/s on the "
                       f"sample, not scaled to the full workload"),
            "krylov_vectors_per_s": r["krylov"] / r["seconds"]}


# --------------------------------------------------------------------------------------
def oracle_args(a):
    """(steps, size, kind, stages) of the bounded oracle sample: 40 steps of a 24^3 mesh, or
    100 steps of a 100-stage chain (about 10 s of one host core each)."""
    if a.workload == "chain":
        return 100, SAMPLE_SIZE, "chain", 100
    return SAMPLE_STEPS, SAMPLE_SIZE, "mesh", 2000


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(a.warmup):
        run_oracle_sample(2, *oracle_args(a)[1:])
    t0 = time.perf_counter()
    kind = "chain" if a.workload == "chain" else "mesh"
    vals = [run_oracle_sample(*oracle_args(a)) for _ in range(max(1, a.steps // 5))]
    wall = time.perf_counter() - t0
    v = statistics.median(x["value"] for x in vals)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_name(a.size, kind, a.stages),
                       "sample_of": "oracle on a reduced circuit of the same generator",
                       "parallelism": "host cores, rank 0"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


def timed_adaptive(sim, t_end, tol, steps, stream, factor_bytes):
    """Time `steps` accepted Algorithm-2 steps on the library's stream with CUDA events: back to
    back when the factor exceeds L2, else each step after a 256 MB write that evicts L2 (the
    write outside the per-step events).  Returns (ms, steps, rejects, l2 note)."""
    import torch
    if factor_bytes > L2_BYTES:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ns, nr = sim.run(t_end, 1e-6 if tol is None else tol, max_steps=steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), ns, nr, "inputs larger than L2 (factor values alone exceed 129 MB)"
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    ns = nr = 0
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(k)
        evs[k][0].record(stream)
        s_k, r_k = sim.run(t_end, tol, max_steps=1)
        evs[k][1].record(stream)
        ns += s_k
        nr += r_k
    torch.cuda.synchronize()
    note = (f"L2 flushed before every step ({FLUSH_BYTES >> 20} MB write on the library's "
            f"stream, outside the per-step events): the factor is {factor_bytes / 1e6:.1f} MB")
    return sum(b.elapsed_time(c) for b, c in evs), ns, nr, note


def chain_line(ers, stream, steps=10, warmup=3):
    """Config [2]: the 2000-stage inverter chain with 100-node RC trees, refactor of G_k every
    step, adaptive h (tol 1e-6, eps 1e-7), steps from DC on the first input edge."""
    import torch
    circ = workload(0, "chain", 2000)
    t_end = workload_t_end("chain")
    sim = ers.Simulator.from_circuit(circ, opts=ers.make_opts(eps_krylov=1e-7, h_max=t_end / 100))
    sim.set_stream(stream)
    sim.dc(circ.nodeset)
    tuned, _ = sim.autotune(nrhs=2, passes=3)
    sim.run(t_end, 1e-6, max_steps=warmup)
    torch.cuda.synchronize()
    st0 = sim.stats()
    ms, ns, nr, note = timed_adaptive(sim, t_end, 1e-6, steps, stream, st0["factor_doubles"] * 8)
    st1 = sim.stats()
    out = {"workload": workload_name(0, "chain", 2000), "n": circ.n, "steps": int(ns),
           "rejects": int(nr), "ms_per_step": ms / max(ns, 1), "steps_per_s": ns / (ms * 1e-3),
           "krylov_vectors_per_s": (st1["krylov_vectors"] - st0["krylov_vectors"]) / (ms * 1e-3),
           "refactors": st1["refactors"] - st0["refactors"],
           "gpu_launches_per_step": (st1["kernel_launches"] - st0["kernel_launches"]) / max(ns, 1),
           "host_syncs_per_step": (st1["host_syncs"] - st0["host_syncs"]) / max(ns, 1),
           "host_polls_per_step": (st1["host_polls"] - st0["host_polls"]) / max(ns, 1),
           "solve_ctas_per_sm": tuned, "l2_flush": note}
    sim.close()
    return out


def mesh2d_line(ers, stream, steps=1000):
    """Config [0]: the 32 x 32 RC mesh, plain ER at fixed h = 1 ps and m = 20 from x = 0 over
    1 ns (1000 steps; the pulse corners lie on the 1 ps grid)."""
    import numpy as np
    import torch
    from synth import circuits as S
    circ = S.rc_mesh_2d(32, 32, seed=0)
    sim = ers.Simulator.from_circuit(circ)
    sim.set_stream(stream)
    sim.set_state(0.0, np.zeros(circ.n))
    sim.step(1e-12, 20)                       # factor G once, warm the kernels
    tuned, tune_ms = sim.autotune(nrhs=1, passes=5)   # resident CTAs per SM of the solves
    sim.set_state(0.0, np.zeros(circ.n))
    torch.cuda.synchronize()
    st0 = sim.stats()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        flush.fill_(1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sim.step(1e-12, 20)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st1 = sim.stats()
    out = {"workload": "rc2d_32x32: linear 2D RC mesh (1024 nodes), 16 pulse sources, fixed "
                       "h = 1 ps, Krylov m = 20, 1000 steps over 1 ns from x = 0",
           "steps": steps, "ms_per_step": ms / steps, "steps_per_s": steps / (ms * 1e-3),
           "krylov_vectors_per_s": (st1["krylov_vectors"] - st0["krylov_vectors"]) / (ms * 1e-3),
           "gpu_launches_per_step": (st1["kernel_launches"] - st0["kernel_launches"]) / steps,
           "host_syncs_per_step": (st1["host_syncs"] - st0["host_syncs"]) / steps,
           "solve_ctas_per_sm": tuned, "autotune_ms_per_pass_at_1_2_3": tune_ms,
           "l2_flush": ("one 256 MB write before the run; the 1024-node factor stays in L2 "
                        "across the 1000 steps of the run, as in any use of this size")}
    sim.close()
    return out


def run_ours(a):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1511_04515_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1511_04515_gb300 import ers

    kind = "chain" if a.workload == "chain" else "mesh"
    circ = workload(a.size, kind, a.stages)
    t_end = workload_t_end(kind)
    opts = ers.make_opts(eps_krylov=1e-7, h_max=t_end / 100, **ordering_kw(a))
    tc = time.perf_counter()
    sim = ers.Simulator.from_circuit(circ, opts=opts)
    create_s = time.perf_counter() - tc
    stream = torch.cuda.Stream()          # the library's stream; events are recorded on it
    sim.set_stream(stream)
    tf = time.perf_counter()
    sim.dc(circ.nodeset)                   # x(0): Newton (linear: factor G once + one solve)
    torch.cuda.synchronize()
    factor_s = time.perf_counter() - tf
    tuned, tune_ms = sim.autotune(nrhs=2, passes=3)     # resident CTAs per SM of the solves
    if a.warmup:
        sim.run(t_end, a.tol, max_steps=a.warmup)
    t_start, x_start, h_start = sim.state()   # start of the timed window (accuracy check)
    sim.profile(True)
    st0 = sim.stats()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk_path = os.path.join(CLOCKS_DIR, f"clocks_rank{rank}.csv")
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    proc, fh = clocks_start(local, clk_path)
    factor_bytes = st0["factor_doubles"] * 8
    torch.cuda.nvtx.range_push("ers_timed")
    ms, ns, nr, l2_note = timed_adaptive(sim, t_end, a.tol, a.steps, stream, factor_bytes)
    torch.cuda.nvtx.range_pop()
    if world > 1:
        torch.distributed.barrier()
    clocks = clocks_stop(proc, fh, clk_path)
    st1 = sim.stats()
    steps = st1["steps"] - st0["steps"]
    kvec = st1["krylov_vectors"] - st0["krylov_vectors"]
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    passes = st1["solve_passes"] - st0["solve_passes"]
    rhs = st1["solve_rhs"] - st0["solve_rhs"]
    solve_ms = st1["solve_ms"]
    tot = torch.tensor([ms, float(steps), float(kvec)], device="cuda")
    if world > 1:
        mx = tot.clone()
        torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
        sm_ = tot.clone()
        torch.distributed.all_reduce(sm_, op=torch.distributed.ReduceOp.SUM)
        ms_max, steps_all, kvec_all = float(mx[0]), float(sm_[1]), float(sm_[2])
    else:
        ms_max, steps_all, kvec_all = ms, float(steps), float(kvec)

    # end to end through the public API with host buffers: state H2D, one step, state D2H
    n = circ.n
    t_now, x_host, h_now = sim.state()
    k_e2e = max(1, min(a.steps, 5))
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(k_e2e):
        sim.set_state(t_now, x_host, h_now)
        sim.run(t_end, a.tol, max_steps=1)
        t_now, x_host, h_now = sim.state()
    e2e_s = time.perf_counter() - te

    if rank != 0:
        sim.close()
        return
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = (clocks or {}).get("sm_max_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    derived_peak = nsm * FP64_FMA_PER_CLK_PER_SM * 2 * sm_max * 1e6 / 1e12   # TFLOP/s
    try:          # the FP64 FMA rate measured on this GPU now (a library kernel)
        alu_peak = ers.fp64_fma_peak(local)
        peak_src = ("measured: ers_fp64_fma_peak on this GPU (8 independent FMA chains per "
                    "thread, 8 x 256 threads per SM, best of 5, CUDA events)")
    except Exception:
        alu_peak = derived_peak
        peak_src = (f"derived: {nsm} SMs x {FP64_FMA_PER_CLK_PER_SM} FP64 FMA/clk x 2 flops x "
                    f"{sm_max:.0f} MHz")
    solve_bytes = st1["solve_bytes_per_pass"] * passes + 16.0 * n * rhs
    solve_flops = 2.0 * st1["solve_fma_per_rhs"] * rhs
    avg_ms = solve_ms / max(passes, 1)
    gbs = solve_bytes / passes / (avg_ms * 1e-3) / 1e9 if passes else 0.0
    tfs = solve_flops / passes / (avg_ms * 1e-3) / 1e12 if passes else 0.0
    traffic = (SOLVE_TRAFFIC_RATIO * solve_bytes / max(passes, 1)
               if SOLVE_TRAFFIC_RATIO is not None else None)
    if tfs / alu_peak >= gbs / hbm:
        roof = {"bound": "alu", "achieved": tfs, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": tfs / alu_peak, "traffic": traffic, "peak_source": peak_src,
                "derived_peak": derived_peak}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "traffic": traffic, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    roof.update({"kernel": "k_trsv_fwd + k_trsv_bwd (one supernodal solve pair)",
                 "traffic_source": (SOLVE_TRAFFIC_SOURCE if traffic is not None else
                                    "no capture of the current solve kernels"),
                 "launches": passes, "avg_ms": avg_ms, "bytes_per_launch": solve_bytes / max(passes, 1),
                 "flops_per_launch": solve_flops / max(passes, 1), "hbm_GBps": gbs,
                 "share_of_step_time": solve_ms / ms if ms else None})
    line = {"metric": METRIC, "value": steps_all / (ms_max * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_max / max(steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(a.size, kind, a.stages), "n": n,
                       "nnz_G": int(circ.G.nnz), "devices": int(len(circ.dev)),
                       "loads": int(circ.p), "nnz_L": int(st1["nnz_L"]),
                       "factor_GB": st1["factor_doubles"] * 8 / 1e9,
                       "l2_flush": l2_note,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "create_s": create_s, "factor_and_dc_s": factor_s,
                       "ordering": int(opts.ordering),
                       "solve_ctas_per_sm": tuned,
                       "autotune_ms_per_pass_at_1_2_3": tune_ms},
            "krylov_vectors_per_s": kvec_all / (ms_max * 1e-3),
            "rejects": int(nr),
            "gpu_launches": int(launches),
            "host_syncs_per_step": (st1["host_syncs"] - st0["host_syncs"]) / max(steps, 1),
            "host_polls_per_step": (st1["host_polls"] - st0["host_polls"]) / max(steps, 1),
            "roofline": roof,
            "clocks": clocks,
            "e2e": {"value": k_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": 8 * n}}
    line["node_steps_per_s"] = line["value"] * n
    # accuracy of the timed window ("rel err 1e-6" of the metric): the same window from the
    # same start state in a second context with a Krylov eps 1000x and a tol 10x tighter
    t_stop, x_stop, _ = sim.state()
    sim.close()
    if world == 1 and not a.no_extras:
        ref = ers.Simulator.from_circuit(
            circ, opts=ers.make_opts(eps_krylov=1e-10, h_max=t_end / 100, **ordering_kw(a)))
        ref.set_stream(stream)
        ref.set_state(t_start, x_start, h_start)
        ref.run(t_stop, a.tol / 10)
        _, x_ref, _ = ref.state()
        ref.close()
        line["accuracy"] = {
            "rel_err_vs_tight_run": float(np.max(np.abs(x_stop - x_ref)) / np.max(np.abs(x_ref))),
            "window_s": [t_start, t_stop],
            "reference": "same start state and window, Krylov eps 1e-10 and tol 1e-7"}
    if not a.no_baseline and world == 1:
        try:
            cb = run_oracle_sample(*oracle_args(a))
            cb["node_steps_per_s"] = cb["value"] * cb.pop("n_sample")
            line["cpu_baseline"] = cb
        except Exception as ex:  # the baseline is reported, never required
            line["cpu_baseline"] = {"value": None, "error": str(ex)[-300:]}
    if world == 1 and not a.no_extras and kind == "mesh":
        # the metric's other configurations, each under its own key
        line["config0_mesh2d"] = mesh2d_line(ers, stream)
        line["config2_chain"] = chain_line(ers, stream)
        ba = argparse.Namespace(**vars(a))
        ba.seq_sample = min(a.seq_sample, 2)
        ba.warmup = max(a.warmup, 3)
        line["batched_plain_vs_learned"] = run_batch_workload(ba, emit=False)
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# the triangular solves alone: G_k x = b passes over the factor of a 3D mesh (for timing and
# profiling the solve kernels in isolation; not the metric's workload)
# --------------------------------------------------------------------------------------
def run_solve_workload(a):
    import numpy as np
    import torch
    from paper_1511_04515_gb300 import build
    build.build()
    from paper_1511_04515_gb300 import ers
    circ = workload(a.size, "mesh")
    tc = time.perf_counter()
    sim = ers.Simulator.from_circuit(circ, opts=ers.make_opts(**ordering_kw(a)))
    create_s = time.perf_counter() - tc
    sim.set_state(0.0, np.zeros(circ.n))
    tf = time.perf_counter()
    sim.refactor()
    factor_s = time.perf_counter() - tf
    for _ in range(max(1, a.warmup)):
        sim.solve(np.ones(circ.n))
    chosen, ms = sim.autotune(nrhs=a.nrhs, passes=max(1, a.steps))
    b = np.random.default_rng(0).normal(size=circ.n)
    x = sim.solve(b)
    G = circ.G.tocsr()
    eta = float(np.max(np.abs(G @ x - b)) /
                (abs(G).sum(axis=1).max() * np.max(np.abs(x)) + np.max(np.abs(b))))
    st = sim.stats()
    best = min(ms)
    fma = st["solve_fma_per_rhs"] * a.nrhs
    line = {"workload": f"solve passes, rc3d_{a.size}^3 mesh ({circ.n} nodes), "
                        f"ordering {ers.make_opts(**ordering_kw(a)).ordering}, {a.nrhs} right-hand sides",
            "ms_per_pass_at_1_2_3_ctas_per_sm": ms, "chosen_ctas_per_sm": chosen,
            "fp64_tflops": 2 * fma / (best * 1e-3) / 1e12,
            "hbm_GBps": (st["solve_bytes_per_pass"] + 16.0 * circ.n * a.nrhs) / (best * 1e-3) / 1e9,
            "fma_per_pass": fma, "bytes_per_pass": st["solve_bytes_per_pass"],
            "nnz_L": st["nnz_L"], "nsn": st["nsn"], "factor_doubles": st["factor_doubles"],
            "create_s": create_s, "refactor_s": factor_s, "backward_error": eta,
            "passes_timed": a.steps}
    print(json.dumps(line), flush=True)
    sim.close()


# --------------------------------------------------------------------------------------
# batched workload: Monte Carlo inverter chains, plain GPU method vs batched (+ learned)
# --------------------------------------------------------------------------------------
BATCH_METRIC = ("wall time to t_end at tol 1e-6 of a Monte Carlo batch of inverter chains: "
                "batched + learned controller (plain GPU method and batched plain alongside)")


def batch_workload_name(a):
    return (f"batch{a.batch_n}_invchain: {a.batch_n} inverter chains, stages uniform "
            f"{a.stage_lo}-{a.stage_hi}, {a.tree}-node RC trees per stage, Vt/k/R/C log-normal "
            f"sigma 5%, 0 -> {a.t_end * 1e9:g} ns (first input edge), tol 1e-6")


def _oracle_instance(args):
    """One batch instance to t_end with the oracle (runs in a spawned worker, 1 BLAS thread)."""
    import numpy as np
    from oracle import ers_oracle as O
    circ, t_end, tol = args
    x0 = O.dc_solution(circ, x0=circ.nodeset)
    t0 = time.perf_counter()
    x, t, st = O.er_run(circ, t_end=t_end, tol=tol, x0=x0)
    return st.steps, time.perf_counter() - t0


def batch_oracle_baseline(circs, idx, t_end, tol):
    """The oracle on the sampled instances, in parallel over the host cores (spawn pool)."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    cores = max(1, min(len(idx), os.cpu_count() or 1))
    w0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_instance, [(circs[k], t_end, tol) for k in idx])
    wall = time.perf_counter() - w0
    steps = sum(r[0] for r in res)
    return {"value": steps / wall, "unit": "instance-steps/s", "cores": cores, "kind": "oracle",
            "sample": (f"{len(idx)} instances of the batch to t_end, one per worker process "
                       f"(spawn, 1 BLAS thread each), the oracle's own sparse LU + numpy; "
                       f"{steps} steps in {wall:.1f} s wall; per-instance seconds "
                       f"{[round(r[1], 1) for r in res]}")}


def run_batch_workload(a, emit=True):
    """The batch comparison; prints its JSON line (emit) or returns it (embedded in the main
    line, rank 0 of a one-rank job)."""
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1 and emit:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1511_04515_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1511_04515_gb300 import ers
    from synth import circuits as S

    def family(n, seed0):
        return S.batch_family(n_inst=n, seed0=seed0, stage_lo=a.stage_lo, stage_hi=a.stage_hi,
                              sigma=0.05, t_end=a.t_end, tree_nodes=a.tree)

    t_start = time.perf_counter()

    def progress(msg):
        print(f"[batch {time.perf_counter() - t_start:7.1f}s] {msg}", file=sys.stderr, flush=True)

    # instances are independent: with N ranks each runs its LPT share (no exchange); every rank
    # trains the same network on the same traces (deterministic kernels: identical weights)
    from paper_1511_04515_gb300.partition import instance_cost, lpt_partition
    stream = torch.cuda.Stream()          # the library's stream; events are recorded on it
    # 1. training set: plain-controller traces of other seeds; the network is trained by the
    #    library's own BF16 forward/backward/Adam kernels
    ttr = time.perf_counter()
    trc = family(a.train_n, 2000)
    tr = ers.BatchSimulator(trc)
    tr.set_stream(stream)
    tr.dc(np.concatenate([c.nodeset for c in trc]))
    tr.trace(True)
    tr.run_batch(a.t_end, a.tol)
    X, T = tr.samples()
    tr.close()
    mlp = ers.Mlp(seed=1)
    loss = mlp.train(X, T, epochs=300, batch=256, lr=2e-3, seed=1)
    train_s = time.perf_counter() - ttr
    progress(f"trained on {X.shape[0]} samples, loss {loss:.3g}")
    # 2. held-out batch
    allc = family(a.batch_n, 5000)
    share = lpt_partition([instance_cost(c) for c in allc], world)[rank]
    circs = [allc[i] for i in share]
    tc = time.perf_counter()
    sim = ers.BatchSimulator(circs)
    create_s = time.perf_counter() - tc
    sim.set_stream(stream)
    sim.dc(np.concatenate([c.nodeset for c in circs]))
    tuned, tune_ms = sim.autotune(nrhs=2, passes=3)
    _, x0, _ = sim.state()
    arms = {}
    clk_path = os.path.join(CLOCKS_DIR, f"clocks_batch_rank{rank}.csv")
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    proc, fh = clocks_start(local, clk_path)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    for name, net in (("batched_plain", None), ("batched_learned", mlp)):
        sim.set_controller(net, a.ctrl_parts if net is not None else 0,
                           a.ctrl_margin if net is not None else 0.0)
        sim.set_state(0.0, x0)
        sim.run_batch(a.t_end, a.tol, max_steps=max(a.warmup, 3))     # warm-up rounds
        sim.set_state(0.0, x0)
        st0 = sim.stats()
        c0 = sim.ctrl_stats()
        with torch.cuda.stream(stream):
            flush.fill_(len(arms))         # evict the warm-up rounds' data from L2
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        e0.record(stream)
        ns, nr = sim.run_batch(a.t_end, a.tol)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        st1 = sim.stats()
        c1 = sim.ctrl_stats()
        progress(f"{name}: {wall:.1f} s, {int(ns.sum())} steps, {int(nr.sum())} rejected")
        arms[name] = {"seconds": e0.elapsed_time(e1) * 1e-3, "wall_s": wall,
                      "steps": int(ns.sum()), "rejected": int(nr.sum()),
                      "rounds": st1["steps"] - st0["steps"],
                      "krylov_vectors": c1["krylov_vectors"] - c0["krylov_vectors"],
                      "proposals": c1["proposals"] - c0["proposals"],
                      "proposals_rejected": c1["rejected"] - c0["rejected"],
                      "gpu_launches": st1["kernel_launches"] - st0["kernel_launches"],
                      "x": [sim.state_inst(k)[1] for k in range(len(circs))]}
    clocks = clocks_stop(proc, fh, clk_path)
    # 3. the plain GPU method: each instance in its own context, one after the other (timed on
    #    an evenly spaced sample of instances and scaled to the batch)
    pick = list(range(0, len(circs), max(1, len(circs) // max(1, a.seq_sample))))[:a.seq_sample]
    seq_s, seq_steps = 0.0, 0
    for k in pick:
        one = ers.Simulator.from_circuit(circs[k])
        one.set_stream(stream)
        one.dc(circs[k].nodeset)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        n1, _ = one.run(a.t_end, a.tol)
        torch.cuda.synchronize()
        seq_s += time.perf_counter() - w0
        seq_steps += n1
        one.close()
    seq_est = seq_s / len(pick) * len(circs)
    progress(f"plain sequential sample: {seq_s:.1f} s for {len(pick)} instances")
    # 4. accuracy on two instances against a run of the same instances at a 10x tighter
    #    tolerance (its own error is about a tenth of the compared runs')
    ref_idx = pick[:2]
    ref = ers.BatchSimulator([circs[k] for k in ref_idx])
    ref.set_stream(stream)
    ref.dc(np.concatenate([circs[k].nodeset for k in ref_idx]))
    ref.run_batch(a.t_end, a.tol / 10)
    xref = [ref.state_inst(q)[1] for q in range(len(ref_idx))]
    ref.close()
    progress("tight reference done")
    cpu = None
    if not a.no_baseline and world == 1:
        try:
            ncpu = max(1, min(len(circs), os.cpu_count() or 1))
            cpu_pick = list(range(0, len(circs), max(1, len(circs) // ncpu)))[:ncpu]
            cpu = batch_oracle_baseline(circs, cpu_pick, a.t_end, a.tol)
            progress(f"oracle baseline: {cpu['value']:.1f} instance-steps/s on {cpu['cores']} cores")
        except Exception as ex:  # the baseline is reported, never required
            cpu = {"value": None, "error": str(ex)[-300:]}
    err = {}
    for name, arm in arms.items():
        err[name] = max(float(np.max(np.abs(arm["x"][k] - xr))) for k, xr in zip(ref_idx, xref))
        del arm["x"]
    sim.close()
    mlp.close()
    if world > 1:   # the job ends when the slowest rank does
        t = torch.tensor([arms["batched_plain"]["seconds"], arms["batched_learned"]["seconds"],
                          seq_est / world], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        arms["batched_plain"]["seconds"], arms["batched_learned"]["seconds"] = float(t[0]), float(t[1])
        seq_est = float(t[2]) * world
    if rank != 0:
        return
    learned = arms["batched_learned"]
    plain = arms["batched_plain"]
    nodes = int(sum(c.n for c in circs))
    line = {"metric": BATCH_METRIC, "value": learned["seconds"], "unit": "s",
            "n_gpus": world, "steps": 1, "warmup": max(a.warmup, 3),
            "ms_per_step": learned["seconds"] * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": batch_workload_name(a), "instances": len(circs),
                       "nodes": nodes, "train_instances": a.train_n,
                       "train_samples": int(X.shape[0]), "train_loss": loss,
                       "train_s": train_s, "create_s": create_s,
                       "controller": {"parts": a.ctrl_parts, "margin_log2": a.ctrl_margin},
                       "solve_ctas_per_sm": tuned, "autotune_ms_per_pass_at_1_2_3": tune_ms,
                       "parallelism": ("instances split over ranks (LPT on node count)"
                                       if world > 1 else "single GPU"),
                       "l2_flush": (f"L2 flushed before each arm's timed run ({FLUSH_BYTES >> 20} "
                                    f"MB write, finished before the timer starts); each arm is "
                                    f"one run to t_end whose rounds follow one another")},
            "arms": {**arms,
                     "plain_sequential": {"seconds_est": seq_est, "sampled_instances": len(pick),
                                          "sample_seconds": seq_s, "sample_steps": seq_steps,
                                          "note": "each instance in its own context, run one "
                                                  "after another; mean over the sample x batch"}},
            "speedup": {"learned_vs_batched_plain": plain["seconds"] / learned["seconds"],
                        "learned_vs_plain_sequential": seq_est / learned["seconds"],
                        "batched_plain_vs_plain_sequential": seq_est / plain["seconds"]},
            "max_abs_err_vs_tight_run": {**err, "instances": ref_idx, "tight_tol": a.tol / 10},
            "instance_steps_per_s": learned["steps"] / learned["seconds"],
            "cpu_baseline": cpu,
            "krylov_vectors_per_s": learned["krylov_vectors"] / learned["seconds"],
            "gpu_launches": learned["gpu_launches"],
            "clocks": clocks}
    if not emit:
        return line
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.oracle_sample:
        print(json.dumps(oracle_sample(a.steps, a.size, a.workload, a.stages)))
        return
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch":
        run_batch_workload(a)
    elif a.workload == "solve":
        run_solve_workload(a)
    elif a.workload == "mesh2d":
        import torch
        from paper_1511_04515_gb300 import build
        build.build()
        from paper_1511_04515_gb300 import ers
        print(json.dumps(mesh2d_line(ers, torch.cuda.Stream(), steps=max(1, a.steps))), flush=True)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
