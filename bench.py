#!/usr/bin/env python
"""Benchmark of the coined-walk spatial search hot path on one B300.

Workload (default): 1024 x 1024 torus (2^20 vertices, 4 * 2^20 arcs), Grover
coin with -I on one seeded marked vertex, flip-flop shift, uniform initial
state over all arcs, 3000 walk steps with the marked-vertex probability
recorded after every step, per-vertex probabilities (double sums) at the end.
One bench "step" is that whole run.  The metric is walk-step arc updates per
second: num_arcs * 3000 / (time of one run).  The headline runs in complex128;
the complex64 mixed form (fp32 amplitudes, fp64 probability sums) is reported
beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs its own replica of the workload (the
walks are independent; there is no collective on the data path) and `value`
is the total arc updates of all ranks over the slowest rank's time.
`--impl reference` times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload.
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

L = 1024
WALK_STEPS = 3000
MARK_SEED = 2
METRIC = "walk-step arc updates/s"
UNIT = "arc-updates/s"

# DRAM bytes per launch of the coin+shift kernel (ncu dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by the SHA-1 of the kernel source they were
# measured on; a changed kernel reports null until it is measured again.
TRAFFIC = {
    # the 1024x1024 torus step (k_coined_em<R,4,grover,torus>, index-free, a
    # block row per torus row, complex128 sums by integer operations and
    # streaming loads and stores), one launch, cold L2
    ("c128", "353bcfad430a774d3180ad7a5bd12c59d60481d2"): 67130624 + 16286976,
    ("c64", "353bcfad430a774d3180ad7a5bd12c59d60481d2"): 33566976 + 327168,
}


def workload():
    n, eu, ev = synth.torus(L)
    row_ptr, col = synth.adjacency_csr(n, eu, ev)
    m = synth.seeded_vertex(MARK_SEED, n)
    return n, eu, ev, row_ptr, col, m


def kernel_source_hash():
    """SHA-1 of the sources of the coin+shift kernels (the ncu traffic below is
    valid only for the kernels it was taken on)."""
    h = hashlib.sha1()
    for f in ("coined.cu", "family.cuh", "internal.h", "sum4.cuh", "fpconv.cuh"):
        with open(os.path.join(ROOT, "paper_2406_08186_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def coin_shift_bytes(arcs, esz, index_free):
    """Algorithmic bytes of one edge-major coin+shift launch: read and write the
    state, plus the reversal table unless the positions come from the labels."""
    return arcs * (2 * esz + (0 if index_free else 4))


# FP64 operations of one Grover step of a degree-4 vertex, per component: four
# FMAs (2/d) S - psi_j (the sum S of the four amplitudes is formed with integer
# operations, rounded once)
FP64_OPS_PER_VERTEX_D4 = 2 * 4


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def measured_tensor_peak():
    """Dense bf16 tensor-core peak (TFLOP/s) measured on the B300s (burst:
    the expm is timed on its own); fp16 runs at the same rate."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["bf16_tflops"]), "MEASURED_PEAKS.json bf16_tflops (measured, burst)"
    except Exception:
        return 1800.0, "fallback 1.8 PFLOP/s bf16 burst"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for name, flag in zip(names, f[2:6]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_max(x, dist=None, device="cuda"):
    """The largest x over all ranks (the slowest rank's time); x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, world, t_max):
    """Whole-job throughput of `world` independent replicas: every rank's units
    over the slowest rank's time."""
    return units_per_rank * world / t_max


def cpu_baseline(n, eu, ev, m, budget_s=12.0):
    """The FP64 oracle, untuned, on the host cores: walk steps of the same search.
    Also returns the oracle's state and per-vertex probabilities after those
    steps, for the error of the GPU results over the same steps."""
    import oracle
    cores = oracle.threads()
    ar = oracle.Arcs(n, eu, ev)
    psi = synth.uniform_state(ar.num_arcs)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        psi = oracle.coined_evolve(ar, psi, 5, marked=[m])
        done += 5
    el = time.perf_counter() - t0
    return ({"value": ar.num_arcs * done / el, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": "%d walk steps of the 1024x1024 torus search (complex128 oracle, OpenMP)" % done},
            done, psi, oracle.prob_coined(ar, psi))


def l2_copy_per_launch(torch):
    """Read + write GB/s of a copy between two 32 MB device buffers, one launch per
    copy (the L2-resident ping-pong of the complex64 step), as a reference rate."""
    a = torch.ones(8 << 20, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    for _ in range(20):
        b.copy_(a)
        a.copy_(b)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(500):
        b.copy_(a)
        a.copy_(b)
    ev[1].record()
    torch.cuda.synchronize()
    per_copy = ev[0].elapsed_time(ev[1]) * 1e-3 / 1000
    return 2.0 * a.numel() * 4 / per_copy / 1e9


def headline_config(n, arcs, m, world):
    """The headline workload's `config`, the same on both arms (the reference
    arm times a bounded sample of it and says so in its cpu_baseline)."""
    return {"workload": "torus1024_search", "n": n, "arcs": arcs, "walk_steps": WALK_STEPS,
            "coin": "grover", "marked": m, "state": "complex128", "record": "p_m(t) every step",
            "l2": "256 MiB written between timed steps; working set 134 MB (two 64 MiB state buffers) > L2",
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    n, eu, ev, _, _, m = workload()
    cores = oracle.threads()
    ar = oracle.Arcs(n, eu, ev)
    psi = synth.uniform_state(ar.num_arcs)
    per = 4   # walk steps per bench step (bounded sample of the 3000-step run)
    for _ in range(args.warmup):
        psi = oracle.coined_evolve(ar, psi, per, marked=[m])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        psi = oracle.coined_evolve(ar, psi, per, marked=[m])
    el = time.perf_counter() - t0
    value = ar.num_arcs * per * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": headline_config(n, ar.num_arcs, m, int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d walk steps per bench step of the 1024x1024 torus search (complex128 "
                                       "oracle on the host cores, uniform start, the same mark)" % per},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_2406_08186_b300 as hw

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    n, eu, ev, row_ptr, col, m = workload()
    G = hw.hw_graph_csr(n, row_ptr, col)
    arcs = G.num_arcs
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def make(dt):
        cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
        psi0 = torch.full((arcs,), 1.0 / math.sqrt(arcs), dtype=cdt, device="cuda")
        return dict(dt=dt, psi0=psi0, out=torch.empty_like(psi0),
                    rec=torch.empty(WALK_STEPS, dtype=torch.float64, device="cuda"),
                    prob=torch.empty(n, dtype=torch.float64, device="cuda"),
                    norm=torch.empty(1, dtype=torch.float64, device="cuda"))

    # steps, layout in and out, final record, probability, norm (2)
    launches_per_run = WALK_STEPS + 2 + 1 + 1 + 2

    def run(b, ev_evolve=None):
        if ev_evolve:
            ev_evolve[0].record(stream)
        hw.hw_coined_evolve(G, hw.HW_COIN_GROVER, [m], b["dt"], 1, WALK_STEPS, b["psi0"], b["out"],
                            b["rec"], stream=stream)
        if ev_evolve:
            ev_evolve[1].record(stream)
        hw.hw_probability(G, n, b["dt"], 1, b["out"], b["prob"], b["norm"], stream=stream)

    def timed(b):
        for _ in range(args.warmup):
            run(b)
        torch.cuda.synchronize()
        barrier()
        total = evolve = 0.0
        pairs = []
        for _ in range(args.steps):
            flush.zero_()       # L2 flush outside the timed events
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(stream)
            run(b, (e[1], e[2]))
            e[3].record(stream)
            pairs.append(e)
        torch.cuda.synchronize()
        barrier()
        for e in pairs:
            total += e[0].elapsed_time(e[3]) / 1e3
            evolve += e[1].elapsed_time(e[2]) / 1e3
        return total, evolve

    peak, peak_src = measured_peaks()
    fp64_peak = hw.hw_measure_fp64()
    l2_peak = hw.hw_measure_l2()
    l2_launch = l2_copy_per_launch(torch)
    kind, _ = hw.hw_graph_structure(G)
    index_free = kind == hw.HW_GRAPH_TORUS   # the default addressing on a recognised torus
    b128 = make(hw.HW_C128)
    with Clocks(local) as clk:
        t128, ev128 = timed(b128)
    clocks = clk.summary()
    b64 = make(hw.HW_C64)
    t64, ev64 = timed(b64)

    # correctness guard on the measured buffers: unit norm, record consistent
    norm128 = float(b128["norm"].item())
    norm64 = float(b64["norm"].item())
    if abs(norm128 - 1) > 1e-10 or abs(norm64 - 1) > 1e-3:
        raise RuntimeError("norm check failed: %r %r" % (norm128, norm64))

    # end to end through the C ABI from pinned host buffers
    host_psi = b128["psi0"].cpu().pin_memory()
    host_prob = torch.empty(n, dtype=torch.float64).pin_memory()
    host_rec = torch.empty(WALK_STEPS, dtype=torch.float64).pin_memory()

    def run_e2e():
        b128["psi0"].copy_(host_psi, non_blocking=True)
        run(b128)
        host_prob.copy_(b128["prob"], non_blocking=True)
        host_rec.copy_(b128["rec"], non_blocking=True)

    for _ in range(max(1, args.warmup)):
        run_e2e()
    torch.cuda.synchronize()
    barrier()
    t_e2e = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_e2e()
        e1.record(stream)
        e1.synchronize()
        t_e2e += e0.elapsed_time(e1) / 1e3
    barrier()

    t128, t64, t_e2e = rank_max(t128, dist), rank_max(t64, dist), rank_max(t_e2e, dist)
    work = arcs * WALK_STEPS * args.steps * world
    value = replica_value(arcs * WALK_STEPS * args.steps, world, t128)
    per_launch128 = ev128 / (args.steps * WALK_STEPS)
    per_launch64 = ev64 / (args.steps * WALK_STEPS)
    bytes128 = coin_shift_bytes(arcs, 16, index_free)
    bytes64 = coin_shift_bytes(arcs, 8, index_free)
    ops128 = FP64_OPS_PER_VERTEX_D4 * n
    src_hash = kernel_source_hash()
    ach128 = bytes128 / per_launch128 / 1e9
    ach64 = bytes64 / per_launch64 / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t128 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(n, arcs, m, world),
        "roofline": {"bound": "hbm",
                     "kernel": "k_coined_em<double,4,grover,%s>" % ("torus" if index_free else "table"),
                     "achieved": ach128, "peak": peak, "unit": "GB/s", "frac": ach128 / peak,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % peak_src,
                     "bytes_per_launch": bytes128, "launch_us": per_launch128 * 1e6,
                     "traffic": TRAFFIC.get(("c128", src_hash)),
                     "fp64": {"achieved": ops128 / per_launch128, "peak": fp64_peak, "unit": "FP64 op/s",
                              "frac": ops128 / per_launch128 / fp64_peak, "ops_per_launch": ops128,
                              "peak_source": "hw_measure_fp64 (register-blocked GEMM loop on this GPU)"}},
        "c64_mixed": {"value": work / t64, "unit": UNIT, "ms_per_step": 1e3 * t64 / args.steps,
                      "dtype": "f32 (fp64 probability sums)",
                      "roofline": {"bound": "l2", "achieved": ach64, "peak": l2_peak, "unit": "GB/s",
                                   "frac": ach64 / l2_peak, "bytes_per_launch": bytes64,
                                   "peak_source": "hw_measure_l2 (32 MB copy, L2-resident, read + write)",
                                   "launch_us": per_launch64 * 1e6,
                                   "traffic": TRAFFIC.get(("c64", src_hash)),
                                   "copy_per_launch": {"gbs": l2_launch, "frac": ach64 / l2_launch,
                                                       "how": "one copy kernel per launch between two 32 MB "
                                                              "buffers (the step's pattern), 500 round trips"},
                                   "note": "the two 32 MB state buffers stay in the 126 MB L2"}},
        "e2e": {"value": work / t_e2e, "unit": UNIT, "h2d_bytes_per_step": arcs * 16,
                "d2h_bytes_per_step": n * 8 + WALK_STEPS * 8},
        "gpu_launches": launches_per_run * args.steps,
        "clocks": clocks,
        "norm_after": {"c128": norm128, "c64": norm64},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, done, psi_ref, p_ref = cpu_baseline(n, eu, ev, m)
        line["cpu_baseline"] = cb
        # the error of both GPU forms against the oracle over the same steps
        errs = {"walk_steps": done}
        for b, tag in ((b128, "c128"), (b64, "c64")):
            hw.hw_coined_evolve(G, hw.HW_COIN_GROVER, [m], b["dt"], 1, done, b["psi0"], b["out"], stream=stream)
            hw.hw_probability(G, n, b["dt"], 1, b["out"], b["prob"], stream=stream)
            torch.cuda.synchronize()
            got = b["out"].cpu().numpy().astype(np.complex128)
            pg = b["prob"].cpu().numpy()
            errs[tag] = {"max_abs_psi": float(np.max(np.abs(got - psi_ref))),
                         "p_L1": float(np.sum(np.abs(pg - p_ref))), "p_m_abs": float(abs(pg[m] - p_ref[m]))}
        line["error_vs_oracle"] = errs
    G.free()
    if world == 1 and not args.no_configs:
        # the other configurations, each with its own timing, clocks, roofline
        # and error figures
        cpu = not args.no_cpu_baseline
        line["cfg1_torus64"] = sub_torus64(hw, reps=max(args.steps, 10), warmup=args.warmup, with_cpu=cpu)
        line["hypercube20_c128"] = sub_hypercube20(hw, reps=5)
        line["cfg3_hypercube12"] = sub_ctqw_q12(hw, reps=3, warmup=1, with_cpu=cpu)
        line["cfg4_er_batched"] = sub_er_batched(hw, reps=3, warmup=1, with_cpu=cpu)
        line["cfg5_serving"] = sub_serving(hw, args.serving_jobs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def _oracle_cores():
    import oracle
    return oracle.threads()


def sub_torus64(hw, reps, warmup, with_cpu):
    """Configuration 1: 64 x 64 torus, Grover, no mark, start on the 4 arcs of
    (32, 32), 100 steps, complex128, per-vertex probabilities.  Time per run
    (evolve + probabilities) from CUDA events; the run is launch-latency bound
    (0.6 MB per walk step)."""
    import torch
    n, eu, ev = synth.torus(64)
    row_ptr, col = synth.adjacency_csr(n, eu, ev)
    G = hw.hw_graph_csr(n, row_ptr, col)
    psi0_h = synth.state_on_vertex_arcs(synth.arc_offsets(n, eu, ev), 32 * 64 + 32)
    psi0 = torch.from_numpy(psi0_h).cuda()
    out = torch.empty_like(psi0)
    prob = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(3, warmup)):
        hw.hw_coined_evolve(G, 0, [], hw.HW_C128, 1, 100, psi0, out)
        hw.hw_probability(G, n, hw.HW_C128, 1, out, prob)
    torch.cuda.synchronize()
    # enough runs for half a second of timed work, so that the clock sampler
    # (every 200 ms) sees the timed region
    e = _events(2)
    e[0].record(stream)
    hw.hw_coined_evolve(G, 0, [], hw.HW_C128, 1, 100, psi0, out)
    e[1].record(stream)
    torch.cuda.synchronize()
    reps = max(reps, int(0.5 / max(e[0].elapsed_time(e[1]) / 1e3, 1e-6)))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    with Clocks(torch.cuda.current_device()) as clk:
        pairs = []
        for _ in range(reps):
            flush.zero_()       # L2 flushed between runs, outside the timed events
            e = _events(2)
            e[0].record(stream)
            hw.hw_coined_evolve(G, 0, [], hw.HW_C128, 1, 100, psi0, out)
            hw.hw_probability(G, n, hw.HW_C128, 1, out, prob)
            e[1].record(stream)
            pairs.append(e)
        torch.cuda.synchronize()
    t = sum(e[0].elapsed_time(e[1]) for e in pairs) / 1e3 / reps
    del flush
    arcs = G.num_arcs
    # the one-launch walk runs on one 16-CTA cluster: its FP64 ceiling is 16/148
    # of the GPU's measured FP64 rate (8 FMAs per vertex and step)
    fp64 = hw.hw_measure_fp64()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fmas = 8.0 * n * 100
    res = {"workload": "torus64_center", "metric": METRIC, "unit": UNIT, "value": arcs * 100 / t,
           "us_per_run": t * 1e6, "us_per_walk_step": t / 100 * 1e6, "reps": reps, "dtype": "f64",
           "l2": "256 MiB written before every timed run (outside the events)",
           "roofline": {"bound": "latency", "bytes_per_walk_step": arcs * 32,
                        "fp64_of_16_sms": {"achieved": fmas / t, "peak": fp64 * 16 / sms, "unit": "FMA/s",
                                           "frac": fmas / t / (fp64 * 16 / sms), "fma_per_run": fmas},
                        "note": "the whole walk in one launch (one 16-CTA thread-block cluster holds the 256 KiB "
                                "state in shared memory; outputs owned by other CTAs go by st.async, counted on "
                                "the owner's mbarrier, and each CTA waits only for its own incoming bytes), then "
                                "one probability launch; per step the integer four-term sums and the FP64 FMAs "
                                "of 4096 vertices on the cluster's 16 SMs and the cross-CTA latency set the time"},
           "clocks": clk.summary()}
    if with_cpu:
        import oracle
        ar = oracle.Arcs(n, eu, ev)
        t0 = time.perf_counter()
        ref = oracle.coined_evolve(ar, psi0_h, 100)
        el = time.perf_counter() - t0
        p_ref = oracle.prob_coined(ar, ref)
        res["cpu_baseline"] = {"value": arcs * 100 / el, "unit": UNIT, "cores": _oracle_cores(), "kind": "oracle",
                               "sample": "the whole 100-step run"}
        # the same run on one host core
        all_cores = oracle.threads()
        oracle.threads(1)
        try:
            t0 = time.perf_counter()
            oracle.coined_evolve(ar, psi0_h, 100)
            el1 = time.perf_counter() - t0
        finally:
            oracle.threads(all_cores)
        res["cpu_baseline_one_core"] = {"value": arcs * 100 / el1, "unit": UNIT, "cores": 1, "kind": "oracle",
                                        "sample": "the whole 100-step run"}
        res["error_vs_oracle"] = {"c128_max_abs_psi": float(np.max(np.abs(out.cpu().numpy() - ref))),
                                  "c128_max_abs_p": float(np.max(np.abs(prob.cpu().numpy() - p_ref)))}
    G.free()
    return res


def sparse_power_figures(n, deg_graph, m_deg, esz, n_marked):
    """Algorithmic bytes and FP64 operations of the sparse Taylor powers of one
    expm (m_deg powers Q_k = Y Q_{k-1} / k of an n x n dense Q, Y with deg_graph
    neighbours per row): per power Q_{k-1} read once (its gathered rows are L2
    hits), Q_k written, U's real or imaginary plane read and written in double.
    complex128 FP64 operations per element: the neighbour groups of four are
    summed by integer operations, their ceil(d/4) - 1 sums added in double, one
    multiply, one add into U (plus one FMA on marked rows)."""
    nn = n * n
    bytes_power = 2 * nn * esz + 2 * nn * 8
    fp64_power = nn * ((deg_graph + 3) // 4 - 1 + 2) + n_marked * n
    return m_deg * bytes_power, m_deg * fp64_power


def sub_ctqw_q12(hw, reps, warmup, with_cpu):
    """Configuration 3: CTQW search on Q_12, gamma = 1/12, one seeded mark,
    U = exp(-iH 0.1) dense (Taylor, scaling and squaring), 2000 applications,
    complex128 and complex64.  Both forms of the Taylor powers are timed: sparse
    x dense products with the graph (the default for complex128) and dense
    GEMMs (FP64 for complex128; tcgen05 tensor cores for complex64, its
    default).  Each result's
    error against the complex128 GPU result and, with the CPU leg, against the
    oracle."""
    import torch
    g = synth.hypercube(12)
    n = 4096
    m = synth.seeded_vertex(3, n)
    row_ptr, col = synth.adjacency_csr(*g)
    G = hw.hw_graph_csr(n, row_ptr, col)
    stream = torch.cuda.current_stream()
    peak, src = measured_peaks()
    tc_peak, tc_src = measured_tensor_peak()
    fp64 = hw.hw_measure_fp64()
    l2_peak = hw.hw_measure_l2()
    res = {"workload": "hypercube12_ctqw", "n": n, "marked": m, "gamma": 1 / 12, "dt": 0.1,
           "applications": 2000, "reps": reps,
           "l2": "256 MiB written before every timed expm and evolve call (outside the events); inside an "
                 "evolve call the complex64 upper triangle of U, packed once per call into 68 MB of "
                 "contiguous 64 x 64 blocks, stays in L2 from one application to the next"}
    deg, sq = hw.hw_ctqw_plan(G, 1 / 12, [m], 0.1)
    kept = {}

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def time_expm(dt, U, opts, count):
        pairs = []
        for _ in range(count):
            flush.zero_()       # L2 flushed between expm calls, outside the timed events
            e = _events(2)
            e[0].record(stream)
            hw.hw_ctqw_expm(G, 1 / 12, [m], 0.1, dt, U, opts=opts)
            e[1].record(stream)
            pairs.append(e)
        torch.cuda.synchronize()
        return sum(e[0].elapsed_time(e[1]) for e in pairs) / 1e3 / count

    with Clocks(torch.cuda.current_device()) as clk:
        for dt, name in ((hw.HW_C128, "c128"), (hw.HW_C64, "c64")):
            cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
            esz = 8 if dt == hw.HW_C128 else 4
            U = torch.empty((n, n), dtype=cdt, device="cuda")
            Ud = torch.empty_like(U)
            Us = torch.empty_like(U)
            x = torch.full((n,), 1 / 64, dtype=cdt, device="cuda")
            y = torch.empty_like(x)
            rec = torch.empty(2000, dtype=torch.float64, device="cuda")
            prob = torch.empty(n, dtype=torch.float64, device="cuda")
            sym = {"u_symmetric": 1}   # U = e^{-iH dt} is complex symmetric
            dense, sparse = {"taylor_powers": 1}, {"taylor_powers": 2}
            for _ in range(max(1, warmup)):
                hw.hw_ctqw_expm(G, 1 / 12, [m], 0.1, dt, U)
                hw.hw_ctqw_expm(G, 1 / 12, [m], 0.1, dt, Ud, opts=dense)
                hw.hw_ctqw_expm(G, 1 / 12, [m], 0.1, dt, Us, opts=sparse)
                hw.hw_ctqw_evolve(U, n, dt, 1, 2000, x, y, [m], rec, opts=sym)
            torch.cuda.synchronize()
            t_exp = time_expm(dt, U, None, max(reps, 10))
            t_dense = time_expm(dt, Ud, dense, reps if dt == hw.HW_C128 else max(reps, 10))
            t_sparse = time_expm(dt, Us, sparse, max(reps, 10))
            pairs = []
            for _ in range(reps):
                flush.zero_()
                e = _events(2)
                e[0].record(stream)
                hw.hw_ctqw_evolve(U, n, dt, 1, 2000, x, y, [m], rec, opts=sym)
                e[1].record(stream)
                pairs.append(e)
            torch.cuda.synchronize()
            t_ev = sum(e[0].elapsed_time(e[1]) for e in pairs) / 1e3 / reps
            hw.hw_probability(None, n, dt, 1, y, prob)
            torch.cuda.synchronize()
            kept[name] = (U, Ud, Us, y, rec, prob)
            sp_bytes, sp_ops = sparse_power_figures(n, 12, deg, esz, 1)
            r = {"expm_ms": t_exp * 1e3, "evolve_ms": t_ev * 1e3, "apply_us": t_ev / 2000 * 1e6,
                 "taylor_degree": deg, "squarings": sq, "p_m_max": float(rec.max().item()),
                 "expm_default_form": "sparse x dense" if dt == hw.HW_C128 else "tensor-core GEMMs",
                 "expm_sparse": {"ms": t_sparse * 1e3,
                                 "roofline": {"bound": "hbm", "achieved": sp_bytes / t_sparse / 1e9, "peak": peak,
                                              "unit": "GB/s", "frac": sp_bytes / t_sparse / 1e9 / peak,
                                              "bytes_per_expm": sp_bytes, "peak_source": src,
                                              "note": "whole expm (identity init, powers, pack) over the powers' "
                                                      "compulsory bytes; the neighbour gathers are L2 reads"}},
                 "expm_dense": {"ms": t_dense * 1e3}}
            if dt == hw.HW_C128:
                r["expm_sparse"]["roofline"]["fp64"] = {"achieved": sp_ops / t_sparse, "peak": fp64, "unit": "op/s",
                                                        "frac": sp_ops / t_sparse / fp64, "ops_per_expm": sp_ops}
                # dense form: FP64 GEMM tiles of 64 x 64 on and above the diagonal
                # (the powers of the real symmetric Y are symmetric)
                nb = (n + 63) // 64
                fmas = (deg - 1) * (nb * (nb + 1) // 2) * 64 * 64 * n
                r["expm_dense"]["roofline"] = {"bound": "fp64", "achieved": fmas / t_dense, "peak": fp64,
                                               "unit": "FMA/s", "frac": fmas / t_dense / fp64, "fma_per_expm": fmas,
                                               "peak_source": "hw_measure_fp64 (register-blocked GEMM loop on this GPU)"}
                # application: three real FMAs per element (the 3M form)
                afma = 3.0 * n * n
                r["apply_roofline"] = {"bound": "fp64", "achieved": afma / (t_ev / 2000), "peak": fp64,
                                       "unit": "FMA/s", "frac": afma / (t_ev / 2000) / fp64, "fma_per_apply": afma}
            else:
                # dense form on the tensor cores: (m - 1) powers, each over the
                # 256 x 256 tiles of CTA pairs on and above the diagonal (136 at
                # n = 4096), two fp16 products per tile
                cl = (n + 255) // 256          # pair tiles per side
                mma = (deg - 1) * (cl * (cl + 1)) * 128 * 256 * n * 2 * 2.0
                r["expm_dense"]["roofline"] = {"bound": "tensor", "achieved": mma / t_dense / 1e12, "peak": tc_peak,
                                               "unit": "TFLOP/s", "frac": mma / t_dense / 1e12 / tc_peak,
                                               "flop_per_expm_issued": mma,
                                               "dense_equivalent_tflops": (deg - 1) * 2.0 * n ** 3 / t_dense / 1e12,
                                               "peak_source": tc_src,
                                               "note": "whole expm (slicing, Taylor sums, finish) over the MMA work"}
                abytes = n * n // 2 * 8 + n * 8
                r["apply_roofline"] = {"bound": "l2", "achieved": abytes / (t_ev / 2000) / 1e9, "unit": "GB/s",
                                       "peak": l2_peak, "frac": abytes / (t_ev / 2000) / 1e9 / l2_peak,
                                       "peak_source": "hw_measure_l2 (32 MB copy, L2-resident, read + write)",
                                       "bytes_per_apply": abytes,
                                       "note": "packed upper triangle of U (68 MB) streamed per application, L2-resident"}
            res[name] = r
    res["clocks"] = clk.summary()
    U128, U128d, U128s, y128, rec128, p128 = kept["c128"]
    U64, U64d, U64s, y64, rec64, p64 = kept["c64"]
    res["c64_vs_c128"] = {"U_max_abs": float((U64.to(torch.complex128) - U128).abs().max().item()),
                          "U_sparse_max_abs": float((U64s.to(torch.complex128) - U128).abs().max().item()),
                          "p_L1": float((p64 - p128).abs().sum().item()),
                          "p_m_record_max_abs": float((rec64 - rec128).abs().max().item())}
    res["c128_sparse_vs_dense_U_max_abs"] = float((U128s - U128d).abs().max().item())
    res["gamma_critical"] = critical_gamma_variant(hw, G, n, m, stream)
    if with_cpu:
        import oracle
        ar = oracle.Arcs(*g)
        t0 = time.perf_counter()
        ref, rr = oracle.ctqw_evolve(ar, 1 / 12, np.full(n, 1 / 64, dtype=np.complex128), 0.1, 2000,
                                     marked=[m], record=True)
        el = time.perf_counter() - t0
        pr = np.abs(ref) ** 2
        res["cpu_baseline"] = {"value": 2000 / el, "unit": "applications/s", "cores": _oracle_cores(),
                               "kind": "oracle", "sample": "the whole 2000-application run (sparse Taylor action)"}
        res["error_vs_oracle"] = {
            "c128_max_abs_psi": float(np.max(np.abs(y128.cpu().numpy() - ref))),
            "c128_record_max_abs": float(np.max(np.abs(rec128.cpu().numpy() - rr))),
            "c64_p_L1": float(np.sum(np.abs(p64.cpu().numpy() - pr))),
            "c64_record_max_abs": float(np.max(np.abs(rec64.cpu().numpy() - rr)))}
    G.free()
    return res


def er_graph():
    n0 = 1 << 20
    n, eu, ev = synth.erdos_renyi(n0, 8.0 / (n0 - 1), seed=5)
    return n, eu, ev


def critical_gamma_variant(hw, G, n, m, stream):
    """Configuration 3 at the critical gamma_c = sum_r C(k, r)/r / (2N) of the
    hypercube Q_k (1/12 is off-critical at k = 12): one expm and 2000
    applications per precision, the marked-probability curve's maximum and
    its time, and the curve's error against the exact Hamming-weight reduction
    (one mark, uniform start: a (k+1)-dimensional H, diagonalised here)."""
    import torch
    k = int(round(math.log2(n)))
    gamma = sum(math.comb(k, r) / r for r in range(1, k + 1)) / (2 * n)
    A = np.zeros((k + 1, k + 1))
    for r in range(k):
        A[r, r + 1] = A[r + 1, r] = math.sqrt((r + 1) * (k - r))
    H = -gamma * A
    H[0, 0] -= 1.0
    w, V = np.linalg.eigh(H)
    x0 = np.array([math.sqrt(math.comb(k, r) / n) for r in range(k + 1)])
    times = 0.1 * np.arange(1, 2001)
    ref = np.abs((V[0, :][None, :] * np.exp(-1j * np.outer(times, w))) @ (V.T @ x0)) ** 2
    out = {"gamma": gamma, "exact_p_m_max": float(ref.max()), "exact_t_at_max": float(times[int(np.argmax(ref))])}
    for dt, name in ((hw.HW_C128, "c128"), (hw.HW_C64, "c64")):
        cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
        U = torch.empty((n, n), dtype=cdt, device="cuda")
        x = torch.full((n,), 1 / math.sqrt(n), dtype=cdt, device="cuda")
        y = torch.empty_like(x)
        rec = torch.empty(2000, dtype=torch.float64, device="cuda")
        e = _events(4)
        e[0].record(stream)
        hw.hw_ctqw_expm(G, gamma, [m], 0.1, dt, U)
        e[1].record(stream)
        e[2].record(stream)
        hw.hw_ctqw_evolve(U, n, dt, 1, 2000, x, y, [m], rec, opts={"u_symmetric": 1})
        e[3].record(stream)
        torch.cuda.synchronize()
        r = rec.cpu().numpy()
        out[name] = {"expm_ms": e[0].elapsed_time(e[1]), "apply_us": e[2].elapsed_time(e[3]) * 1e3 / 2000,
                     "p_m_max": float(r.max()), "t_at_max": float(times[int(np.argmax(r))]),
                     "record_max_abs_vs_exact": float(np.max(np.abs(r - ref)))}
        del U
    return out


def sub_hypercube20(hw, reps):
    """The complex128 Grover coin of degree 20 (the 2^20-vertex hypercube,
    index-free, uniform start, one seeded mark): the two-pass kernel that the
    serving mix's largest coined jobs run.  Time per walk step = (evolve of 120
    steps - evolve of 20 steps) / 100, each call after an L2 flush, median of
    `reps`; bytes per step = the state read and written once."""
    import torch
    k = 20
    n, eu, ev = synth.hypercube(k)
    row_ptr, col = synth.adjacency_csr(n, eu, ev)
    G = hw.hw_graph_csr(n, row_ptr, col)
    arcs = G.num_arcs
    x = torch.full((arcs,), 1 / math.sqrt(arcs), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    m = synth.seeded_vertex(3, n)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    hw.hw_coined_evolve(G, 0, [m], hw.HW_C128, 1, 20, x, y)
    torch.cuda.synchronize()
    times = {}
    with Clocks(torch.cuda.current_device()) as clk:
        for steps in (20, 120):
            ts = []
            for _ in range(reps):
                flush.zero_()
                e = _events(2)
                e[0].record(stream)
                hw.hw_coined_evolve(G, 0, [m], hw.HW_C128, 1, steps, x, y)
                e[1].record(stream)
                torch.cuda.synchronize()
                ts.append(e[0].elapsed_time(e[1]) / 1e3)
            times[steps] = sorted(ts)[len(ts) // 2]
    per = (times[120] - times[20]) / 100
    peak, src = measured_peaks()
    byts = 2 * 16 * arcs
    norm = float((y.abs() ** 2).sum().item())
    del flush
    G.free()
    return {"workload": "hypercube20_c128_coined", "n": n, "arcs": arcs, "marked": m, "dtype": "f64",
            "us_per_walk_step": per * 1e6, "value": arcs / per, "unit": "arc-updates/s",
            "l2": "256 MiB written before every timed call; the 671 MB step exceeds L2",
            "roofline": {"bound": "hbm", "kernel": "k_coined_em_rt<double,cube>", "achieved": byts / per / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": byts / per / 1e9 / peak, "bytes_per_step": byts,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % src},
            "norm_after": norm, "clocks": clk.summary()}


def sub_er_batched(hw, reps, warmup, with_cpu):
    """Configuration 4: batched coined walks on the Erdos-Renyi graph (n = 2^20,
    mean degree 8, isolated vertices dropped), 64 complex64 Gaussian states
    drawn on the device by the seeded recipe (the inputs the parity test
    checks), Grover coin, 500 steps, one SpMM-shaped launch per step."""
    import torch
    n, eu, ev = er_graph()
    row_ptr, col = synth.adjacency_csr(n, eu, ev)
    G = hw.hw_graph_csr(n, row_ptr, col)
    A2, B, steps = G.num_arcs, 64, 500
    psi0 = synth.gaussian_states_device(A2, B, seed=4, dtype=torch.complex64)
    out = torch.empty_like(psi0)
    norm = torch.empty(B, dtype=torch.float64, device="cuda")
    prob = torch.empty(n * B, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    hw.hw_coined_evolve(G, 0, [], hw.HW_C64, B, 2, psi0, out)   # autotunes the launch shape once
    for _ in range(max(1, warmup)):
        hw.hw_coined_evolve(G, 0, [], hw.HW_C64, B, steps, psi0, out)
    torch.cuda.synchronize()
    tot = ev_t = 0.0
    with Clocks(torch.cuda.current_device()) as clk:
        for _ in range(reps):
            flush.zero_()
            e = _events(3)
            e[0].record(stream)
            hw.hw_coined_evolve(G, 0, [], hw.HW_C64, B, steps, psi0, out)
            e[1].record(stream)
            hw.hw_probability(G, n, hw.HW_C64, B, out, prob, norm)
            e[2].record(stream)
            torch.cuda.synchronize()
            tot += e[0].elapsed_time(e[2]) / 1e3
            ev_t += e[0].elapsed_time(e[1]) / 1e3
    peak, src = measured_peaks()
    per_launch = ev_t / (reps * steps)
    bytes_launch = A2 * (2 * B * 8 + 4) + 4 * (n + 1)
    nm = norm.cpu().numpy()
    res = {"workload": "er_batched", "metric": METRIC, "unit": UNIT,
           "value": A2 * B * steps * reps / tot, "ms_per_run": 1e3 * tot / reps, "ms_per_walk_step": per_launch * 1e3,
           "n": n, "arcs": A2, "batch": B, "walk_steps": steps, "reps": reps, "dtype": "f32 (fp64 sums)",
           "l2": "256 MiB written before every timed run; the 4.3 GB states exceed L2",
           "input": "synth.gaussian_states_device(seed 4), complex64",
           "roofline": {"bound": "hbm", "achieved": bytes_launch / per_launch / 1e9, "peak": peak,
                        "unit": "GB/s", "frac": bytes_launch / per_launch / 1e9 / peak,
                        "bytes_per_launch": bytes_launch, "launch_us": per_launch * 1e6, "peak_source": src},
           "norm_minmax": [float(nm.min()), float(nm.max())], "clocks": clk.summary()}
    del flush
    # the same run in complex128 (pinned to the oracle at 1e-12 by the tests)
    # as the reference for the complex64 result's error
    x128 = psi0.to(torch.complex128)
    y128 = torch.empty_like(x128)
    hw.hw_coined_evolve(G, 0, [], hw.HW_C128, B, steps, x128, y128)
    p128 = torch.empty(n * B, dtype=torch.float64, device="cuda")
    hw.hw_probability(G, n, hw.HW_C128, B, y128, p128)
    torch.cuda.synchronize()
    dp = (prob - p128).view(n, B).abs().sum(dim=0)
    res["c64_vs_c128"] = {"p_L1_max_over_columns": float(dp.max().item()),
                          "psi_max_abs": float((out.to(torch.complex128) - y128).abs().max().item())}
    del x128, y128, p128
    if with_cpu:
        import oracle
        ar = oracle.Arcs(n, eu, ev)
        start = psi0[:, 0].cpu().numpy().astype(np.complex128)
        t0 = time.perf_counter()
        ref = oracle.coined_evolve(ar, start, steps)
        el = time.perf_counter() - t0
        got = out[:, 0].cpu().numpy().astype(np.complex128)
        res["cpu_baseline"] = {"value": A2 * steps / el, "unit": UNIT, "cores": _oracle_cores(), "kind": "oracle",
                               "sample": "batch column 0, all 500 steps (one of the 64 columns)"}
        res["error_vs_oracle"] = {
            "column": 0, "c64_max_abs_psi": float(np.max(np.abs(got - ref))),
            "c64_p_L1": float(np.sum(np.abs(prob.view(n, B)[:, 0].cpu().numpy() - oracle.prob_coined(ar, ref))))}
    G.free()
    return res


def run_workload_weighted(args):
    """CTQW with a weighted adjacency H = -gamma W - |m><m|: (1) the Q_12 search of the
    CTQW workload with seeded real edge weights in [0.25, 1.75) (dense U by the
    Taylor series; complex64 needs two fp16 slices of Y, the unweighted walk one),
    (2) the sparse-action series on the 2^20-vertex hypercube with real and with
    complex (Hermitian) weights, gamma = 1/20, dt = 0.1, 20 applications."""
    import torch
    import paper_2406_08186_b300 as hw
    stream = torch.cuda.current_stream()
    fp64 = hw.hw_measure_fp64()
    res = {"workload": "weighted_ctqw", "fp64_peak_ops": fp64}
    n, eu, ev = synth.hypercube(12)
    m = synth.seeded_vertex(3, n)
    rp, col, w = synth.weighted_csr(n, eu, ev, synth.edge_weights(eu.size, seed=9))
    G = hw.hw_graph_csr_weighted(n, rp, col, w)
    for dt, name in ((hw.HW_C128, "q12_expm_c128"), (hw.HW_C64, "q12_expm_c64")):
        cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
        U = torch.empty((n, n), dtype=cdt, device="cuda")
        for _ in range(max(1, args.warmup)):
            hw.hw_ctqw_expm(G, 1 / 12, [m], 0.1, dt, U)
        torch.cuda.synchronize()
        e = _events(2)
        e[0].record(stream)
        for _ in range(args.steps):
            hw.hw_ctqw_expm(G, 1 / 12, [m], 0.1, dt, U)
        e[1].record(stream)
        torch.cuda.synchronize()
        t = e[0].elapsed_time(e[1]) / 1e3 / args.steps
        deg, sq = hw.hw_ctqw_plan(G, 1 / 12, [m], 0.1)
        res[name] = {"ms": t * 1e3, "taylor_degree": deg, "squarings": sq,
                     "gemm_tflops_useful": (deg - 1) * 2.0 * n ** 3 / t / 1e12}
    G.free()
    k = 20
    n, eu, ev = synth.hypercube(k)
    m = synth.seeded_vertex(3, n)
    walk = 20
    for cplx in (False, True):
        rp, col, w = synth.weighted_csr(n, eu, ev, synth.edge_weights(eu.size, seed=5, complex_phase=cplx))
        G = hw.hw_graph_csr_weighted(n, rp, col, w)
        deg, sq = hw.hw_ctqw_plan(G, 1.0 / k, [m], 0.1)
        terms = walk * deg * (1 << sq)
        for dt, esz in ((hw.HW_C128, 16), (hw.HW_C64, 8)):
            cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
            x = torch.full((n,), 1.0 / math.sqrt(n), dtype=cdt, device="cuda")
            y = torch.empty_like(x)
            hw.hw_ctqw_evolve_sparse(G, 1.0 / k, [m], 0.1, dt, 1, 2, x, y)
            torch.cuda.synchronize()
            e = _events(2)
            e[0].record(stream)
            for _ in range(args.steps):
                hw.hw_ctqw_evolve_sparse(G, 1.0 / k, [m], 0.1, dt, 1, walk, x, y)
            e[1].record(stream)
            torch.cuda.synchronize()
            per_term = e[0].elapsed_time(e[1]) / 1e3 / args.steps / terms
            r = {"us_per_term": per_term * 1e6, "terms": terms, "gathers_per_s": (G.num_arcs + n) / per_term}
            if dt == hw.HW_C128:
                # FP64 operations per vertex: 2 (real) or 4 (complex) FMAs per
                # neighbour, two multiplies and two adds for the term and the sum
                ops = n * ((4 if cplx else 2) * k + 4)
                r["fp64_ops_per_s"] = ops / per_term
                r["frac_fp64_measured"] = ops / per_term / fp64
            res["q20_sparse_%s_%s" % ("complex" if cplx else "real", "c128" if dt == hw.HW_C128 else "c64")] = r
        G.free()
    print(json.dumps(res), flush=True)


def run_workload_sampled(args):
    """The 1024 x 1024 torus search sampled like simulate(range=(0, 3000, 100)): the
    per-vertex probabilities of 30 states (states not kept) and the search curve, for
    complex128 and complex64, against one plain 3000-step evolve of the same walk."""
    import torch
    import paper_2406_08186_b300 as hw
    n, eu, ev, row_ptr, col, m = workload()
    G = hw.hw_graph_csr(n, row_ptr, col)
    stream = torch.cuda.current_stream()
    res = {"workload": "torus1024_sampled", "metric": METRIC, "unit": UNIT, "range": [0, WALK_STEPS, 100]}
    R = hw.sample_count(0, WALK_STEPS, 100)
    for dt, name in ((hw.HW_C128, "c128"), (hw.HW_C64, "c64")):
        cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
        psi0 = torch.full((G.num_arcs,), 1.0 / math.sqrt(G.num_arcs), dtype=cdt, device="cuda")
        out = torch.empty_like(psi0)
        prob = torch.empty((R, n), dtype=torch.float64, device="cuda")
        steps_total = (R - 1) * 100
        for _ in range(max(1, args.warmup)):
            hw.hw_coined_sample(G, 0, [m], dt, 1, 0, WALK_STEPS, 100, psi0, None, prob)
        torch.cuda.synchronize()
        e = _events(4)
        e[0].record(stream)
        for _ in range(args.steps):
            hw.hw_coined_sample(G, 0, [m], dt, 1, 0, WALK_STEPS, 100, psi0, None, prob)
        e[1].record(stream)
        for _ in range(args.steps):
            hw.hw_coined_evolve(G, 0, [m], dt, 1, steps_total, psi0, out)
        e[2].record(stream)
        torch.cuda.synchronize()
        t_s = e[0].elapsed_time(e[1]) / 1e3 / args.steps
        t_p = e[1].elapsed_time(e[2]) / 1e3 / args.steps
        curve, k, pmax = hw.success_curve(prob, [m])
        res[name] = {"samples": R, "value": G.num_arcs * steps_total / t_s, "ms_sampled": t_s * 1e3,
                     "ms_plain_evolve": t_p * 1e3, "overhead": t_s / t_p - 1.0,
                     "best_sample_step": k * 100, "best_p_m": pmax}
    print(json.dumps(res), flush=True)
    G.free()


# nominal FP64 rate of the B300 (1.25 TFLOP/s): 0.625e12 FP64 pipe operations
# (FMA, add or multiply) per second
FP64_OPS_NOMINAL = 0.625e12


def run_workload_sparse_ctqw(args):
    """Continuous-time walk by the sparse action of e^{-iH dt} (no dense U) on the
    2^20-vertex hypercube: gamma = 1/20, one seeded mark, dt = 0.1, uniform start,
    20 walk steps of m Taylor terms each; complex128 and complex64, with the
    neighbours computed from the labels (default) and read from the CSR."""
    import torch
    import paper_2406_08186_b300 as hw
    k = 20
    n, eu, ev = synth.hypercube(k)
    row_ptr, col = synth.adjacency_csr(n, eu, ev)
    G = hw.hw_graph_csr(n, row_ptr, col)
    m = synth.seeded_vertex(3, n)
    gamma, tstep, walk = 1.0 / k, 0.1, 20
    deg, sq = hw.hw_ctqw_plan(G, gamma, [m], tstep)
    terms = walk * deg * (1 << sq)
    stream = torch.cuda.current_stream()
    res = {"workload": "hypercube20_sparse_ctqw", "n": n, "arcs": G.num_arcs, "walk_steps": walk,
           "taylor_degree": deg, "terms": terms}
    peak, _ = measured_peaks()
    for dt, name, esz in ((hw.HW_C128, "c128", 16), (hw.HW_C64, "c64", 8)):
        cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
        x = torch.full((n,), 1.0 / math.sqrt(n), dtype=cdt, device="cuda")
        y = torch.empty_like(x)
        for addressing, tag in ((0, ""), (1, "_csr")):
            opts = {"addressing": addressing}
            for _ in range(max(1, args.warmup)):
                hw.hw_ctqw_evolve_sparse(G, gamma, [m], tstep, dt, 1, 2, x, y, opts=opts)
            torch.cuda.synchronize()
            e = _events(2)
            e[0].record(stream)
            for _ in range(args.steps):
                hw.hw_ctqw_evolve_sparse(G, gamma, [m], tstep, dt, 1, walk, x, y, opts=opts)
            e[1].record(stream)
            torch.cuda.synchronize()
            t = e[0].elapsed_time(e[1]) / 1e3 / args.steps
            per_term = t / terms
            # compulsory DRAM bytes per term: t_{k-1} once (its neighbour gathers
            # hit L2), t_k written, the sum (or x) read and written; the CSR path
            # adds row_ptr and head.  The complex64 working set (four 8 MB
            # vectors) stays in L2, so its bytes are L2 traffic.
            term_bytes = 4 * esz * n + (4 * (n + 1) + 4 * G.num_arcs if addressing else 0)
            # FP64 operations per term (complex128): d - 1 adds per component for
            # the neighbour sum, two multiplies, two adds into the sum
            fp64_ops = n * (2 * (k - 1) + 4)
            r = {"ms": t * 1e3, "us_per_term": per_term * 1e6, "gathers_per_s": (G.num_arcs + n) / per_term,
                 "bytes_per_term": term_bytes, "achieved_gbs": term_bytes / per_term / 1e9,
                 "frac_hbm": term_bytes / per_term / 1e9 / peak}
            if dt == hw.HW_C128:
                r["fp64_ops_per_s"] = fp64_ops / per_term
                r["frac_fp64_nominal"] = fp64_ops / per_term / FP64_OPS_NOMINAL
            res[name + tag] = r
    print(json.dumps(res), flush=True)
    G.free()


def serving_jobs(count, seed=6):
    """The serving mix: kind, graph family, size, steps, dtype and marks per job, all from
    SplitMix64(seed).  n = 2^k with k uniform in 10..20 for coined jobs and in 10..13 for
    CTQW jobs (log-uniform sizes); steps log-uniform in [10, 5000]; coined/CTQW and
    complex64/complex128 50/50; 0-4 marked vertices; gamma = 1/degree, dt = 0.1."""
    u = synth.uniform01(seed, 8 * count).reshape(count, 8)
    fams = ["torus", "hypercube", "reg3", "reg4", "reg8"]
    jobs = []
    for i in range(count):
        kind = int(u[i, 0] < 0.5)                       # 0 coined, 1 CTQW
        fam = fams[min(4, int(u[i, 1] * 5))]
        k = 10 + (min(10, int(u[i, 2] * 11)) if kind == 0 else min(3, int(u[i, 2] * 4)))
        steps = int(round(math.exp(math.log(10) + u[i, 3] * (math.log(5000) - math.log(10)))))
        dt = 1 if u[i, 4] < 0.5 else 2
        nm = min(4, int(u[i, 5] * 5))
        jobs.append({"kind": kind, "fam": fam, "k": k, "steps": steps, "dt": dt, "n_marked": nm,
                     "mark_seed": 1000 + i})
    return jobs


def menu_graph(fam, k):
    """(n, row_ptr, col, degree) of one graph of the serving mix (host only)."""
    if fam == "torus":
        L = int(round(math.sqrt(1 << k)))
        n, eu, ev = synth.torus(L)
        d = 4
    elif fam == "hypercube":
        n, eu, ev = synth.hypercube(k)
        d = k
    else:
        d = int(fam[3:])
        n, eu, ev = synth.random_regular(1 << k, d, seed=100 + k * 10 + d)
    row_ptr, col = synth.adjacency_csr(n, eu, ev)
    return n, row_ptr, col, d


def _menu_graph_star(key):
    return key, menu_graph(*key)


class GraphMenu:
    """Resident graphs of the serving mix, generated on the host cores by a
    process pool (spawned, so no worker inherits a CUDA context) and uploaded
    before any timing."""

    def __init__(self, hw, keys):
        import concurrent.futures
        import multiprocessing
        self.hw = hw
        self.g = {}
        keys = sorted(set(keys), key=lambda fk: -fk[1])       # largest first
        workers = max(1, min(16, os.cpu_count() or 1, len(keys)))
        ctx = multiprocessing.get_context("spawn")
        with concurrent.futures.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as pool:
            for key, (n, row_ptr, col, d) in pool.map(_menu_graph_star, keys):
                self.g[key] = (hw.hw_graph_csr(n, row_ptr, col), d)

    def get(self, fam, k):
        return self.g[(fam, k)]

    def free(self):
        for G, _ in self.g.values():
            G.free()


def sub_serving(hw, count, substeps=16, arena_gb=64.0, baseline_jobs=None):
    """Configuration 5: a stream of `count` walk jobs (the serving mix of seed 6)
    served by continuous batching, saturated (all jobs at t = 0) and with Poisson
    arrivals at 0.8 x the saturated rate: walks/s and p50/p99 latency (arrival to
    result on the host), against the plain one-job-at-a-time complex128 path on
    the same jobs (the first `baseline_jobs` of them when given); each served
    result's error against that complex128 result."""
    import torch
    jobs = serving_jobs(count)
    menu = GraphMenu(hw, [(j["fam"], j["k"]) for j in jobs])
    for j in jobs:
        G, d = menu.get(j["fam"], j["k"])
        j["G"], j["d"] = G, d
        j["marked"] = sorted({synth.seeded_vertex(j["mark_seed"] + r, G.n) for r in range(j["n_marked"])})
    arena = int(arena_gb * (1 << 30))
    kept = {}

    def serve(arrivals, keep):
        srv = hw.Server(arena, max_jobs=512, substeps=substeps, host_bytes=4 << 30)
        t0 = time.perf_counter()
        pending = sorted(range(len(jobs)), key=lambda i: arrivals[i])
        nxt = 0
        idmap, lat = {}, []
        while len(lat) < len(jobs):
            now = time.perf_counter() - t0
            while nxt < len(pending) and arrivals[pending[nxt]] <= now:
                i = pending[nxt]
                j = jobs[i]
                idmap[srv.submit(j["G"], j["kind"], j["dt"], j["steps"], j["marked"], gamma=1.0 / j["d"],
                                 time=0.1)] = i
                nxt += 1
            srv.run()
            for jid in srv.poll():
                i = idmap.pop(jid)
                lat.append(time.perf_counter() - t0 - arrivals[i])
                prob, rec, _ = srv.result(jid)
                if keep:
                    kept[i] = (prob, rec)
            if nxt < len(pending) and not idmap:
                time.sleep(max(0.0, min(0.001, arrivals[pending[nxt]] - (time.perf_counter() - t0))))
        el = time.perf_counter() - t0
        srv.close()
        lat = np.sort(np.array(lat))
        return {"walks_per_s": len(jobs) / el, "makespan_s": el, "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean())}

    with Clocks(torch.cuda.current_device()) as clk:
        sat = serve([0.0] * len(jobs), True)
        lam = 0.8 * sat["walks_per_s"]
        gaps = -np.log1p(-synth.uniform01(61, len(jobs))) / lam
        poisson = serve(list(np.cumsum(gaps)), False)
    clocks = clk.summary()

    # plain one-job-at-a-time complex128 path on the same jobs, each result
    # copied back like a served one; the served results are compared with it
    base_jobs = list(range(len(jobs) if baseline_jobs is None else min(len(jobs), baseline_jobs)))
    err = {"c128_max_abs_p": 0.0, "c64_max_L1_p": 0.0, "record_max_abs": 0.0}
    torch.cuda.synchronize()
    t_plain = 0.0
    for i in base_jobs:
        j = jobs[i]
        G = j["G"]
        t0 = time.perf_counter()
        dim = G.num_arcs if j["kind"] == 0 else G.n
        x = torch.full((dim,), 1.0 / math.sqrt(dim), dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        rec = torch.empty(j["steps"], dtype=torch.float64, device="cuda") if j["marked"] else None
        if j["kind"] == 0:
            hw.hw_coined_evolve(G, 0, j["marked"], hw.HW_C128, 1, j["steps"], x, y, rec)
        else:
            hw.hw_ctqw_evolve_sparse(G, 1.0 / j["d"], j["marked"], 0.1, hw.HW_C128, 1, j["steps"], x, y, rec)
        prob = torch.empty(G.n, dtype=torch.float64, device="cuda")
        hw.hw_probability(G if j["kind"] == 0 else None, G.n, hw.HW_C128, 1, y, prob)
        p_h = prob.cpu().numpy()
        r_h = rec.cpu().numpy() if rec is not None else None
        t_plain += time.perf_counter() - t0
        sp, sr = kept[i]
        if j["dt"] == hw.HW_C128:
            err["c128_max_abs_p"] = max(err["c128_max_abs_p"], float(np.max(np.abs(sp - p_h))))
        else:
            err["c64_max_L1_p"] = max(err["c64_max_L1_p"], float(np.sum(np.abs(sp - p_h))))
        if r_h is not None:
            err["record_max_abs"] = max(err["record_max_abs"], float(np.max(np.abs(sr - r_h))))
    base_rate = len(base_jobs) / t_plain
    menu.free()
    return {"workload": "serving", "jobs": len(jobs), "metric": "walks/s", "unit": "walks/s",
            "saturated": sat, "poisson_0.8": poisson, "lambda_per_s": lam,
            "plain_c128_one_at_a_time": {"walks_per_s": base_rate, "jobs_timed": len(base_jobs),
                                         "same_jobs": len(base_jobs) == len(jobs), "seconds": t_plain},
            "speedup_saturated_vs_plain": sat["walks_per_s"] / base_rate,
            "speedup_poisson_vs_plain": poisson["walks_per_s"] / base_rate,
            "served_vs_plain_c128_error": err,
            "substeps_per_round": substeps, "arena_gb": arena_gb, "clocks": clocks}


def run_workload_serving(args):
    import paper_2406_08186_b300 as hw  # noqa: F401
    print(json.dumps(sub_serving(hw, args.jobs, args.substeps, args.arena_gb, args.baseline_jobs)), flush=True)


def run_profile(args):
    """A few launches of one kernel on the bench workload, for ncu captures."""
    import torch
    import paper_2406_08186_b300 as hw
    if args.profile == "batched_c64":
        # Erdos-Renyi n = 2^18, mean degree 8, 64 complex64 states (about 2 GB on the device)
        n0 = 1 << 18
        n, eu, ev = synth.erdos_renyi(n0, 8.0 / (n0 - 1), seed=5)
        row_ptr, col = synth.adjacency_csr(n, eu, ev)
        G = hw.hw_graph_csr(n, row_ptr, col)
        gen = torch.Generator(device="cuda").manual_seed(4)
        x = torch.randn((G.num_arcs, 64), dtype=torch.complex64, device="cuda", generator=gen)
        out = torch.empty_like(x)
        hw.hw_coined_evolve(G, 0, [], hw.HW_C64, 64, args.profile_steps, x, out,
                            opts={"tile": args.profile_tile})
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "steps": args.profile_steps, "tile": args.profile_tile}))
        G.free()
        return
    if args.profile == "cluster_torus64":
        # configuration 1: one 100-step run of the 64 x 64 torus (one cluster launch)
        n, eu, ev = synth.torus(64)
        row_ptr, col = synth.adjacency_csr(n, eu, ev)
        G = hw.hw_graph_csr(n, row_ptr, col)
        psi0 = torch.from_numpy(synth.state_on_vertex_arcs(synth.arc_offsets(n, eu, ev), 32 * 64 + 32)).cuda()
        out = torch.empty_like(psi0)
        hw.hw_coined_evolve(G, 0, [], hw.HW_C128, 1, 100, psi0, out)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile}))
        G.free()
        return
    if args.profile.startswith("cube20_"):
        # the 2^20-vertex hypercube (degree 20), uniform start, one seeded mark, profile_steps steps
        k = 20
        n, eu, ev = synth.hypercube(k)
        row_ptr, col = synth.adjacency_csr(n, eu, ev)
        G = hw.hw_graph_csr(n, row_ptr, col)
        dt = hw.HW_C128 if args.profile.endswith("c128") else hw.HW_C64
        cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
        x = torch.full((G.num_arcs,), 1.0 / math.sqrt(G.num_arcs), dtype=cdt, device="cuda")
        y = torch.empty_like(x)
        hw.hw_coined_evolve(G, 0, [synth.seeded_vertex(3, n)], dt, 1, args.profile_steps, x, y)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "steps": args.profile_steps}))
        G.free()
        return
    if args.profile in ("expm_sparse_c128", "expm_sparse_c64"):
        # the 4096-vertex hypercube CTQW: one expm with the Taylor powers as sparse x dense products
        n = 4096
        m = synth.seeded_vertex(3, n)
        row_ptr, col = synth.adjacency_csr(*synth.hypercube(12))
        G = hw.hw_graph_csr(n, row_ptr, col)
        dt = hw.HW_C128 if args.profile.endswith("c128") else hw.HW_C64
        U = torch.empty((n, n), dtype=torch.complex128 if dt == hw.HW_C128 else torch.complex64, device="cuda")
        hw.hw_ctqw_expm(G, 1 / 12, [m], 0.1, dt, U, opts={"taylor_powers": 2})
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile}))
        G.free()
        return
    if args.profile in ("expm_c64", "apply_c128", "apply_c64", "apply_sym_c64"):
        # the 4096-vertex hypercube CTQW: one expm (11 tensor-core powers) or a few applications
        n = 4096
        m = synth.seeded_vertex(3, n)
        row_ptr, col = synth.adjacency_csr(*synth.hypercube(12))
        G = hw.hw_graph_csr(n, row_ptr, col)
        dt = hw.HW_C128 if args.profile.endswith("c128") else hw.HW_C64
        cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
        U = torch.empty((n, n), dtype=cdt, device="cuda")
        hw.hw_ctqw_expm(G, 1 / 12, [m], 0.1, dt, U)
        if args.profile.startswith("apply"):
            x = torch.full((n,), 1 / 64, dtype=cdt, device="cuda")
            y = torch.empty_like(x)
            opts = {"u_symmetric": 1} if args.profile == "apply_sym_c64" else None
            hw.hw_ctqw_evolve(U, n, dt, 1, args.profile_steps, x, y, [m], opts=opts)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile}))
        G.free()
        return
    if args.profile.startswith("sparse_"):
        # sparse-action CTQW on the 1024 x 1024 torus or the 2^20-vertex hypercube,
        # gamma = 1/4 (1/20), one seeded mark, dt = 0.1, profile_steps applications
        if "torus" in args.profile:
            n, eu, ev = synth.torus(1024)
            gamma = 0.25
        else:
            n, eu, ev = synth.hypercube(20)
            gamma = 1.0 / 20
        row_ptr, col = synth.adjacency_csr(n, eu, ev)
        G = hw.hw_graph_csr(n, row_ptr, col)
        m = synth.seeded_vertex(3, n)
        dt = hw.HW_C128 if args.profile.endswith("c128") else hw.HW_C64
        cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
        x = torch.full((n,), 1.0 / math.sqrt(n), dtype=cdt, device="cuda")
        y = torch.empty_like(x)
        hw.hw_ctqw_evolve_sparse(G, gamma, [m], 0.1, dt, 1, args.profile_steps, x, y)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "steps": args.profile_steps}))
        G.free()
        return
    n, eu, ev, row_ptr, col, m = workload()
    G = hw.hw_graph_csr(n, row_ptr, col)
    dt = hw.HW_C128 if args.profile.endswith("c128") else hw.HW_C64
    cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
    psi0 = torch.full((G.num_arcs,), 1.0 / math.sqrt(G.num_arcs), dtype=cdt, device="cuda")
    out = torch.empty_like(psi0)
    rec = torch.empty(args.profile_steps, dtype=torch.float64, device="cuda")
    hw.hw_coined_evolve(G, hw.HW_COIN_GROVER, [m], dt, 1, args.profile_steps, psi0, out, rec)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "steps": args.profile_steps,
                      "p_m_last": float(rec[-1].item())}))
    G.free()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", choices=["coined_c128", "coined_c64", "batched_c64", "expm_c64", "apply_c128",
                                          "apply_c64", "apply_sym_c64", "sparse_torus_c64", "sparse_torus_c128",
                                          "sparse_cube_c64", "sparse_cube_c128", "cluster_torus64",
                                          "cube20_c128", "cube20_c64", "expm_sparse_c128", "expm_sparse_c64"],
                    help="run a few coin+shift launches of the workload and exit (for ncu)")
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--profile-tile", type=int, default=10)
    ap.add_argument("--workload", default="torus1024_search",
                    choices=["torus1024_search", "torus64_center", "hypercube12_ctqw", "er_batched",
                             "serving", "sampled", "sparse_ctqw", "weighted_ctqw"],
                    help="the default is the benchmarked workload; the others print their own line")
    ap.add_argument("--jobs", type=int, default=10000, help="serving: number of jobs")
    ap.add_argument("--baseline-jobs", type=int, default=None,
                    help="serving: jobs timed on the plain path (default: all of them)")
    ap.add_argument("--serving-jobs", type=int, default=1000,
                    help="default line: jobs of the serving stream in its serving record")
    ap.add_argument("--no-configs", action="store_true",
                    help="default line without the records of configurations 1, 3, 4 and 5")
    ap.add_argument("--substeps", type=int, default=16, help="serving: sub-steps per round")
    ap.add_argument("--arena-gb", type=float, default=64.0, help="serving: device arena")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
    elif args.workload in ("er_batched", "hypercube12_ctqw", "torus64_center"):
        import paper_2406_08186_b300 as hw
        fn = {"er_batched": sub_er_batched, "hypercube12_ctqw": sub_ctqw_q12,
              "torus64_center": sub_torus64}[args.workload]
        print(json.dumps(fn(hw, reps=args.steps, warmup=args.warmup, with_cpu=not args.no_cpu_baseline)),
              flush=True)
    elif args.workload == "sampled":
        run_workload_sampled(args)
    elif args.workload == "sparse_ctqw":
        run_workload_sparse_ctqw(args)
    elif args.workload == "weighted_ctqw":
        run_workload_weighted(args)
    elif args.workload == "serving":
        run_workload_serving(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
