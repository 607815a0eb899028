"""Benchmark: incidence-constrained multilevel partitioning of the 16k-node
random SNN hypergraph (16,384 neurons, 128 pins per hyperedge, 2,097,152
pins; Omega = 2^10 nodes, Delta = 2^12 inbound hyperedges) on GB300.

One step = the whole path over one input: hgp_create (level-0 incidence
build from the device-resident CSR) + hgp_partition (every coarsening level:
Eq. (2) scoring with deferred checks, matching, contraction; every
refinement level: Eq. (3) moves, in-sequence gains, prefix validity;
projection; output) + hgp_destroy.

value = level-0 pins / step time (pins/s), whole job over all ranks, from
        steps with no instrumentation; a few separate steps with CUDA events
        around every phase give the kernel split and the rooflines.
e2e   = the same through the C ABI with pinned HOST input and output
        buffers, the copies inside the timed region.
The L2 (129 MB) is flushed between timed steps (the inputs are 8.4 MB).
The same line also reports the learned candidate order on this workload
(model trained untimed on seeded 16k-64k-node graphs), the constraint-only
fill as a quality floor, and whole plain and learned partitions of the
262,144-node SNN (67 M pins) with their cost and time ratio.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

cpu_baseline and --impl reference time the CPU oracle (the plain
single-threaded C restatement of the method used for parity) on the host
cores on a bounded sample of this same workload: the method cut after its
first coarsening level (the GPU's time on the same cut is reported beside
it).  Multi-GPU: independent replicas (the method does not shard), one per
rank under torchrun.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "coarsening pins/s and partition wall-time at equal λ−1 cost, plain vs learned"
OMEGA, DELTA = 1 << 10, 1 << 12
WORKLOAD = "random SNN hypergraph, 16,384 nodes, one hyperedge per node of 128 pins (src + 127 distinct targets), 2,097,152 pins, int32 CSR, Omega=2^10, Delta=2^12, seed 0"
# training set of the learned order: random SNN graphs of 16k, 32k and 64k
# nodes (cycling), hyperedges of 128..256 pins, seeds 100..115
LEARN_TRAIN_GRAPHS, LEARN_TRAIN_SIZES = 16, (16384, 32768, 65536)
LEARN_PER_NODE, LEARN_STEPS, LEARN_BATCH, LEARN_LR, LEARN_KEY_BITS = 4, 2000, 4096, 3e-3, 6
LEARN_SM_GHZ = 2.07          # maximum SM clock of the GB300
INSTRUMENTED_STEPS = 2       # separate steps with phase events, for the kernel split
CUT_LEVELS = 1               # the CPU baseline's bounded prefix of the method
SAMPLE_DESC = ("the same workload (16k SNN, Omega=2^10, Delta=2^12) through the method's first "
               f"{CUT_LEVELS} coarsening level(s): incidence build, Eq. 2 scoring with the "
               "Omega/Delta checks, matching, then refinement of that level from the matched "
               "clusters (hgp_options.max_levels / the oracle's cut; the whole method takes "
               "435 levels and ~2,100 s of oracle time on one core)")


# DRAM bytes (read + write) per launch from one ncu capture of the kernel
# (dram__bytes_read.sum + dram__bytes_write.sum, mean of launches 201-202 of
# one step of this workload: a mid-level sample, since a full-set capture is
# kept to a few launches), valid only while the kernel's sources are the ones
# captured.
MEASURED_TRAFFIC = {
    "k_score": (13991680.0, {
        "paper_2604_14411_gb300/csrc/k_score.cuh":
            "d1ac607cacbceedd1e8699efce2e59181c1c7a040096f6d3d70075d7b0404f9e",
        "paper_2604_14411_gb300/csrc/k_score.cu":
            "704c92398342b82947d3edf68c6c170214439b1e3a853f5a05862c5dbce5681a"}),
}

def measured_traffic(kernel):
    entry = MEASURED_TRAFFIC.get(kernel)
    if entry is None:
        return None
    value, files = entry
    for rel, digest in files.items():
        path = os.path.join(ROOT, rel)
        if not os.path.exists(path):
            return None
        with open(path, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    return value


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks sampled every 200 ms while running."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, gpu_index=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9 or parts[0] != str(gpu_index):
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def clocks_path(args, rank):
    """Where the nvidia-smi samples of the timed region go (--clocks-dir)."""
    d = args.clocks_dir or tempfile.gettempdir()
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, f"clocks_{args.workload}_rank{rank}.csv")


def job_time_ms(local_ms: float, dist=None, device=None) -> float:
    """Timed region of the whole job: the maximum over ranks of each rank's
    summed step time (ranks run independent replicas)."""
    if dist is None:
        return local_ms
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_step: int, steps: int, world: int, job_ms: float) -> float:
    """Whole-job throughput: units processed by all ranks / job time."""
    return units_per_step * steps * world / (job_ms / 1000.0)


def _oracle_cut_step(g):
    """One bounded sample on the CPU oracle: build + the method cut after
    CUT_LEVELS levels, as one GPU step builds and partitions."""
    import oracle
    t = time.perf_counter()
    with oracle.Run.from_graph(g) as r:
        r.partition(OMEGA, DELTA, 1, CUT_LEVELS)
    return time.perf_counter() - t


def oracle_sample(steps=1):
    """Times the CPU oracle on the bounded sample; returns (pins/s, seconds)."""
    import synth
    g = synth.snn_16k(0)
    ts = [_oracle_cut_step(g) for _ in range(steps)]
    return g.num_pins / statistics.median(ts), ts


def run_reference(args, rank, world):
    """CPU oracle arm: rank 0 only, K timed steps of the bounded sample."""
    if rank != 0:
        return
    import synth
    g = synth.snn_16k(0)
    for _ in range(args.warmup):
        _oracle_cut_step(g)
    ts = [_oracle_cut_step(g) for _ in range(args.steps)]
    tot = sum(ts)
    value = g.num_pins * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pins/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "omega": OMEGA, "delta": DELTA, "pins": 2097152,
                       "sample": SAMPLE_DESC},
            "cpu_baseline": {"value": value, "unit": "pins/s", "cores": 1, "kind": "oracle",
                             "sample": SAMPLE_DESC},
            "e2e": {"value": value, "unit": "pins/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BATCH_WORKLOAD = ("64 SNN hypergraphs, N log-uniform in [2048, 65536] (seed 0); even: random, edge "
                  "size U{32..256}; odd: layered conv-style 8 x 16x16 x ch; Omega=2^10, Delta=2^12 "
                  "for all; 150,771,047 pins in total")


def run_batch(args, rank, world):
    """64 uneven hypergraphs per step through hgp_partition_batch (instances on
    concurrent streams); also times them one at a time once for comparison."""
    import torch
    import synth
    from paper_2604_14411_gb300 import hgp as H

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    H.load()
    inst = synth.batch_instances(64, 0)
    pins = sum(g.num_pins for g in inst)
    graphs = [H.Graph.from_hypergraph(g) for g in inst]
    om, de = [OMEGA] * len(graphs), [DELTA] * len(graphs)
    for _ in range(args.warmup):
        H.hgp_partition_batch(graphs, om, de)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(clocks_path(args, rank))
    sampler.start()
    t = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = H.hgp_partition_batch(graphs, om, de)
        torch.cuda.synchronize()
        t.append(1000.0 * (time.perf_counter() - t0))
    clocks = sampler.stop(local)
    job = job_time_ms(sum(t), dist, torch.device("cuda", local))
    t0 = time.perf_counter()
    for G in graphs:
        G.partition(OMEGA, DELTA)
    seq_ms = 1000.0 * (time.perf_counter() - t0)
    learned = None
    if not args.no_learned:
        # the same batch with the learned order (model trained untimed on 16k-node graphs)
        model, _, train_s, _ = train_learned_model(H, None)
        H.hgp_partition_batch(graphs, om, de, model=model)
        torch.cuda.synchronize()
        lt = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            lres = H.hgp_partition_batch(graphs, om, de, model=model)
            torch.cuda.synchronize()
            lt.append(1000.0 * (time.perf_counter() - t0))
        lms = statistics.median(lt)
        feas = all(recount(g, r.part_ids, OMEGA, DELTA)[1] for g, r in zip(inst, lres))
        lcost = int(sum(r.cost for r in lres))
        learned = {"ms_per_step": lms, "pins_per_s": pins / (lms / 1000.0), "total_cost": lcost,
                   "cost_ratio_vs_plain": lcost / max(1, int(sum(r.cost for r in res))),
                   "time_ratio_vs_plain": lms / (job / args.steps), "all_feasible": feas,
                   "training_seconds": train_s, "steps": len(lt)}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": job_value(pins, args.steps, world, job), "unit": "pins/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": job / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "pins": pins, "instances": len(graphs),
                       "timing": "host clock around hgp_partition_batch (device-resident inputs)"},
            "sequential_ms": seq_ms, "batch_speedup_vs_sequential": seq_ms / (job / args.steps),
            "total_cost": int(sum(r.cost for r in res)), "total_parts": int(sum(r.num_parts for r in res)),
            "clocks": clocks, **({"learned": learned} if learned else {})}), flush=True)
    for G in graphs:
        G.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def recount(g, ids, omega, delta):
    """Cost (Eq. 1) and feasibility of a partition recounted on the host."""
    off = g.offsets.astype(np.int64)
    E = len(off) - 1
    sizes = np.diff(off)
    edge = np.repeat(np.arange(E, dtype=np.int64), sizes)
    part = ids[g.pins].astype(np.int64)
    K = int(ids.max()) + 1
    lam = np.bincount(np.unique(edge * K + part) // K, minlength=E)
    cost = int((lam - 1).sum())
    weight = np.bincount(ids, minlength=K)
    dst = np.ones(len(g.pins), dtype=bool)
    dst[off[:-1]] = False                                  # first pin = source
    inbound = np.bincount(np.unique(part[dst] * E + edge[dst]) // E, minlength=K)
    return cost, bool(weight.max() <= omega and inbound.max() <= delta)


def train_learned_model(H, stream):
    """The learned order's model, trained (untimed) on the seeded training set."""
    import synth
    t0 = time.perf_counter()
    train = synth.training_graphs(LEARN_TRAIN_GRAPHS, 100, sizes=LEARN_TRAIN_SIZES)
    model, losses = H.train_model(train, OMEGA, DELTA, seed=0, per_node=LEARN_PER_NODE,
                                  steps=LEARN_STEPS, batch=LEARN_BATCH, lr=LEARN_LR,
                                  key_bits=LEARN_KEY_BITS, init_params=synth.initial_params(0),
                                  stream=stream)
    pairs = LEARN_PER_NODE * sum(t.num_nodes for t in train)
    return model, losses, time.perf_counter() - t0, pairs


def learned_leg(args, timed, g, d_ids, plain_cost, plain_ms, H, stream):
    """Learned candidate order: train on seeded graphs of the same family
    (untimed), then time partitions of the workload with the trained model.
    Returns (report, model)."""
    import torch
    model, losses, train_s, pairs = train_learned_model(H, stream)
    if args.save_model:
        np.savez(args.save_model, w1=model.w1, b1=model.b1, w2=model.w2, b2=model.b2,
                 key_bits=model.key_bits)
    timed(model=model)
    torch.cuda.synchronize()
    runs = [timed(model=model) for _ in range(max(1, min(args.steps, 3)))]
    times = [r[0] for r in runs]
    res = runs[-1][1]
    stats = [timed(H.HGP_DEBUG_TIMING, model=model)[2] for _ in range(INSTRUMENTED_STEPS)]
    ms = statistics.median(times)
    ids = d_ids.cpu().numpy()
    cost, feasible = recount(g, ids, OMEGA, DELTA)
    # the same model with the hidden layer on tensor cores (learned_eval = 1)
    timed(model=model, learned_eval=1)
    truns = [timed(model=model, learned_eval=1) for _ in range(max(1, min(args.steps, 3)))]
    tms = statistics.median(r[0] for r in truns)
    tres = truns[-1][1]
    tcost, tfeas = recount(g, d_ids.cpu().numpy(), OMEGA, DELTA)
    tstats = [timed(H.HGP_DEBUG_TIMING, model=model, learned_eval=1)[2]
              for _ in range(INSTRUMENTED_STEPS)]
    tsc = sum(s["ms_score"] for s in tstats) / len(tstats)
    tensor = {"learned_eval": 1, "ms_per_step": tms, "pins_per_s": g.num_pins / (tms / 1000.0),
              "levels": tres[2], "cost": tres[0], "cost_recounted": tcost, "feasible": tfeas,
              "cost_ratio_vs_plain": tres[0] / plain_cost, "time_ratio_vs_plain": tms / plain_ms,
              "score_ms_per_step": tsc,
              "note": "hidden layer by mma.sync m16n8k8 (TF32 in, FP32 accumulate) over each warp's "
                      "32 queued candidates; scores agree with FP32 to ~1e-3, so the partition may "
                      "differ from the FMA-chain order's"}
    # the learned scorer's FP32 roofline: 1,152 FLOP per network evaluation
    # (64 x 8 + 64 FMA) against 152 SMs x 128 FP32 lanes x 2 FLOP x the SM clock
    sc_ms = sum(s["ms_score"] for s in stats)
    evals = sum(s["learned_evals"] for s in stats)
    flops = 1152.0 * evals
    peak_tflops = 152 * 128 * 2 * LEARN_SM_GHZ / 1000.0
    achieved = flops / (sc_ms / 1000.0) / 1e12 if sc_ms > 0 else 0.0
    return {"model": f"8-64-1 MLP, bfloat16 weights, key_bits {LEARN_KEY_BITS}",
            "training": {"graphs": f"{LEARN_TRAIN_GRAPHS} random SNN hypergraphs of "
                                   f"{'/'.join(str(x) for x in LEARN_TRAIN_SIZES)} nodes (cycling), "
                                   f"hyperedge size 128..256, seeds 100..{99 + LEARN_TRAIN_GRAPHS}",
                         "labels": "co-location in the plain partition", "pairs": pairs,
                         "steps": LEARN_STEPS, "batch": LEARN_BATCH, "seconds": train_s,
                         "loss_first": float(losses[:20].mean()), "loss_last": float(losses[-20:].mean())},
            "ms_per_step": ms, "pins_per_s": g.num_pins / (ms / 1000.0),
            "timing": "uninstrumented steps; split and roofline from separate instrumented steps",
            "coarsen_ms": statistics.median(s["ms_coarsen"] for s in stats),
            "coarsening_pins_per_s": g.num_pins / (statistics.median(s["ms_coarsen"] for s in stats) / 1000.0),
            "levels": stats[-1]["num_levels"], "cost": res[0], "num_parts": res[1],
            "cost_recounted": cost, "feasible": feasible,
            "cost_ratio_vs_plain": res[0] / plain_cost, "time_ratio_vs_plain": ms / plain_ms,
            "steps": len(times), "tensor_cores": tensor,
            "roofline": {"kernel": "k_score_learned (network-ranked scoring)", "bound": "alu",
                         "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved / peak_tflops, "traffic": None,
                         "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz",
                         "evals_per_step": evals / len(stats),
                         "score_ms_per_step": sc_ms / len(stats),
                         "hbm_achieved_gbs": (sum(s["score_bytes"] for s in stats) / 1e9) / (sc_ms / 1000.0)
                         if sc_ms > 0 else 0.0}}, model


LEARNED_LARGE = {
    "learned256k": ("learned candidate order on a random SNN hypergraph, 262,144 nodes, one "
                    "hyperedge per node of 256 pins, 67,108,864 pins, int32 CSR, Omega=2^10, "
                    "Delta=2^12, seed 0; model trained on 16 seeded 16k-64k-node graphs",
                    "snn_256k", 1 << 10, 1 << 12),
    "learnedconv200k": ("learned candidate order on a layered conv-style SNN hypergraph, 8 layers x "
                        "16x16 x 100 channels (204,800 nodes), 3x3 windows on 88..100 channels, "
                        "~1.4e8 pins, int32 CSR, Omega=2^12, Delta=2^16, seed 0; model trained on 16 "
                        "seeded 16k-64k-node random SNN graphs", "conv_200k", 1 << 12, 1 << 16),
}


def run_learned_large(args, rank, world):
    """The learned order on a large workload: train (untimed), then time whole
    partitions (create + partition + destroy, device-resident inputs)."""
    import torch
    import synth
    from paper_2604_14411_gb300 import hgp as H
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    H.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    model, losses, train_s, _ = train_learned_model(H, stream)
    desc, make, omega, delta = LEARNED_LARGE[args.workload]
    g = getattr(synth, make)(0)
    N, P = g.num_nodes, g.num_pins
    d_off = torch.from_numpy(g.offsets.copy()).to(dev)
    d_pins = torch.from_numpy(g.pins.copy()).to(dev)
    d_ids = torch.empty(N, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(debug=0):
        h = H.hgp_create(N, d_off, d_pins, stream=stream)
        try:
            res = H.hgp_partition(h, omega, delta, d_ids, None, None, 1, debug, 0, model)
            st = H.hgp_get_stats(h)
        finally:
            H.hgp_destroy(h)
        return res, st

    warm = 1 if args.warmup >= 1 else 0
    for _ in range(warm):
        step()
    sampler = ClockSampler(clocks_path(args, rank))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    times, stats, res = [], [], None
    for _ in range(args.steps):
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res, st = step(H.HGP_DEBUG_TIMING)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
        stats.append(st)
    torch.cuda.synchronize()
    clocks = sampler.stop(local)
    job = job_time_ms(sum(times), dist, dev)
    ids = d_ids.cpu().numpy()
    cost, feasible = recount(g, ids, omega, delta)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": job_value(P, args.steps, world, job), "unit": "pins/s",
            "n_gpus": world, "steps": args.steps, "warmup": warm, "ms_per_step": job / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": desc, "omega": omega, "delta": delta, "pins": P,
                       "l2": "flushed between timed steps (256 MB write)"},
            "coarsen_ms": statistics.median(s["ms_coarsen"] for s in stats),
            "coarsening_pins_per_s": P / (statistics.median(s["ms_coarsen"] for s in stats) / 1000.0),
            "refine_ms": statistics.median(s["ms_refine"] for s in stats),
            "score_ms": statistics.median(s["ms_score"] for s in stats),
            "levels": stats[-1]["num_levels"], "cost": res[0], "num_parts": res[1],
            "cost_recounted": cost, "feasible": feasible,
            "training_seconds": train_s, "loss_last": float(losses[-20:].mean()),
            "gpu_launches": int(stats[-1]["kernel_launches"] + stats[-1]["create_launches"]) * args.steps,
            "clocks": clocks}), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def profile_large(levels):
    """One plain partition of the 262k SNN cut after `levels` levels."""
    import torch
    import synth
    from paper_2604_14411_gb300 import hgp as H
    H.load()
    g = synth.snn_256k(0)
    dev = torch.device("cuda", 0)
    d_off = torch.from_numpy(g.offsets.copy()).to(dev)
    d_pins = torch.from_numpy(g.pins.copy()).to(dev)
    d_ids = torch.empty(g.num_nodes, dtype=torch.int32, device=dev)
    h = H.hgp_create(g.num_nodes, d_off, d_pins)
    try:
        res = H.hgp_partition(h, 1 << 10, 1 << 12, d_ids, None, None, 1, 0, levels)
    finally:
        H.hgp_destroy(h)
    torch.cuda.synchronize()
    print(json.dumps({"profile_large": True, "levels": res[2], "cost": res[0], "parts": res[1]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="snn16k",
                    choices=["snn16k", "batch64", "learned256k", "learnedconv200k"],
                    help="snn16k: the default single-hypergraph workload; batch64: 64 uneven "
                         "hypergraphs through hgp_partition_batch; learned256k / learnedconv200k: "
                         "the learned order on the 262,144-node SNN / the 204,800-node conv-style "
                         "SNN (these print their own JSON line)")
    ap.add_argument("--clocks-dir", default=None,
                    help="directory for the clock samples of the timed region (default: temp dir)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-order leg (training + timed learned partitions)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the whole plain and learned partitions of the 262,144-node SNN")
    ap.add_argument("--save-model", default=None,
                    help="write the learned leg's trained model to this .npz file")
    ap.add_argument("--learned-model", default=None,
                    help="with --profile-step: profile one step with this saved model")
    ap.add_argument("--profile-step", action="store_true",
                    help="warm up, run exactly one step, exit (for ncu launch lists)")
    ap.add_argument("--profile-large", type=int, default=0, metavar="LEVELS",
                    help="one plain partition of the 262,144-node SNN cut after LEVELS "
                         "coarsening levels, then exit (for ncu captures of its large levels)")
    args = ap.parse_args()
    if args.warmup < 3 and not args.profile_step:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.profile_large:
        return profile_large(args.profile_large)
    if args.workload == "batch64":
        return run_batch(args, rank, world)
    if args.workload in ("learned256k", "learnedconv200k"):
        return run_learned_large(args, rank, world)

    import torch
    import synth
    from paper_2604_14411_gb300 import hgp as H

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    H.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    g = synth.snn_16k(0)
    P = g.num_pins
    N = g.num_nodes
    d_off = torch.from_numpy(g.offsets.copy()).to(dev)
    d_pins = torch.from_numpy(g.pins.copy()).to(dev)
    d_ids = torch.empty(N, dtype=torch.int32, device=dev)
    d_pw = torch.empty(N, dtype=torch.int64, device=dev)
    d_pin = torch.empty(N, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > 129 MB L2

    def step(debug=0, model=None, max_levels=0, learned_eval=0):
        h = H.hgp_create(N, d_off, d_pins, stream=stream)
        try:
            res = H.hgp_partition(h, OMEGA, DELTA, d_ids, d_pw, d_pin, 1, debug, max_levels, model,
                                  learned_eval=learned_eval)
            st = H.hgp_get_stats(h)
        finally:
            H.hgp_destroy(h)
        return res, st

    def timed(debug=0, model=None, max_levels=0, learned_eval=0):
        """One step between CUDA events on the library's stream, L2 flushed first."""
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res, st = step(debug, model, max_levels, learned_eval)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b), res, st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if args.profile_step:
        model = None
        if args.learned_model:
            z = np.load(args.learned_model)
            model = H.Model(z["w1"], z["b1"], z["w2"], int(z["b2"]), int(z["key_bits"]))
        res, st = step(model=model)
        torch.cuda.synchronize()
        print(json.dumps({"profile_step": True, "levels": st["num_levels"], "cost": res[0],
                          "launches": st["kernel_launches"] + st["create_launches"]}))
        return

    # ---- timed region: K whole steps, no instrumentation inside ----
    sampler = ClockSampler(clocks_path(args, rank))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    times, stats, res = [], [], None
    for _ in range(args.steps):
        ms, res, st = timed()
        times.append(ms)
        stats.append(st)
    torch.cuda.synchronize()
    clocks = sampler.stop(local)
    if dist:
        dist.barrier()
    t_total = job_time_ms(sum(times), dist, dev)
    ms_per_step = t_total / args.steps
    value = job_value(P, args.steps, world, t_total)

    # ---- per-kernel split: separate steps with CUDA events around every phase ----
    inst = [timed(H.HGP_DEBUG_TIMING) for _ in range(INSTRUMENTED_STEPS)]
    istats = [x[2] for x in inst]

    # end to end through the C ABI with pinned host buffers
    h_off = torch.from_numpy(g.offsets.copy()).pin_memory()
    h_pins = torch.from_numpy(g.pins.copy()).pin_memory()
    h_ids = torch.empty(N, dtype=torch.int32).pin_memory()
    h_pw = torch.empty(N, dtype=torch.int64).pin_memory()
    h_pin = torch.empty(N, dtype=torch.int32).pin_memory()
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = H.hgp_create(N, h_off.numpy(), h_pins.numpy(), stream=stream)
        try:
            cost, nparts, _ = H.hgp_partition(h, OMEGA, DELTA, h_ids.numpy(), h_pw.numpy(), h_pin.numpy())
        finally:
            H.hgp_destroy(h)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_value = P * world * len(e2e_times) / sum(e2e_times)
    h2d = g.offsets.nbytes + g.pins.nbytes
    d2h = h_ids.numel() * 4 + nparts * 8 + nparts * 4 + 8 + 4

    learned, model = None, None
    if not args.no_learned:
        learned, model = learned_leg(args, timed, g, d_ids, res[0], statistics.median(times), H, stream)
    # quality floor: the constraint-only comparison (parts filled in node-id order)
    with H.Graph(N, d_off, d_pins, stream=stream) as G:
        fill = G.fill_baseline(OMEGA, DELTA)
    quality = {"fill_baseline_cost": fill.cost, "fill_baseline_parts": fill.num_parts,
               "plain_cost_vs_fill": res[0] / fill.cost}
    if learned is not None:
        quality["learned_cost_vs_fill"] = learned["cost"] / fill.cost

    # the CPU baseline's sample on the GPU: the same cut prefix of the method
    cut_ms = statistics.median(timed(max_levels=CUT_LEVELS)[0] for _ in range(5))

    st = istats[-1]
    peak, peak_kind = load_peaks()
    # roofline of the kernel with the largest summed device time in the instrumented steps
    kern = {
        "k_score": ("Eq. 2 scoring with deferred Omega/Delta checks",
                    sum(s["ms_score"] for s in istats), sum(s["score_launches"] for s in istats),
                    sum(s["score_bytes"] for s in istats)),
        "k_propose": ("Eq. 3 in-isolation move proposals",
                      sum(s["ms_propose"] for s in istats), sum(s["propose_launches"] for s in istats),
                      sum(s["propose_bytes"] for s in istats)),
    }
    top = max(kern, key=lambda k: kern[k][1])
    desc, ms_k, n_k, bytes_k = kern[top]
    achieved = (bytes_k / 1e9) / (ms_k / 1000.0) if ms_k > 0 else 0.0
    launches = int(stats[-1]["kernel_launches"] + stats[-1]["create_launches"])
    inst_ms = sum(x[0] for x in inst)

    large = None
    if not args.no_large:
        del flush
        torch.cuda.empty_cache()
        large = large_leg(model, stream, H, peak)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pins/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "omega": OMEGA, "delta": DELTA, "pins": P,
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "partition_ms": statistics.median(s["ms_partition"] for s in stats),
            "levels": stats[-1]["num_levels"], "cost": res[0], "num_parts": res[1],
            "gpu_launches": launches * args.steps,
            "instrumented": {"steps": len(inst), "ms_per_step": inst_ms / len(inst),
                             "note": "separate steps with CUDA events around every phase; the "
                                     "split and the roofline below come from these"},
            "coarsen_ms": statistics.median(s["ms_coarsen"] for s in istats),
            "coarsening_pins_per_s": P / (statistics.median(s["ms_coarsen"] for s in istats) / 1000.0),
            "refine_ms": statistics.median(s["ms_refine"] for s in istats),
            "e2e": {"value": e2e_value, "unit": "pins/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "roofline": {"kernel": f"{top} ({desc})", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": measured_traffic(top),
                         "peak_kind": f"{peak_kind} (hbm copy)",
                         "launches": int(n_k), "avg_launch_us": 1000.0 * ms_k / max(n_k, 1),
                         "bytes_per_launch": bytes_k / max(n_k, 1),
                         "share_of_step": ms_k / inst_ms},
            "contraction_roofline": contraction_roofline(istats, peak, peak_kind, "16k SNN, all levels"),
            "kernel_ms_per_step": {k: v[1] / len(istats) for k, v in kern.items()},
            "clocks": clocks,
        }
        if learned is not None:
            line["learned"] = learned
        line["quality"] = quality
        if large is not None:
            line["snn256k"] = large
        if not args.no_cpu_baseline:
            v, ts = oracle_sample(steps=3)
            gpu_cut = P / (cut_ms / 1000.0)
            line["cpu_baseline"] = {"value": v, "unit": "pins/s", "cores": 1, "kind": "oracle",
                                    "sample": SAMPLE_DESC + f"; median of {len(ts)} runs",
                                    "gpu_same_sample": {"value": gpu_cut, "unit": "pins/s",
                                                        "ms": cut_ms, "ratio_vs_oracle": gpu_cut / v}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def contraction_roofline(stats, peak, peak_kind, where):
    """Contraction kernels (count and write phases, without the host read in
    between) against the HBM copy peak, from HGP_DEBUG_TIMING steps."""
    ms = sum(s["ms_contract_kernels"] for s in stats)
    by = sum(s["contract_bytes"] for s in stats)
    ach = (by / 1e9) / (ms / 1000.0) if ms > 0 else 0.0
    return {"kernels": "k_coarse_nodes, k_carry, k_union_count, k_union_merged, k_coarse_pins, "
                       "k_union_copy, k_coarse_src + offset scans", "where": where, "bound": "hbm",
            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_kind": f"{peak_kind} (hbm copy)", "ms": ms / len(stats),
            "bytes": by / len(stats), "traffic": None}


def large_leg(model, stream, H, peak):
    """Whole partitions of the 262,144-node SNN (67 M pins): the plain order
    and the learned one with the model trained above, each once, L2 flushed,
    with phase events on (for the contraction roofline at these sizes)."""
    import torch
    import synth
    g = synth.snn_256k(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    d_off = torch.from_numpy(g.offsets.copy()).to(dev)
    d_pins = torch.from_numpy(g.pins.copy()).to(dev)
    d_ids = torch.empty(g.num_nodes, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = {"workload": "random SNN hypergraph, 262,144 nodes, one hyperedge per node of 256 pins, "
                       "67,108,864 pins, int32 CSR, Omega=2^10, Delta=2^12, seed 0",
           "timing": "one whole create + partition + destroy each, CUDA events on the library's "
                     "stream, L2 flushed before, phase events on"}
    legs = [("plain", None, 0)] + ([("learned", model, 0), ("learned_tensor_cores", model, 1)]
                                   if model is not None else [])
    for name, m, tc in legs:
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        alloc = H.TorchAllocator()
        a.record(stream)
        h = H.hgp_create(g.num_nodes, d_off, d_pins, stream=stream, allocator=alloc)
        try:
            res = H.hgp_partition(h, 1 << 10, 1 << 12, d_ids, None, None, 1, H.HGP_DEBUG_TIMING, 0, m,
                                  learned_eval=tc)
            st = H.hgp_get_stats(h)
        finally:
            H.hgp_destroy(h)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        cost, feas = recount(g, d_ids.cpu().numpy(), 1 << 10, 1 << 12)
        out[name] = {"ms": ms, "pins_per_s": g.num_pins / (ms / 1000.0), "levels": res[2],
                     "cost": res[0], "num_parts": res[1], "cost_recounted": cost, "feasible": feas,
                     "coarsen_ms": st["ms_coarsen"], "refine_ms": st["ms_refine"],
                     "score_ms": st["ms_score"], "peak_device_gb": alloc.peak_bytes / 1e9}
        if name == "plain":
            out["contraction_roofline"] = contraction_roofline([st], peak, load_peaks()[1],
                                                               "262k SNN, all 201 levels")
    for name in ("learned", "learned_tensor_cores"):
        if name in out:
            out[name]["cost_ratio_vs_plain"] = out[name]["cost"] / out["plain"]["cost"]
            out[name]["time_ratio_vs_plain"] = out[name]["ms"] / out["plain"]["ms"]
    del d_off, d_pins, d_ids, flush
    torch.cuda.empty_cache()
    return out

if __name__ == "__main__":
    main()
