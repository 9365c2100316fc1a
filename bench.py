#!/usr/bin/env python3
"""Benchmark of the SdBG construction path on synthetic reads.

One step = the whole path on one read set: mh_pack_reads (from reads already
in HBM), mh_count_kmers, mh_mercy_kmers, mh_build_sdbg.  The default
workload is the simulated metagenome: 100 random genomes (lognormal lengths,
median 2 Mbp; lognormal abundances), 10 M read pairs of 2 x 150 bp (3.0 Gbp),
substitution rate rising to 1% at the 3' end, k = 31, d = 2.

value       (k+1)-mers counted per second: |K| (every (k+1)-mer on both
            strands) of all ranks' read sets / max-over-ranks step time
e2e         the same through the C ABI from pinned host buffers, with the
            read upload and the download of the SdBG arrays in the timed region
roofline    the radix scatter pass (the dominant kernel): algorithmic bytes
            (2 x key bytes per key, + 2 x 4 for a payload) / its CUDA-event
            time, against the measured HBM copy bandwidth
cpu_baseline  the CPU oracle, single thread, on the first 24,000 reads

``--impl reference`` times the CPU oracle alone (rank 0) on that sample.
Multi-GPU (torchrun): every rank builds its own independent read set (seed +
rank), so per-GPU work is fixed (weak scaling); there is no collective on the
data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "(k+1)-mers sorted+counted/s and SdBG edges built/s, % of HBM peak; served p50/p99"
UNIT = "(k+1)-mers/s"
CPU_SAMPLE_READS = 24_000

WORKLOADS = {
    "metagenome": {
        "name": "simulated metagenome: 100 genomes (lognormal lengths, median 2 Mbp, sigma 0.5; "
                "lognormal abundances, sigma 1.5), 10M pairs 2x150 bp, 3' error ramp to 1% (mean 0.5%), "
                "k=31, d=2, mercy on",
        "k": 31, "d": 2, "seed": 2,
        "gen": lambda seed, pairs=10_000_000: __import__("synth").metagenome_reads(seed=seed, n_pairs=pairs),
        "sample": lambda seed, n: __import__("synth").metagenome_reads(seed=seed, n_pairs=n // 2),
    },
    "outofcore": {
        "name": "out-of-core: the simulated metagenome at 100M pairs 2x150 bp (200M reads, 30 Gbp) held in "
                "pinned host memory, streamed to the device every step; keys counted in buckets of their "
                "top bits under the device-memory plan, k=31, d=2, mercy on",
        "k": 31, "d": 2, "seed": 4, "host_input": True, "pairs": 100_000_000, "pool": True,
        "gen": lambda seed, pairs=100_000_000, out=None: __import__("synth").metagenome_reads(
            seed=seed, n_pairs=pairs, out=out),
        "sample": lambda seed, n: __import__("synth").metagenome_reads(seed=seed, n_pairs=n // 2),
    },
    "plain": {
        "name": "plain single job: uniform 50 kbp genome, 10,000 x 100 bp single-end reads, 1% errors, "
                "k=21, d=2, mercy on",
        "k": 21, "d": 2, "seed": 1,
        "gen": lambda seed, pairs=None: __import__("synth").uniform_genome_reads(seed=seed),
        "sample": lambda seed, n: __import__("synth").uniform_genome_reads(seed=seed, n_reads=min(n, 10_000)),
    },
}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="metagenome",
                   choices=sorted(WORKLOADS) + ["multik", "served", "batched"])
    p.add_argument("--e2e-steps", type=int, default=12)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the bounded served and batched runs the default metagenome line carries")
    p.add_argument("--workers", type=int, default=None, help="worker streams of the batched workload (4)")
    p.add_argument("--torch-alloc", action="store_true",
                   help="library buffers from torch's caching allocator in every workload")
    p.add_argument("--pairs", type=int, default=None,
                   help="read pairs (default: 10M for metagenome, 20M for multik; smaller values: "
                        "profiling and test cases only)")
    return p.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic_record():
    """ncu DRAM bytes per key of the scatter pass, if recorded for the current
    kernel source."""
    path = os.path.join(ROOT, "profiles", "radix_onesweep_traffic.json")
    try:
        rec = json.load(open(path))
        return rec if rec.get("sources_sha256") == sort_sources_sha() else None
    except Exception:
        return None


def sort_sources_sha() -> str:
    """sha256 of the scatter pass's kernel source (mh_sort_kernels.cuh)."""
    h = hashlib.sha256()
    h.update(open(os.path.join(ROOT, "paper_1409_7208_gb300", "csrc", "mh_sort_kernels.cuh"), "rb").read())
    return h.hexdigest()


class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        self.proc = None
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        self.index = vis.split(",")[local_rank] if vis else str(local_rank)
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.index, "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for name, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def job_totals(dist, device, kmers: int, edges: int, ms: float, e2e_s: float = 0.0) -> dict:
    """Whole-job figures over all ranks: (k+1)-mers and SdBG entries are
    summed, the timed durations take the maximum over ranks (a job ends when
    its slowest rank does).  With dist None (one process) the local figures
    are returned as they are."""
    if dist is None:
        return {"kmers": kmers, "edges": edges, "ms": ms, "e2e_s": e2e_s}
    import torch
    sums = torch.tensor([float(kmers), float(edges)], dtype=torch.float64, device=device)
    maxs = torch.tensor([ms, e2e_s], dtype=torch.float64, device=device)
    dist.all_reduce(sums, op=dist.ReduceOp.SUM)
    dist.all_reduce(maxs, op=dist.ReduceOp.MAX)
    return {"kmers": int(sums[0].item()), "edges": int(sums[1].item()), "ms": float(maxs[0].item()),
            "e2e_s": float(maxs[1].item())}


def cpu_oracle_run(ascii, offs, k, d, threads=1):
    import oracle
    t0 = time.perf_counter()
    r = oracle.count(ascii, offs, k, d, mercy=True, threads=threads)
    oracle.build_sdbg(k, r["solid_keys"], r["solid_cnt"], r["mercy_keys"], r["mercy_cnt"])
    return r["n_kmers"], time.perf_counter() - t0


def _host_cpu():
    """(cores, model) of the host the oracle runs on."""
    n = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return n, model or "unknown"


def cpu_baseline_pair(ascii, offs, k, d, sample):
    """The oracle on the sample on every host core (counting split by prefix,
    mercy by fragment; the SdBG build one thread) and on one core."""
    n_cores, model = _host_cpu()
    n1, t1 = cpu_oracle_run(ascii, offs, k, d, 1)
    nn, tn = cpu_oracle_run(ascii, offs, k, d, n_cores)
    return {"value": nn / tn, "unit": UNIT, "cores": n_cores, "kind": "oracle", "sample": sample,
            "seconds": tn, "one_thread": {"value": n1 / t1, "cores": 1, "seconds": t1},
            "nproc": n_cores, "cpu_model": model,
            "note": "value: counting and mercy on every core, the SdBG build on one"}


def run_reference(args, wl, rank, world):
    """The CPU oracle as it stands, on the bounded sample: counting and mercy
    split over every host core (the threaded form, equal to the one-thread
    oracle by test), the SdBG build on one."""
    if rank != 0:
        return
    ascii, offs = wl["sample"](wl["seed"], CPU_SAMPLE_READS)
    n_cores, model = _host_cpu()
    for _ in range(args.warmup):
        cpu_oracle_run(ascii, offs, wl["k"], wl["d"], n_cores)
    total_n, total_t = 0, 0.0
    for _ in range(args.steps):
        n, t = cpu_oracle_run(ascii, offs, wl["k"], wl["d"], n_cores)
        total_n += n
        total_t += t
    v = total_n / total_t
    sample = ("first %d reads of the workload (%d (k+1)-mers on both strands); counting and mercy on %d "
              "threads (%s), the SdBG build on one" % (len(offs) - 1, n, n_cores, model))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": wl["name"], "k": wl["k"], "d": wl["d"],
                                            "sample_reads": len(offs) - 1},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": n_cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


MULTIK = {
    "name": "multiple-k iteration: uniform genome at 20x (200 Mbp for 20M pairs), read pairs as single-end "
            "100 bp reads, 1% iid errors, k in {27,47,67,87,99}, d=2; per k 16384 contig walks of <= 10 kbp, "
            "carried into the next k as d copies each",
    "ks": (27, 47, 67, 87, 99), "d": 2, "seed": 3, "walks": 16384, "max_len": 10_000,
}


def _multik_reads(seed, pairs):
    import synth
    n_reads = 2 * pairs
    return synth.uniform_genome_reads(seed, n_reads * 100 // 20, n_reads, 100, 0.01)


def _multik_oracle(ascii, offs):
    from oracle import walk as ow
    t0 = time.perf_counter()
    steps = ow.iterate(ascii, offs, MULTIK["ks"], MULTIK["d"], 64, 500, MULTIK["seed"])
    return sum(st["counts"]["n_kmers"] for st in steps), time.perf_counter() - t0


def run_multik(args, rank, world, local):
    """One step = the whole iteration over MULTIK's k list (count, mercy, SdBG
    and contig walks per k); value = (k+1)-mers of all k per second."""
    import numpy as np
    import torch

    import paper_1409_7208_gb300 as mh
    from paper_1409_7208_gb300 import multik

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pairs = args.pairs or 20_000_000
    ascii, offs = _multik_reads(MULTIK["seed"] + 1000 * rank, pairs)
    # one stream for torch and the library: the launching stream of every
    # kernel, on which every timing event is recorded
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = mh.Context(device=local, stream=stream)
    d_ascii = torch.from_numpy(ascii).cuda()
    d_offs = torch.from_numpy(offs.view(np.int64)).cuda()
    ks, d = MULTIK["ks"], MULTIK["d"]

    def step(a, o):
        return multik.iterate(ctx, a, o, ks, d, MULTIK["walks"], MULTIK["max_len"], MULTIK["seed"])

    for _ in range(args.warmup):
        sizes = step(d_ascii, d_offs)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    ctx.profile_reset()
    ctx.set_profile(True)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        sizes = step(d_ascii, d_offs)
    t1.record(stream)
    torch.cuda.synchronize()
    ctx.set_profile(False)
    clk = clocks.stop()
    n_kmers = sum(st["n_kmers"] for st in sizes)
    n_edges = sum(st["m"] for st in sizes)
    tot = job_totals(dist, "cuda", n_kmers, n_edges, t0.elapsed_time(t1))
    ms = tot["ms"]
    prof = ctx.profile()
    e2e = None
    if args.e2e_steps > 0:
        pin_a = torch.from_numpy(ascii).pin_memory()
        pin_o = torch.from_numpy(offs.view(np.int64)).pin_memory()
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            a = pin_a.to("cuda", non_blocking=True)
            o = pin_o.to("cuda", non_blocking=True)
            res = multik.iterate(ctx, a, o, ks, d, MULTIK["walks"], MULTIK["max_len"], MULTIK["seed"],
                                 keep=False)
            torch.cuda.synchronize()
        e_s = job_totals(dist, "cuda", n_kmers, n_edges, 0.0, time.perf_counter() - e0)["e2e_s"]
        e2e = {"value": tot["kmers"] * args.e2e_steps / e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(ascii.nbytes + offs.nbytes),
               "d2h_bytes_per_step": 8 * 7 * len(res),
               "note": "the per-k sizes come back to the host; the graphs stay on the device"}
    peak, peak_kind = _peak_hbm()
    launches, o_ms, o_bytes = prof.get("radix_onesweep", (0, 0.0, 0))
    achieved = o_bytes / (o_ms / 1e3) / 1e9 if o_ms > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": "radix_onesweep", "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "launches": launches}
    kernels = {name: {"launches": la, "ms_per_step": t / args.steps}
               for name, (la, t, b) in sorted(prof.items(), key=lambda kv: -kv[1][1])[:12]}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        sa, so = _multik_reads(MULTIK["seed"], 2000)
        n_s, t_s = _multik_oracle(sa, so)
        cpu = {"value": n_s / t_s, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "4000 reads of the generator (genome 20 kbp), walks 64 x <= 500 bp, %d (k+1)-mers "
                         "over the k list, %.1f s" % (n_s, t_s)}
    if rank == 0:
        line = {"metric": METRIC, "value": tot["kmers"] * args.steps / (ms / 1e3), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic",
                "config": {"workload": MULTIK["name"], "reads": len(offs) - 1, "bases": len(ascii),
                           "ks": list(ks), "d": d, "walks": MULTIK["walks"], "max_len": MULTIK["max_len"],
                           "l2": "inputs larger than L2 (%.1f GB of reads)" % (len(ascii) / 1e9)},
                "sdbg_edges_per_s": tot["edges"] * args.steps / (ms / 1e3),
                "per_k": sizes, "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": sum(la for (la, _, _) in prof.values()), "clocks": clk}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


BATCHED = {
    "name": "batched: 64 independent read sets, reads per set lognormal (ln-median halfway between 50k and 5M, "
            "sigma a quarter of that span) clipped to [50k, 5M], pairs of 2x150 bp, each set a 10-genome "
            "mini-metagenome (genomes lognormal, median 2 Mbp), 3' error ramp to 1% (mean 0.5%), k=31, d=2, "
            "mercy on; the whole batch through mh_run_batch on 4 worker streams, counting plan autotuned",
    "n_sets": 64, "k": 31, "d": 2, "seed": 5, "workers": 4,
}


def batched_figures(local, n_sets, steps, warmup, workers, seed=None):
    """The batched workload on `n_sets` sets: the whole path on every set
    through mh_run_batch (worker streams, largest set first, tile shape
    autotuned), against the same sets through the plain calls one after
    another on one stream.  Returns a dict of the figures."""
    import numpy as np
    import torch

    import paper_1409_7208_gb300 as mh
    import synth

    sets = synth.batch_sets(BATCHED["seed"] if seed is None else seed, n_sets)
    n_reads = sum(len(o) - 1 for _, o in sets)
    n_bases = sum(len(a) for a, _ in sets)
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = mh.Context(device=local, stream=stream, torch_allocator=False)
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(o.view(np.int64)).cuda()) for a, o in sets]
    torch.cuda.synchronize()
    k, d = BATCHED["k"], BATCHED["d"]
    info = {}

    def batched(inputs):
        res = mh.mh_run_batch(ctx, inputs, k, d, workers=workers, autotune=True)
        info["n_kmers"] = sum(r["solid"].view().n_kmers for r in res)
        info["m"] = sum(r["sdbg"].view().m for r in res)
        for r in res:
            for key in ("sdbg", "mercy", "solid"):
                r[key].free()

    def serial(inputs):
        for a, o in inputs:
            reads = mh.mh_pack_reads(ctx, a, o)
            solid = mh.mh_count_kmers(ctx, reads, k, d)
            mercy = mh.mh_mercy_kmers(ctx, reads, solid)
            g = mh.mh_build_sdbg(ctx, solid, mercy)
            del g, mercy, solid, reads

    def timed(fn, n):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(n):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / n

    for _ in range(warmup):
        batched(dev)
    serial(dev)
    ctx.profile_reset()
    ctx.set_profile(True)
    serial_ms = timed(lambda: serial(dev), 1)
    ctx.set_profile(False)
    prof_serial = ctx.profile()
    ctx.profile_reset()
    ctx.set_profile(True)
    ms = timed(lambda: batched(dev), steps)
    ctx.set_profile(False)
    prof = ctx.profile()
    out = {"sets": len(sets), "reads": n_reads, "bases": n_bases, "k": k, "d": d, "workers": workers,
           "sort_shape": mh.mh_sort_shape(ctx), "count_plan": mh.mh_get_count_plan(ctx), "ms": ms,
           "serial_ms": serial_ms,
           "kmers_per_s": info["n_kmers"] / (ms / 1e3), "serial_kmers_per_s": info["n_kmers"] / (serial_ms / 1e3),
           "jobs_per_s": len(sets) / (ms / 1e3), "serial_jobs_per_s": len(sets) / (serial_ms / 1e3),
           "batch_speedup": serial_ms / ms, "n_kmers": info["n_kmers"], "m": info["m"],
           "prof": prof, "prof_serial": prof_serial, "sets_data": sets, "ctx": ctx, "stream": stream,
           "dev": dev, "batched_fn": batched}
    return out


def run_batched(args, rank, world, local):
    """One step = the whole path on all 64 read sets through mh_run_batch
    (worker streams, largest set first); value = (k+1)-mers of all sets per
    second.  The same sets through the plain calls one after another on one
    stream are timed beside it (serial_value)."""
    import numpy as np
    import torch

    import paper_1409_7208_gb300 as mh

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = args.workers or BATCHED["workers"]
    clocks = Clocks(local)
    clocks.start()
    f = batched_figures(local, BATCHED["n_sets"], args.steps, args.warmup, W, BATCHED["seed"] + 1000 * rank)
    clk = clocks.stop()
    sets, ctx, stream, batched = f["sets_data"], f["ctx"], f["stream"], f["batched_fn"]
    n_reads, n_bases, k, d = f["reads"], f["bases"], f["k"], f["d"]
    prof, prof_serial = f["prof"], f["prof_serial"]
    tot = job_totals(dist, "cuda", f["n_kmers"], f["m"], f["ms"])
    ms = tot["ms"]
    value = tot["kmers"] / (ms / 1e3)

    e2e = None
    if args.e2e_steps > 0:
        pinned = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(o.view(np.int64)).pin_memory())
                  for a, o in sets]
        nbytes = {"d2h": 0}

        def download(g):
            t = g.tensors()
            with torch.cuda.stream(stream):
                for key in ("W", "last", "valid", "dummy", "aux"):
                    src = t[key]
                    buf = torch.empty(max(1, src.numel()), dtype=src.dtype, pin_memory=True)
                    if src.numel():
                        buf[: src.numel()].view(src.shape).copy_(src, non_blocking=True)
                    nbytes["d2h"] += src.numel() * src.element_size()
            stream.synchronize()

        def batched_dl(inputs):
            res = mh.mh_run_batch(ctx, inputs, k, d, workers=W, autotune=True)
            for r in res:
                download(r["sdbg"])
            for r in res:
                for key in ("sdbg", "mercy", "solid"):
                    r[key].free()

        batched_dl(pinned)
        torch.cuda.synchronize()
        nbytes["d2h"] = 0
        e0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            batched_dl(pinned)
        torch.cuda.synchronize()
        e_s = (time.perf_counter() - e0) / args.e2e_steps
        e2e = {"value": f["n_kmers"] / e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(n_bases + 8 * (n_reads + len(sets))),
               "d2h_bytes_per_step": int(nbytes["d2h"] / args.e2e_steps + 48 * len(sets))}

    peak, peak_kind = _peak_hbm()
    launches, o_ms, o_bytes = prof_serial.get("radix_onesweep", (0, 0.0, 0))
    achieved = o_bytes / (o_ms / 1e3) / 1e9 if o_ms > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": "radix_onesweep", "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "launches": launches,
                "note": "from the plain serial pass (kernels timed alone); in the batch, kernels of "
                        "several streams share the GPU and per-launch times overlap"}
    kernels = {name: {"launches": la, "ms_per_step": t / args.steps}
               for name, (la, t, b) in sorted(prof.items(), key=lambda kv: -kv[1][1])[:12]}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        sa, so = sets[0]
        ns = min(CPU_SAMPLE_READS, len(so) - 1)
        sa, so = sa[: int(so[ns])], so[: ns + 1]
        cpu = cpu_baseline_pair(sa, so, k, d, "first %d reads of set 0" % ns)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": BATCHED["name"], "sets": len(sets), "reads": n_reads, "bases": n_bases,
                           "k": k, "d": d, "workers": W, "count_plan": f["count_plan"],
                           "l2": "inputs larger than L2 (%.1f GB of reads)" % (n_bases / 1e9)},
                "serial_value": f["serial_kmers_per_s"], "serial_ms": f["serial_ms"],
                "batch_speedup": f["batch_speedup"],
                "sdbg_edges_per_s": tot["edges"] / (ms / 1e3),
                "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": sum(la for (la, _, _) in prof.values()) // args.steps * args.steps,
                "clocks": clk}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


SERVED = {
    "name": "served: Poisson arrivals (20/s) for 60 s of count+mercy+build jobs; reads per job lognormal "
            "(median 447k, sigma ln(2000)/4) clipped to [10k, 20M]; read length uniform 100-150 bp; k uniform "
            "over {21,31,41,61}; d=2; reads of each job from a uniform genome at 20x with 0.5% errors, drawn "
            "from a pool of 96 distinct read sets in pinned host memory; 4 slots under an HBM budget of 150 GB",
    "rate": 20.0, "secs": 60.0, "median": 447_000, "sigma": 1.9002, "lo": 10_000, "hi": 20_000_000,
    "ks": (21, 31, 41, 61), "slots": 4, "budget": 150 << 30, "seed": 5, "pool": 96,
}


def _served_pool(seed, size):
    """The distinct read sets the jobs draw from: sizes from the served
    distribution, each its own uniform genome at 20x, in pinned host memory."""
    import numpy as np
    import torch

    import synth
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(size):
        n = int(np.clip(rng.lognormal(np.log(SERVED["median"]), SERVED["sigma"]), SERVED["lo"], SERVED["hi"]))
        L = int(rng.integers(100, 151))
        ascii, offs = synth.uniform_genome_reads(int(rng.integers(1 << 30)), max(5000, n * L // 20), n, L, 0.005)
        pool.append((torch.from_numpy(ascii).pin_memory().numpy(), offs))
    return pool


def _served_jobs(pool, seed, secs):
    """Poisson arrivals over `secs` seconds; each job a pool read set (drawn
    uniformly) with k drawn uniformly."""
    import numpy as np

    from paper_1409_7208_gb300 import serve
    rng = np.random.default_rng(seed)
    t, jobs = 0.0, []
    while True:
        t += rng.exponential(1.0 / SERVED["rate"])
        if t > secs:
            break
        ascii, offs = pool[int(rng.integers(len(pool)))]
        k = int(rng.choice(SERVED["ks"]))
        j = serve.Job(ascii, offs, k, 2, tag=len(jobs))
        j.arrival = t
        jobs.append(j)
    return jobs


def _run_stream(jobs, srv, paced):
    """Submit jobs to the server at their arrival times (paced) or all at
    once; wait for all.  Returns (wall seconds, most bytes held)."""
    srv.reset_max()
    t0 = time.perf_counter()
    for j in jobs:
        if paced:
            dt = t0 + j.arrival - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
        srv.submit(j)
    for j in jobs:
        j.wait(3600)
    t1 = max(j.end_t for j in jobs)
    for j in jobs:
        j.release()
    return t1 - t0, srv.max_held


def _fresh(jobs):
    """The same jobs again, not yet submitted."""
    out = []
    for j in jobs:
        n = type(j)(j.ascii, j.offs, j.k, j.d, j.tag)
        n.arrival = getattr(j, "arrival", 0.0)
        out.append(n)
    return out


def served_figures(local, secs, pool_size, warmup, cpu_baseline):
    """The served workload: a Poisson stream over `secs` seconds of jobs drawn
    from a pool of `pool_size` read sets, submitted at their arrival times to
    the serving loop (4 slots, HBM budget); then the same jobs all queued at
    once on the 4 slots, and one at a time through the plain path (one slot).
    Returns a dict of the figures."""
    import numpy as np

    from paper_1409_7208_gb300 import serve
    t_gen = time.perf_counter()
    # the library's request server: 4 slots under the budget, and 1 slot for
    # the plain path one job at a time; both kept warm across the runs
    srv = serve.Server(slots=SERVED["slots"], hbm_budget=SERVED["budget"], device=local, auto_release=True)
    one = serve.Server(slots=1, hbm_budget=SERVED["budget"], device=local, auto_release=True)
    pool = _served_pool(SERVED["seed"], pool_size)
    t_gen = time.perf_counter() - t_gen
    warm = _served_jobs(pool, SERVED["seed"] + 100, 0.5)
    for _ in range(max(1, warmup)):
        _run_stream(_fresh(warm), srv, False)
        _run_stream(_fresh(warm), one, False)
    jobs = _served_jobs(pool, SERVED["seed"], secs)
    for c in srv.contexts:
        c.profile_reset()
        c.set_profile(True)
    wall, held = _run_stream(jobs, srv, True)
    for c in srv.contexts:
        c.set_profile(False)
    lat = np.array([j.latency for j in jobs]) * 1e3
    kmers = sum(2 * max(0, j.n_bases - j.n_reads * j.k) for j in jobs)
    prof = {}
    for c in srv.contexts:
        for name, (la, t, b) in c.profile().items():
            p = prof.setdefault(name, [0, 0.0, 0])
            p[0] += la
            p[1] += t
            p[2] += b
    # all jobs queued at once: on the 4 slots (overlapped), then one at a time
    # through the plain path (one slot)
    burst_wall, _ = _run_stream(_fresh(jobs), srv, False)
    serial_jobs = _fresh(jobs)
    serial_wall, _ = _run_stream(serial_jobs, one, False)
    svc = np.array([j.end_t - j.start_t for j in serial_jobs]) * 1e3
    cpu = None
    if cpu_baseline:
        small = sorted(jobs, key=lambda j: j.n_bases)[:3]
        t_c = 0.0
        for j in small:
            t_c += cpu_oracle_run(j.ascii, j.offs, j.k, j.d)[1]
        cpu = {"value": len(small) / t_c, "unit": "jobs/s", "cores": 1, "kind": "oracle",
               "sample": "the 3 smallest jobs of the stream (%d reads), %.1f s"
                         % (sum(j.n_reads for j in small), t_c)}
    srv.close()
    one.close()
    return {"secs": secs, "pool": pool_size, "jobs": len(jobs), "reads": int(sum(j.n_reads for j in jobs)),
            "bases": int(sum(j.n_bases for j in jobs)), "wall_s": wall, "jobs_per_s": len(jobs) / wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "kmers_per_s": kmers / wall, "max_held_bytes": int(held),
            "serial": {"jobs_per_s": len(jobs) / serial_wall, "service_p50_ms": float(np.percentile(svc, 50)),
                       "service_p99_ms": float(np.percentile(svc, 99))},
            "burst": {"jobs_per_s": len(jobs) / burst_wall, "slots": SERVED["slots"],
                      "vs_serial": serial_wall / burst_wall, "note": "every job of the stream queued at once"},
            "pool_generation_s": t_gen, "prof": prof, "cpu": cpu,
            "h2d_bytes": int(sum(j.n_bases + 8 * (j.n_reads + 1) for j in jobs))}


def run_served(args, rank, local):
    import torch

    if rank != 0:
        return
    torch.cuda.set_device(local)
    clocks = Clocks(local)
    clocks.start()
    f = served_figures(local, SERVED["secs"], SERVED["pool"], args.warmup, not args.no_cpu_baseline)
    clk = clocks.stop()
    prof = f["prof"]
    peak, peak_kind = _peak_hbm()
    la, o_ms, o_bytes = prof.get("radix_onesweep", (0, 0.0, 0))
    achieved = o_bytes / (o_ms / 1e3) / 1e9 if o_ms > 0 else 0.0
    line = {"metric": METRIC, "value": f["jobs_per_s"], "unit": "jobs/s", "n_gpus": 1, "steps": 1,
            "warmup": args.warmup, "ms_per_step": f["wall_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": SERVED["name"], "jobs": f["jobs"], "reads": f["reads"], "bases": f["bases"]},
            "p50_ms": f["p50_ms"], "p99_ms": f["p99_ms"], "kmers_per_s": f["kmers_per_s"],
            "max_held_bytes": f["max_held_bytes"], "serial": f["serial"], "burst": f["burst"],
            "roofline": {"bound": "hbm", "kernel": "radix_onesweep", "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                         "note": "concurrent launches on 4 streams: per-launch times overlap"},
            "cpu_baseline": f["cpu"],
            "e2e": {"value": f["jobs_per_s"], "unit": "jobs/s", "h2d_bytes_per_step": f["h2d_bytes"],
                    "d2h_bytes_per_step": 0,
                    "note": "reads come from host memory in every job; results stay resident until released"},
            "gpu_launches": int(sum(p[0] for p in prof.values())), "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    rank, world, local = _dist()
    if args.workload == "served":
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the served workload has no CPU arm: "
                                  "the oracle would take hours for its jobs"}), flush=True)
            return
        return run_served(args, rank, local)
    if args.workload == "batched":
        if args.impl == "reference":
            if rank == 0:
                import synth
                sa, so = synth.batch_sets(BATCHED["seed"], 1)[0]
                ns = min(CPU_SAMPLE_READS, len(so) - 1)
                sa, so = sa[: int(so[ns])], so[: ns + 1]
                n_cores, model = _host_cpu()
                for _ in range(args.warmup):
                    cpu_oracle_run(sa, so, BATCHED["k"], BATCHED["d"], n_cores)
                n_s = t_s = 0
                for _ in range(args.steps):
                    n, t = cpu_oracle_run(sa, so, BATCHED["k"], BATCHED["d"], n_cores)
                    n_s += n
                    t_s += t
                v = n_s / t_s
                print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
                                  "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                                  "ms_per_step": 1e3 * t_s / args.steps, "higher_is_better": True,
                                  "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                                  "config": {"workload": BATCHED["name"], "sample_reads": ns},
                                  "cpu_baseline": {"value": v, "unit": UNIT, "cores": n_cores, "kind": "oracle",
                                                   "sample": "first %d reads of set 0; counting and mercy on "
                                                             "%d threads (%s), the SdBG build on one"
                                                             % (ns, n_cores, model)},
                                  "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0}}), flush=True)
            return
        return run_batched(args, rank, world, local)
    if args.workload == "multik":
        if args.impl == "reference":
            if rank == 0:
                sa, so = _multik_reads(MULTIK["seed"], 2000)
                for _ in range(args.warmup):
                    _multik_oracle(sa, so)
                n_s = t_s = 0
                for _ in range(args.steps):
                    n, t = _multik_oracle(sa, so)
                    n_s += n
                    t_s += t
                v = n_s / t_s
                print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
                                  "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                                  "ms_per_step": 1e3 * t_s / args.steps, "higher_is_better": True,
                                  "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                                  "config": {"workload": MULTIK["name"], "sample_reads": len(so) - 1},
                                  "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                                   "sample": "4000 reads, walks 64 x <= 500 bp"},
                                  "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0}}), flush=True)
            return
        return run_multik(args, rank, world, local)
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl, rank, world)

    import numpy as np
    import torch

    import paper_1409_7208_gb300 as mh

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    k, d = wl["k"], wl["d"]
    host_input = wl.get("host_input", False)
    pairs = args.pairs or wl.get("pairs", 10_000_000)
    if host_input:
        # the reads live in pinned host memory and stream to the device in
        # every step (the library's staged upload overlaps the packing)
        pin_ascii = torch.empty(2 * pairs * 150, dtype=torch.uint8, pin_memory=True)
        ascii, offs = wl["gen"](wl["seed"] + 1000 * rank, pairs, out=pin_ascii.numpy())
        pin_offs = torch.from_numpy(offs.view(np.int64)).pin_memory()
    else:
        ascii, offs = wl["gen"](wl["seed"] + 1000 * rank, pairs)
    n_bases = len(ascii)
    # one stream for torch and the library: the launching stream of every
    # kernel, on which every timing event is recorded
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    # "pool": the library's own stream-ordered pool instead of torch's
    # caching allocator (at 180 GB of live buffers the caching allocator
    # falls back to freeing its cache in the middle of a step)
    ctx = mh.Context(device=local, stream=stream, torch_allocator=not (wl.get("pool") and not args.torch_alloc))
    if host_input:
        d_ascii, d_offs = pin_ascii, pin_offs
    else:
        d_ascii = torch.from_numpy(ascii).cuda()
        d_offs = torch.from_numpy(offs.view(np.int64)).cuda()
    torch.cuda.synchronize()

    info = {}

    def step(ascii_in, offs_in, phases=None, download=None):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)] if phases is not None else None
        if ev:
            ev[0].record(stream)
        reads = mh.mh_pack_reads(ctx, ascii_in, offs_in)
        if ev:
            ev[1].record(stream)
        solid = mh.mh_count_kmers(ctx, reads, k, d)
        if ev:
            ev[2].record(stream)
        mercy = mh.mh_mercy_kmers(ctx, reads, solid)
        if ev:
            ev[3].record(stream)
        g = mh.mh_build_sdbg(ctx, solid, mercy)
        if ev:
            ev[4].record(stream)
        sv, gv = solid.view(), g.view()
        info.update(n_kmers=sv.n_kmers, n_distinct=sv.n_distinct, solid=sv.n, mercy=mercy.view().n,
                    m=gv.m, t=gv.t, u=gv.u)
        if download is not None:
            download(g)
        if ev:
            phases.append(ev)
        del g, mercy, solid, reads

    for _ in range(args.warmup):
        step(d_ascii, d_offs)
    torch.cuda.synchronize()
    barrier()

    clocks = Clocks(local)
    clocks.start()
    ctx.profile_reset()
    ctx.set_profile(True)
    phases = []
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    t_start.record(stream)
    for _ in range(args.steps):
        step(d_ascii, d_offs, phases)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    ctx.set_profile(False)
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end)
    prof = ctx.profile()
    info["buckets"] = prof.get("extract_bucket", (0, 0, 0))[0] // args.steps or 1
    info["peak_GB"] = round(ctx.memory()[1] / 1e9, 1)
    tot = job_totals(dist, "cuda", info["n_kmers"], info["m"], ms)
    ms = tot["ms"]
    n_kmers = info["n_kmers"]
    value = tot["kmers"] * args.steps / (ms / 1e3)
    phase_ms = {name: sum(p[i].elapsed_time(p[i + 1]) for p in phases) / len(phases)
                for i, name in enumerate(["pack", "count", "mercy", "build"])}

    # end to end through host buffers: upload of the reads and download of the SdBG
    if not host_input:
        pin_ascii = torch.from_numpy(ascii).pin_memory()
        pin_offs = torch.from_numpy(offs.view(np.int64)).pin_memory()
    d2h = {"bytes": 0}
    host_bufs = {}

    def download(g, ev=None):
        t = g.tensors()
        nbytes = 0
        with torch.cuda.stream(stream):  # copies in order behind the library's work
            for key in ("W", "last", "valid", "dummy", "aux"):
                src = t[key]
                buf = host_bufs.get(key)
                if buf is None or buf.numel() < src.numel():
                    buf = torch.empty(max(1, src.numel()), dtype=src.dtype, pin_memory=True)
                    host_bufs[key] = buf
                if src.numel():
                    buf[: src.numel()].view(src.shape).copy_(src, non_blocking=True)
                nbytes += src.numel() * src.element_size()
        if ev is not None:
            ev.record(stream)
        stream.synchronize()
        d2h["bytes"] = nbytes + 48  # + F, returned by value

    e2e = None
    if args.e2e_steps > 0:
        step(pin_ascii, pin_offs, None, download)  # warm the host path
        torch.cuda.synchronize()
        barrier()
        h2d = int(n_bases + offs.nbytes)
        # one step with the library's own host-input path (mh_pack_reads from
        # pinned host memory: staged copy overlapped with the packing), timed
        # part by part
        h0 = time.perf_counter()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        reads = mh.mh_pack_reads(ctx, pin_ascii, pin_offs)
        ev[1].record(stream)
        solid = mh.mh_count_kmers(ctx, reads, k, d)
        mercy = mh.mh_mercy_kmers(ctx, reads, solid)
        g = mh.mh_build_sdbg(ctx, solid, mercy)
        ev[2].record(stream)
        download(g, ev[3])
        del g, mercy, solid, reads
        wall = 1e3 * (time.perf_counter() - h0)
        up, comp, down = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])
        serial = {"step_ms": wall, "upload_ms": up, "upload_GBps": h2d / (up / 1e3) / 1e9 if up else None,
                  "compute_ms": comp, "download_ms": down,
                  "download_GBps": d2h["bytes"] / (down / 1e3) / 1e9 if down else None,
                  "host_wait_ms": wall - ev[0].elapsed_time(ev[3])}
        # the timed end-to-end steps: each step's reads go up from pinned host
        # memory into one of two device buffers on a copy stream while the
        # step before computes (the first upload is not overlapped); then the
        # same calls on device pointers, and the SdBG arrays come back
        up_stream = torch.cuda.Stream(device=local)
        dbuf = [(torch.empty(n_bases, dtype=torch.uint8, device="cuda"),
                 torch.empty(offs.shape[0], dtype=torch.int64, device="cuda")) for _ in range(2)]
        up_done = [torch.cuda.Event() for _ in range(2)]
        buf_free = [torch.cuda.Event() for _ in range(2)]
        for e in buf_free:
            e.record(stream)

        def upload(i):
            with torch.cuda.stream(up_stream):
                up_stream.wait_event(buf_free[i % 2])
                dbuf[i % 2][0].copy_(pin_ascii, non_blocking=True)
                dbuf[i % 2][1].copy_(pin_offs, non_blocking=True)
                up_done[i % 2].record(up_stream)

        torch.cuda.synchronize()
        barrier()
        e0 = time.perf_counter()
        marks = []
        upload(0)
        for i in range(args.e2e_steps):
            marks.append(time.perf_counter())
            if i + 1 < args.e2e_steps:
                upload(i + 1)
            stream.wait_event(up_done[i % 2])
            reads = mh.mh_pack_reads(ctx, dbuf[i % 2][0], dbuf[i % 2][1])
            buf_free[i % 2].record(stream)
            solid = mh.mh_count_kmers(ctx, reads, k, d)
            mercy = mh.mh_mercy_kmers(ctx, reads, solid)
            g = mh.mh_build_sdbg(ctx, solid, mercy)
            download(g)
            del g, mercy, solid, reads
        torch.cuda.synchronize()
        marks.append(time.perf_counter())
        e_s = time.perf_counter() - e0
        e_tot = job_totals(dist, "cuda", info["n_kmers"], info["m"], 0.0, e_s)
        e_s = e_tot["e2e_s"]
        e2e = {"value": e_tot["kmers"] * args.e2e_steps / e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(d2h["bytes"]),
               "step_ms": 1e3 * e_s / args.e2e_steps,
               "upload_ms": serial["upload_ms"], "upload_GBps": serial["upload_GBps"],
               "download_ms": serial["download_ms"], "host_wait_ms": serial["host_wait_ms"],
               "how": "per step: the reads' upload from pinned host memory (overlapped with the previous "
                      "step's compute, the first one not), pack + count + mercy + build through the C ABI, "
                      "the SdBG arrays back to pinned host memory; upload/download/host-wait figures from "
                      "one further step through the library's host-input path, timed part by part",
               "each_step_ms": [round(1e3 * (b - a), 2) for a, b in zip(marks, marks[1:])],
               "serial_step": serial}
    # roofline of the dominant kernel (radix scatter pass)
    peak, peak_kind = _peak_hbm()
    launches, o_ms, o_bytes = prof.get("radix_onesweep", (0, 0.0, 0))
    achieved = o_bytes / (o_ms / 1e3) / 1e9 if o_ms > 0 else 0.0
    rec = _traffic_record()
    traffic = None
    if rec and launches:
        # DRAM bytes per algorithmic byte of the captured launch, times the
        # algorithmic bytes of an average timed launch
        traffic = rec["dram_bytes_per_key"] / rec["algorithmic_bytes_per_key"] * (o_bytes / launches)
    roofline = {"bound": "hbm", "kernel": "radix_onesweep", "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "algorithmic_bytes_per_launch": (o_bytes / launches) if launches else 0,
                "avg_launch_ms": (o_ms / launches) if launches else 0, "launches": launches}
    kernels = {name: {"launches": la, "ms_per_step": t / args.steps,
                      "GB_per_s": (b / (t / 1e3) / 1e9) if (b and t) else None}
               for name, (la, t, b) in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    total_ms = sum(t for (_, t, _) in prof.values())
    for name in kernels:
        kernels[name]["share"] = prof[name][1] / total_ms if total_ms else 0
    gpu_launches = sum(la for (la, _, _) in prof.values())

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        sa, so = wl["sample"](wl["seed"], CPU_SAMPLE_READS)
        cpu = cpu_baseline_pair(sa, so, k, d, "first %d reads of the workload (%d (k+1)-mers on both strands)"
                                % (len(so) - 1, 2 * int(np.maximum(np.diff(so).astype(np.int64) - k, 0).sum())))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": wl["name"], "reads": len(offs) - 1, "bases": n_bases, "k": k, "d": d,
                       "per_rank": "independent read set per rank (seed + 1000 * rank)",
                       "input": "pinned host memory, uploaded inside every step" if host_input
                                else "device memory (HBM)",
                       "count_buckets": info.get("buckets"), "peak_device_GB": info.get("peak_GB"),
                       "l2": "inputs larger than L2 (%.1f GB of reads, %.1f GB of keys per step)"
                             % (n_bases / 1e9, info["n_kmers"] * 4 / 1e9)},
            "sdbg_edges_per_s": tot["edges"] * args.steps / (ms / 1e3),
            # per call, device-timed: (k+1)-mers over mh_count_kmers, entries over mh_build_sdbg
            "count_kmers_per_s": n_kmers / (phase_ms["count"] / 1e3) if phase_ms["count"] else None,
            "build_edges_per_s": info["m"] / (phase_ms["build"] / 1e3) if phase_ms["build"] else None,
            "phases_ms": phase_ms,
            "sizes": {key: int(v) for key, v in info.items() if key not in ("buckets", "peak_GB")},
            "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": gpu_launches, "clocks": clk,
        }
    ctx.close()
    if rank == 0 and world == 1 and args.workload == "metagenome" and not args.no_extras:
        # the NEXT rows' forms on the same GPU, bounded (a few minutes in all):
        # the served stream (jobs/s, p50/p99) against the same jobs through
        # the plain path one at a time, and the batched sets against the plain
        # path one set after another
        del d_ascii, d_offs
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        line["served"] = _served_extra(local, args)
        torch.cuda.empty_cache()
        line["batched"] = _batched_extra(local, args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


EXTRA_SERVED_SECS = 20.0
EXTRA_SERVED_POOL = 32
EXTRA_BATCHED_STEPS = 2


def _served_extra(local, args):
    f = served_figures(local, EXTRA_SERVED_SECS, EXTRA_SERVED_POOL, 1, False)
    return {"workload": "the served stream (arrivals 20/s) over %.0f s instead of 60, jobs drawn from a pool of "
                        "%d read sets instead of 96; otherwise as the served config" % (EXTRA_SERVED_SECS,
                                                                                   EXTRA_SERVED_POOL),
            "jobs": f["jobs"], "jobs_per_s": f["jobs_per_s"], "p50_ms": f["p50_ms"], "p99_ms": f["p99_ms"],
            "kmers_per_s": f["kmers_per_s"], "serial_jobs_per_s": f["serial"]["jobs_per_s"],
            "burst_jobs_per_s": f["burst"]["jobs_per_s"], "burst_vs_serial": f["burst"]["vs_serial"],
            "max_held_GB": round(f["max_held_bytes"] / 1e9, 1)}


def _batched_extra(local, args):
    import torch

    f = batched_figures(local, BATCHED["n_sets"], EXTRA_BATCHED_STEPS, 1, BATCHED["workers"])
    out = {"workload": "the batched config (64 sets), %d timed batches" % EXTRA_BATCHED_STEPS,
           "sets": f["sets"], "reads": f["reads"], "ms": f["ms"], "serial_ms": f["serial_ms"],
           "jobs_per_s": f["jobs_per_s"], "serial_jobs_per_s": f["serial_jobs_per_s"],
           "kmers_per_s": f["kmers_per_s"], "serial_kmers_per_s": f["serial_kmers_per_s"],
           "batch_speedup": f["batch_speedup"], "count_plan": f["count_plan"]}
    f["ctx"].close()
    del f
    torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    main()
