#!/usr/bin/env python
"""Throughput of the fused relational pipeline (filter -> hash join -> group-by) on GB300.

Default workload: the 600M-row fact / 15M-row dim star query (fk uniform over the dim keys,
pred < 30, group by grp with 100 000 values; SUM, COUNT, MIN, MAX), seeded synthetic data
generated on the device.  One step = one sirius_run_pipeline call: build over the dim, one
fused filter/probe/aggregate pass over the fact table, finalize.  Prints one JSON line; besides
the main line's keys it carries the end-to-end run through host columns (`e2e`), the 512-query
batch (`batched`), the Poisson-served workload (`served`), the 1M-row query's latency and the
300M-row Zipf query with its TABLE_FULL retry (`configs`), and the oracle on the host cores
(`cpu_baseline`).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

N > 1 runs under torchrun, one rank per GPU: every rank runs its own query on its own
seeded tables (independent problems: weak scaling, no data-path collective); the timed region
is bracketed by barriers and the max over ranks is taken.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pipeline rows/s & HBM GB/s vs peak; batched/served vs plain; p50/p99 latency"
WORKLOADS = ("plain_600M", "plain_600M_composite", "skewed_300M", "plain_1M")
PROBE_SOURCES = ["paper_2508_04701_gb300/csrc/pipeline.cu", "paper_2508_04701_gb300/csrc/tables.cuh",
                 "paper_2508_04701_gb300/csrc/common.cuh", "paper_2508_04701_gb300/csrc/pipeline.cuh"]


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="plain_600M", choices=WORKLOADS)
    p.add_argument("--load-factor", type=float, default=0.0)
    p.add_argument("--agg-mode", default="auto")
    p.add_argument("--block-threads", type=int, default=0)
    p.add_argument("--blocks-per-sm", type=int, default=0)
    p.add_argument("--probe-variant", default="auto", choices=["auto", "direct", "staged"])
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--cpu-sample-rows", type=int, default=0,
                   help="fact rows the CPU baseline runs the oracle on (0: the whole workload)")
    p.add_argument("--ref-rows", type=int, default=100_000_000,
                   help="fact rows per step of the reference arm (the oracle on the host cores)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-served", action="store_true")
    p.add_argument("--no-configs", action="store_true")
    p.add_argument("--no-operators", action="store_true")
    p.add_argument("--batch-queries", type=int, default=512)
    p.add_argument("--serve-rate", type=float, default=2000.0)
    p.add_argument("--serve-seconds", type=float, default=10.0)
    p.add_argument("--fifo-seconds", type=float, default=3.0)
    p.add_argument("--serve-sweep", default="8000,16000,32000,64000",
                   help="further arrival rates (q/s), one second each, to find where serving saturates")
    return p.parse_args(argv)


def spec_for(name: str, rank: int):
    from paper_2508_04701_gb300 import datagen as dg
    if name == "plain_600M":
        return dg.plain_scale(seed=rank), 100_000
    if name == "plain_600M_composite":
        return dg.plain_scale(composite=True, seed=rank), 100_000
    if name == "skewed_300M":
        s = dg.skewed(seed=rank)
        return s, s.m
    if name == "plain_1M":
        return dg.plain_small(seed=rank), 1000
    raise ValueError(name)


# ----------------------------------------------------------------------------- environment
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(t: float, world: int, device) -> float:
    """The largest of every rank's t: the slowest rank sets the job's time (t itself on one
    rank).  Every rank must call it, at the same point of its run."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rows_per_s(world: int, rows_per_rank: int, seconds: float) -> float:
    """Whole-job throughput: every rank processes its own rows_per_rank rows (weak scaling)."""
    return world * rows_per_rank / seconds


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def cudart():
    """The CUDA runtime library (for plain copies that measure the host link), or None."""
    import ctypes
    import glob
    cands = []
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib", "/usr/local/cuda/targets/x86_64-linux/lib"):
        cands += sorted(glob.glob(os.path.join(d, "libcudart.so*")))
    for c in cands:
        try:
            lib = ctypes.CDLL(c)
            lib.cudaMemcpyAsync.restype = ctypes.c_int
            lib.cudaMemcpyAsync.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                            ctypes.c_void_p]
            return lib
        except OSError:
            continue
    return None


def source_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def probe_record(workload: str):
    """The committed ncu record of the probe kernel for this workload (DRAM bytes and L2 tag
    requests per launch, the L2's request peak), or None when the kernel's sources changed
    since that capture."""
    path = os.path.join(ROOT, "profiles", "pipe_probe_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    ent = rec.get(workload)
    if not ent or ent.get("source_hash") != source_hash(PROBE_SOURCES):
        return None
    return ent


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
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
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- CPU baseline
def cpu_baseline(spec, rows: int):
    """The oracle as it stands on every host core: the first `rows` fact rows (0 = all) in
    chunks over one worker process per core, each worker's chunks generated beforehand (hot
    inputs, as on the GPU), one timed run from the start message to the merged result."""
    import oracle
    rows = spec.n if rows <= 0 else min(rows, spec.n)
    t0 = time.perf_counter()
    with oracle.HotOracle(spec, rows=rows) as h:
        setup = time.perf_counter() - t0
        res, dt = h.run()
        cores = h.workers
    return {"value": rows / dt, "unit": "rows/s", "cores": cores, "kind": "oracle",
            "sample": f"first {rows} of {spec.n} fact rows of the same query against the full "
                      f"{spec.m}-row dim table, in chunks of up to 20M rows over {cores} worker processes "
                      f"(one per core of sched_getaffinity); {len(res['key'])} groups; one run "
                      f"of {dt:.2f} s after {setup:.1f} s of generation",
            "seconds": dt}


def run_reference(args):
    """--impl reference: the CPU oracle timed on the host cores for the same metric.  Each step
    runs the oracle over a bounded sample of the workload (its first `--ref-rows` fact rows,
    against the full dim table) on every host core; inputs are generated once, before the
    warm-up steps."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    spec, _ = spec_for(args.workload, 0)
    rows = min(spec.n, args.ref_rows)
    with oracle.HotOracle(spec, rows=rows) as h:
        for _ in range(args.warmup):
            h.run()
        times = [h.run()[1] for _ in range(args.steps)]
        cores = h.workers
    per = sum(times) / len(times)
    value = rows / per
    line = {"metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "fact_rows_per_step": rows, "dim_rows": spec.m,
                       "predicate": f"pred < {spec.t}"},
            "cpu_baseline": {"value": value, "unit": "rows/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: the first {rows} of {spec.n} fact rows against the "
                                       f"full {spec.m}-row dim, in chunks of up to 20M rows over {cores} worker "
                                       "processes (one per core of sched_getaffinity)"},
            "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- ours
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2508_04701_gb300 import build
    build.build()
    from paper_2508_04701_gb300 import datagen as dg
    from paper_2508_04701_gb300 import sirius as S

    spec, hint = spec_for(args.workload, rank)
    stream = torch.cuda.current_stream(dev)
    dim = dg.gen_dim_device(spec, dev)
    fact = dg.gen_fact_device(spec, dim, dev)
    aggs = spec.aggs
    desc = S.make_desc(fact, dim, "lt", spec.t, aggs, hint, args.load_factor, args.agg_mode,
                       args.block_threads, args.blocks_per_sm, probe_variant=args.probe_variant)
    out_cap = hint + 1
    outs = S.PipelineOutputs(out_cap, dev)
    scratch = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    # one synchronous run: status and group count
    groups = S.sirius_run_pipeline(desc, outs, scratch, stream, sync=True)
    for _ in range(max(args.warmup, 3) - 1):
        S.sirius_run_pipeline(desc, outs, scratch, stream, sync=False)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    l0 = S.launch_count()
    S.profile_start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        S.sirius_run_pipeline(desc, outs, scratch, stream, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    phases = S.profile_stop()
    launches = S.launch_count() - l0
    barrier()
    clk = clocks.stop()
    t_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_step = t_ms / args.steps
    value = job_rows_per_s(world, spec.n, ms_step / 1e3)
    status = int(outs.d_status.item())

    # roofline of the dominant kernel: the fused probe pass
    peaks, peak_kind = measured_peaks()
    probe_ms, probe_n = phases.get("pipe_probe", (0.0, 0))
    probe_avg_ms = probe_ms / max(probe_n, 1)
    alg_bytes = spec.n * spec.fact_bytes_per_row
    achieved = alg_bytes / (probe_avg_ms / 1e3) / 1e9 if probe_avg_ms > 0 else 0.0
    peak = float(peaks.get("hbm_gbs", 6800.0))
    rec = probe_record(args.workload)
    traffic = rec.get("bytes_per_launch") if rec else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "pipe_probe_kernel",
                "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                "algorithmic_bytes_per_launch": alg_bytes,
                "avg_launch_ms": probe_avg_ms}
    if rec and rec.get("l2_tag_requests_per_launch") and probe_avg_ms > 0:
        # the unit that actually bounds this kernel: L2 tag lookups (each joined row's
        # reductions and direct-array read); requests per launch and the peak rate from the
        # ncu record, the time live
        l2_ach = rec["l2_tag_requests_per_launch"] / (probe_avg_ms / 1e3) / 1e9
        l2_peak = rec["l2_tag_requests_peak_per_s"] / 1e9
        roofline["l2"] = {"unit": "G tag requests/s", "achieved": l2_ach, "peak": l2_peak,
                          "frac": l2_ach / l2_peak,
                          "requests_per_launch": rec["l2_tag_requests_per_launch"],
                          "source": "ncu lts__t_tag_requests (profiles/pipe_probe_traffic.json)"}
    phase_ms = {k: v[0] / max(v[1], 1) for k, v in phases.items()}

    # end to end through the C-ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(S, torch, spec, fact, dim, hint, aggs, args, dev, stream, world)

    # the unfused C-ABI operators on the same tables (filter, join build / probe, gathers,
    # group-by), each against its own roofline, and their chain against the fused call
    operators = None
    if not args.no_operators:
        del scratch
        torch.cuda.empty_cache()
        operators = run_operators(S, torch, spec, fact, dim, dev, stream, ms_step)
        scratch = None
    # release the 600M-row tables before the batched and served workloads
    del fact, dim, desc, scratch
    torch.cuda.empty_cache()
    batched = None
    if not args.no_batched:
        batched = run_batched(S, torch, args, dev, rank)
        torch.cuda.empty_cache()
    served = None
    if not args.no_served:
        served = run_served(S, torch, args, dev, rank)
        torch.cuda.empty_cache()

    configs = None
    if not args.no_configs:
        configs = run_configs(S, torch, dev, rank)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(spec, args.cpu_sample_rows)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": args.workload, "fact_rows": spec.n, "dim_rows": spec.m,
                       "predicate": f"pred < {spec.t}", "groups": groups, "aggregates": aggs,
                       "fact_bytes": alg_bytes, "l2": "inputs larger than L2 (fact columns "
                       f"{alg_bytes / 1e9:.1f} GB read once per step)",
                       "load_factor": args.load_factor or 0.5, "agg_mode": args.agg_mode},
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clk, "e2e": e2e,
            "gpu_launches": launches, "phase_ms": phase_ms, "device_status": status,
            "batched": batched, "served": served, "configs": configs, "operators": operators,
            "hbm_gbs_effective_step": alg_bytes / (ms_step / 1e3) / 1e9,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_operators(S, torch, spec, fact, dim, dev, stream, fused_ms):
    """The query's operators as separate C-ABI calls on the resident 600M-row tables, outputs
    and scratch allocated once, no host synchronisation inside a timed call: filter (pred < t)
    -> join build over the dim keys -> probe of the selected rows' keys -> gather of their
    values and of the matched dim rows' group keys -> hash group-by.  Each is timed with CUDA
    events (mean of 3 after a warm-up) against its algorithmic bytes and the measured copy
    bandwidth; the chain's total is set beside the fused call's time per query."""
    import ctypes
    L = S.lib()
    peak = float(measured_peaks()[0].get("hbm_gbs", 6800.0))
    n, m = spec.n, spec.m
    st = stream.cuda_stream

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def line(ms, rows, alg_bytes, what):
        gbs = alg_bytes / (ms / 1e3) / 1e9
        return {"ms": ms, "rows_per_s": rows / (ms / 1e3), "algorithmic_bytes": alg_bytes,
                "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak, "bytes": what}

    def ok(status):
        if status != S.OK:
            raise RuntimeError(S.last_error())

    out = {}
    # ---- A2 filter
    ids = torch.empty(n, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    fscr = torch.empty(L.sirius_filter_scratch_bytes(n), dtype=torch.uint8, device=dev)
    pred = fact["pred"]
    f_ms = timed(lambda: ok(L.sirius_filter(pred.data_ptr(), n, S.OPS["lt"], spec.t, ids.data_ptr(),
                                            cnt.data_ptr(), None, fscr.data_ptr(), fscr.numel(), st)))
    n_sel = int(cnt.item())
    out["filter"] = line(f_ms, n, 4 * n + 4 * n_sel, "4 B per row read + 4 B per selected row id written")
    out["filter"]["selected"] = n_sel
    del fscr
    # ---- A1 join build (hash table over the dim keys, load factor 1/2)
    tab = S.HashJoinTable(m, 4, 0.5, dev)
    cap = tab.capacity
    b_ms = timed(lambda: ok(L.sirius_hash_join_build(dim["pk"].data_ptr(), None, m, ctypes.byref(tab.struct),
                                                     None, st)))
    out["join_build"] = line(b_ms, m, 8 * cap + 4 * m + 8 * m,
                             "table cleared (8 B per slot) + 4 B key read + one 8 B slot written per row")
    out["join_build"]["capacity"] = cap
    # ---- A3 probe: the selected rows' keys against the table
    pp = torch.empty(n_sel, dtype=torch.int32, device=dev)
    pb = torch.empty(n_sel, dtype=torch.int32, device=dev)
    pc = torch.zeros(1, dtype=torch.int64, device=dev)
    p_ms = timed(lambda: ok(L.sirius_hash_join_probe(ctypes.byref(tab.struct), fact["fk"].data_ptr(), None,
                                                     ids.data_ptr(), n_sel, pp.data_ptr(), pb.data_ptr(),
                                                     n_sel, pc.data_ptr(), None, st)))
    pairs = int(pc.item())
    out["join_probe"] = line(p_ms, n_sel, n_sel * (4 + 4 + 32) + pairs * 8,
                             "4 B row id + 4 B key + one 32 B bucket sector per probe, 8 B per pair out")
    out["join_probe"]["pairs"] = pairs
    # A/B: four rows per thread (variant 1) against four lanes per key (variant 2, warp-
    # cooperative), at load factors 1/2 and 0.9 (the same probes; pairs must agree)
    ab = {}
    for lf in (0.5, 0.9):
        for var in (1, 2):
            t2 = S.HashJoinTable(m, 4, lf, dev, probe_variant=var)
            ok(L.sirius_hash_join_build(dim["pk"].data_ptr(), None, m, ctypes.byref(t2.struct), None, st))
            ms2 = timed(lambda: ok(L.sirius_hash_join_probe(ctypes.byref(t2.struct), fact["fk"].data_ptr(), None,
                                                            ids.data_ptr(), n_sel, pp.data_ptr(), pb.data_ptr(),
                                                            n_sel, pc.data_ptr(), None, st)))
            ab[f"lf{lf}_variant{var}"] = {"ms": ms2, "pairs_agree": int(pc.item()) == pairs,
                                          "table_mb": t2.mem.numel() / 1e6}
            del t2
    out["join_probe"]["variants"] = ab
    ok(L.sirius_hash_join_probe(ctypes.byref(tab.struct), fact["fk"].data_ptr(), None, ids.data_ptr(), n_sel,
                                pp.data_ptr(), pb.data_ptr(), n_sel, pc.data_ptr(), None, st))
    del tab
    # ---- A4 gathers: values by probe row, group keys by build row
    gv = torch.empty(pairs, dtype=torch.int64, device=dev)
    gk = torch.empty(pairs, dtype=torch.int64, device=dev)
    v_ms = timed(lambda: ok(L.sirius_gather_i64(fact["val"].data_ptr(), pp.data_ptr(), pairs, gv.data_ptr(), st)))
    out["gather_val"] = line(v_ms, pairs, pairs * (4 + 8 + 8), "4 B index + 8 B value read + 8 B written")
    k_ms = timed(lambda: ok(L.sirius_gather_group_key(dim["grp"].data_ptr(), None, pb.data_ptr(), pairs,
                                                      gk.data_ptr(), st)))
    out["gather_group_key"] = line(k_ms, pairs, pairs * (4 + 4 + 8), "4 B index + 4 B grp read + 8 B key written")
    del pp, pb
    # ---- A5/A6 hash group-by of the joined rows
    hint = 100_000
    gouts = S.groupby_outputs(L.sirius_groupby_capacity(hint) + 1, dev)
    gscr = torch.empty(L.sirius_groupby_scratch_bytes(hint), dtype=torch.uint8, device=dev)
    g_ms = timed(lambda: S.sirius_groupby_agg(gk, gv, group_cap_hint=hint, stream=stream, outputs=gouts,
                                               scratch=gscr, sync=False))
    out["groupby"] = line(g_ms, pairs, pairs * 16, "8 B key + 8 B value per row")
    out["groupby"]["groups"] = int(gouts["groups"].item())
    chain = f_ms + b_ms + p_ms + v_ms + k_ms + g_ms
    out["unfused_chain_ms"] = chain
    out["fused_ms_per_query"] = fused_ms
    out["fused_speedup_vs_unfused"] = chain / fused_ms if fused_ms > 0 else None
    del ids, gv, gk, gouts, gscr
    torch.cuda.empty_cache()
    return out


def run_batched(S, torch, args, dev, rank):
    """512 independent pipelines (sizes log-uniform 10K-20M fact rows, 1K-2M dim rows,
    t uniform 5..90): one batch plan (persistent launches, CUDA graph) against 512 plain
    sirius_run_pipeline calls on the same stream, identical results required."""
    from paper_2508_04701_gb300 import autotune
    from paper_2508_04701_gb300 import datagen as dg
    nq = args.batch_queries
    specs = [dg.batch_query(q, seed=rank) for q in range(nq)]
    tabs = []
    for sp in specs:
        dim = dg.gen_dim_device(sp, dev)
        tabs.append((dim, dg.gen_fact_device(sp, dim, dev)))
    descs = [S.make_desc(f, d, "lt", sp.t, "sum,count,min,max", 1000) for sp, (d, f) in zip(specs, tabs)]
    cap = S.lib().sirius_groupby_capacity(1000) + 1
    outs_b = [S.PipelineOutputs(cap, dev) for _ in range(nq)]
    outs_p = [S.PipelineOutputs(cap, dev) for _ in range(nq)]
    rows = sum(sp.n for sp in specs)
    fact_bytes = sum(sp.n * sp.fact_bytes_per_row for sp in specs)
    torch.cuda.synchronize()

    def ev_time(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # plain: one sirius_run_pipeline per query, back to back on one stream
    p_scr = torch.empty(max(S.pipeline_scratch_bytes(d) for d in descs), dtype=torch.uint8, device=dev)

    def plain():
        for d, o in zip(descs, outs_p):
            S.sirius_run_pipeline(d, o, p_scr, sync=False)
    t_plain = ev_time(plain, 3)
    plan = S.BatchPlan(nq)
    scr = torch.empty(S.batch_scratch_bytes(descs), dtype=torch.uint8, device=dev)
    t_batch = ev_time(lambda: plan.run(descs, outs_b, scratch=scr, sync=False), 3)
    S.profile_start()
    plan.run(descs, outs_b, scratch=scr, sync=False)
    torch.cuda.synchronize()
    batch_phases = {k: v[0] for k, v in S.profile_stop().items()}
    t_graph = ev_time(lambda: plan.run(descs, outs_b, scratch=scr, use_graph=True, sync=False), 5)
    tuned = autotune.tune_batch(plan, descs, outs_b, use_graph=True, use_cache=False,
                                units=(16_384, 65_536, 262_144), load_factors=(0.35, 0.5, 0.7))
    scr = torch.empty(S.batch_scratch_bytes(descs), dtype=torch.uint8, device=dev)
    t_tuned = ev_time(lambda: plan.run(descs, outs_b, scratch=scr, use_graph=True,
                                       rows_per_unit=tuned["rows_per_unit"], sync=False), 5)
    # identical results: every query's groups equal between the batched and the plain run
    gb = plan.run(descs, outs_b, scratch=scr, use_graph=True, rows_per_unit=tuned["rows_per_unit"])
    for d in descs:
        d.load_factor = 0.0
    same = True
    for d, ob, op, g in zip(descs, outs_b, outs_p, gb):
        S.sirius_run_pipeline(d, op, p_scr, sync=False)
        if int(op.d_groups.item()) != g:
            same = False
            break
        kb, ib = torch.sort(ob.t["key"][:g])
        kp, ip = torch.sort(op.t["key"][:g])
        for c in ("sum", "count", "min", "max"):
            if not torch.equal(ob.t[c][:g][ib], op.t[c][:g][ip]):
                same = False
        if not torch.equal(kb, kp):
            same = False
    plan.close()
    res = {"queries": nq, "fact_rows": rows, "fact_bytes": fact_bytes,
           "plain_ms": t_plain, "batched_ms": t_batch, "batched_graph_ms": t_graph, "autotuned_graph_ms": t_tuned,
           "plain_rows_per_s": rows / (t_plain / 1e3), "batched_rows_per_s": rows / (t_batch / 1e3),
           "batched_graph_rows_per_s": rows / (t_graph / 1e3),
           "autotuned_rows_per_s": rows / (t_tuned / 1e3), "speedup_vs_plain": t_plain / min(t_graph, t_tuned),
           "autotuned": {k: tuned[k] for k in ("rows_per_unit", "load_factor")},
           "batched_phase_ms": batch_phases,
           "hbm_gbs_effective": fact_bytes / (min(t_graph, t_tuned) / 1e3) / 1e9,
           "results_identical_to_plain": same}
    del tabs
    return res


def run_served(S, torch, args, dev, rank):
    """Open-loop Poisson arrivals (rate args.serve_rate) over a resident pool of 512 fact
    tables and 64 dim tables with their dim indexes; continuous batching against plain
    sequential execution (FIFO, one request at a time) on the same GPU."""
    from paper_2508_04701_gb300 import serve
    pool = serve.ResidentPool(n_facts=512, n_dims=64, seed=rank, device=dev)
    dur = args.serve_seconds + 1.0
    reqs = serve.poisson_requests(args.serve_rate, dur, len(pool.facts), seed=rank)
    srv = serve.Server(pool, slots=4, max_batch=64, budget_bytes=150 * 10**9)
    warm = serve.poisson_requests(args.serve_rate, 0.3, len(pool.facts), seed=rank + 99)
    srv.run(warm)
    batches0 = srv.batches
    srv.run(reqs)
    st = serve.latency_stats(reqs, warmup=1.0)
    st.update(overlap_stats(srv, reqs))
    st["batches_this_run"] = srv.batches - batches0
    rows = sum(pool.fact_rows[r.fact_id] for r in reqs if r.arrival >= 1.0)
    st["rows_per_s"] = rows / (args.serve_seconds) if args.serve_seconds > 0 else 0.0
    st["batches"] = srv.batches
    st["statuses_ok"] = all(r.status == 0 for r in reqs)
    st["pool_bytes"] = pool.bytes()
    st["budget_bytes"] = srv.admission.budget
    st["admission_deferrals"] = srv.admission.rejected
    # plain sequential FIFO on the same arrival schedule (a bounded prefix of it)
    fifo_reqs = [serve.Request(r.rid, r.fact_id, r.t, r.arrival) for r in reqs if r.arrival < args.fifo_seconds]
    serve.sequential_fifo(pool, fifo_reqs)
    fst = serve.latency_stats(fifo_reqs)
    # the arrival rate swept upwards: throughput follows the offered rate until the GPU (or the
    # host loop) saturates, then the queue and the p99 grow
    sweep = []
    for k, rate in enumerate(float(x) for x in args.serve_sweep.split(",") if x.strip()):
        rq = serve.poisson_requests(rate, 1.3, len(pool.facts), seed=rank + 1000 + k)
        b0 = srv.batches
        srv.run(rq)
        sw = serve.latency_stats(rq, warmup=0.3)
        sw.update(overlap_stats(srv, rq))
        sw["batches"] = srv.batches - b0
        sw["offered_qps"] = rate
        done = [r for r in rq if r.arrival >= 0.3 and r.done == r.done]  # completed (done is not NaN)
        span = (max(r.done for r in done) - min(r.arrival for r in done)) if done else 0.0
        sw["rows_per_s"] = sum(pool.fact_rows[r.fact_id] for r in done) / span if span > 0 else 0.0
        sw["statuses_ok"] = all(r.status == 0 for r in rq)
        sweep.append({k2: sw.get(k2) for k2 in ("offered_qps", "throughput_qps", "p50_ms", "p99_ms", "rows_per_s",
                                                "requests", "statuses_ok", "batches", "max_busy_slots",
                                                "max_busy_device", "device_busy_frac", "host_ms_per_request",
                                                "host_busy_frac")})
    return {"rate_qps": args.serve_rate, "seconds": args.serve_seconds, "served": st,
            "plain_fifo": fst, "fifo_seconds": args.fifo_seconds, "rate_sweep": sweep}


def overlap_stats(srv, reqs):
    """How the last Server.run used the device and the host: the most batches in flight on the
    device at once (from per-batch CUDA events), the fraction of the run's device span with at
    least one batch in flight, the most slots the host loop had busy at once, and the host
    loop's own time (launching batches, reading results back) per request and as a fraction of
    the run's wall time."""
    spans = srv.spans
    out = {"max_busy_slots": srv.max_busy_slots, "max_busy_device": srv.max_busy_device}
    if spans:
        t0, t1 = min(a for a, _ in spans), max(b for _, b in spans)
        out["device_busy_frac"] = srv.device_busy_ms() / (t1 - t0) if t1 > t0 else None
    n = max(len(reqs), 1)
    host_s = srv.host_launch_s + srv.host_complete_s
    out["host_ms_per_request"] = host_s * 1e3 / n
    done = [r.done for r in reqs if r.done == r.done]
    wall = max(done) - min(r.arrival for r in reqs) if done else 0.0
    out["host_busy_frac"] = host_s / wall if wall > 0 else None
    return out


def run_configs(S, torch, dev, rank):
    """The metric's other single-GPU configurations, measured beside the main line.
    1M-row query: latency per query, median of 100 timed runs after 10 warm-ups, as a plain
    sirius_run_pipeline call (the single launch), through the per-phase kernels, as the same
    call captured once in a CUDA graph and replayed (both
    must give the same groups), and as a one-query batch plan.  The 600M-row query on two-column join keys (hash-table join):
    rows/s and phases.  300M-row Zipf(1.1) query with (grp, flag) group keys: rows/s
    and G, then the same query with group_cap_hint a quarter of the dim's 10M group keys, which
    must fail with TABLE_FULL, its retry with the full hint, and the top 100 of its groups by
    COUNT (sirius_topn_groups over 5.9M groups)."""
    from paper_2508_04701_gb300 import datagen as dg
    stream = torch.cuda.current_stream(dev)
    out = {}

    def median_us(fn, warm=10, reps=100):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        return statistics.median(ts)

    # ---- 1M-row query
    spec = dg.plain_small(seed=rank)
    dim = dg.gen_dim_device(spec, dev)
    fact = dg.gen_fact_device(spec, dim, dev)
    desc = S.make_desc(fact, dim, "lt", spec.t, spec.aggs, 1000)
    o1, o2 = S.PipelineOutputs(1001, dev), S.PipelineOutputs(1001, dev)
    scr = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device=dev)
    g1 = S.sirius_run_pipeline(desc, o1, scr, stream, sync=True)
    us_plain = median_us(lambda: S.sirius_run_pipeline(desc, o1, scr, stream, sync=False))
    # the same query through the per-phase kernels (the default above is the single launch)
    desc_multi = S.make_desc(fact, dim, "lt", spec.t, spec.aggs, 1000, probe_variant="direct")
    us_multi = median_us(lambda: S.sirius_run_pipeline(desc_multi, o1, scr, stream, sync=False))
    # the same call captured once into a CUDA graph and replayed
    scr2 = torch.empty_like(scr)
    us_graph, graph_error = None, None
    try:
        graph = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream(dev)
        cs.wait_stream(stream)
        S.sirius_run_pipeline(desc, o2, scr2, cs, sync=False)
        cs.synchronize()
        with torch.cuda.graph(graph, stream=cs):
            S.sirius_run_pipeline(desc, o2, scr2, cs, sync=False)
        us_graph = median_us(lambda: graph.replay())
    except Exception as e:  # capture refused: report why instead of a number
        graph_error = str(e).splitlines()[0][:200]
    torch.cuda.synchronize()
    g2 = int(o2.d_groups.item())
    same = g1 == g2
    if same:
        a, b = o1.trimmed(g1), o2.trimmed(g2)
        ia, ib = torch.sort(a["key"]).indices, torch.sort(b["key"]).indices
        same = all(torch.equal(a[c][ia], b[c][ib]) for c in a)
    # a one-query batch plan replaying its own graph; its time includes the plan's host work
    # per call (task table, copy in, status copy out)
    plan = S.BatchPlan(1)
    o3 = S.PipelineOutputs(1001, dev)
    bscr = torch.empty(S.batch_scratch_bytes([desc]), dtype=torch.uint8, device=dev)
    plan.run([desc], [o3], scratch=bscr, use_graph=True, stream=stream)
    us_plan = median_us(lambda: plan.run([desc], [o3], scratch=bscr, use_graph=True, stream=stream, sync=False))
    plan.close()
    out["plain_1M"] = {"rows": spec.n, "groups": g1, "us_per_query_median": us_plain,
                       "path": "single launch (probe_variant auto)",
                       "us_per_query_multi_kernel_median": us_multi,
                       "rows_per_s": spec.n / (us_plain / 1e6), "us_per_query_graph_median": us_graph,
                       "rows_per_s_graph": spec.n / (us_graph / 1e6) if us_graph else None,
                       "graph_error": graph_error, "graph_results_identical": bool(same),
                       "us_per_query_one_query_plan_median": us_plan,
                       "timing": "CUDA events per query, median of 100 after 10 warm-ups"}
    del fact, dim, desc, desc_multi, scr, scr2, bscr, o1, o2, o3

    # ---- 600M-row query on two-column join keys: the hash-table join at full size
    spec = dg.plain_scale(composite=True, seed=rank)
    dim = dg.gen_dim_device(spec, dev)
    fact = dg.gen_fact_device(spec, dim, dev)
    desc = S.make_desc(fact, dim, "lt", spec.t, spec.aggs, 100_000)
    o = S.PipelineOutputs(100_001, dev)
    scr = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device=dev)
    g = S.sirius_run_pipeline(desc, o, scr, stream, sync=True)
    S.profile_start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        S.sirius_run_pipeline(desc, o, scr, stream, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ph = {k: v[0] / max(v[1], 1) for k, v in S.profile_stop().items()}
    ms = e0.elapsed_time(e1) / 3
    out["plain_600M_composite"] = {"rows": spec.n, "groups": g, "ms_per_query": ms,
                                   "rows_per_s": spec.n / (ms / 1e3), "phase_ms": ph,
                                   "join": "hash table (two-column keys), 20 B/row of fact columns"}
    del fact, dim, desc, scr, o
    torch.cuda.empty_cache()

    # ---- the 600M-row query forced through the hash-table join, its load factor swept (the
    # autotuner's knob: a fuller table is smaller, 0.95 -> 126 MB against the 129 MB L2)
    spec = dg.plain_scale(seed=rank)
    dim = dg.gen_dim_device(spec, dev)
    fact = dg.gen_fact_device(spec, dim, dev)
    peak = float(measured_peaks()[0].get("hbm_gbs", 6800.0))
    sweep = {}
    for lf in (0.5, 0.7, 0.9, 0.95):
        desc = S.make_desc(fact, dim, "lt", spec.t, spec.aggs, 100_000, load_factor=lf, join_mode="hash")
        o = S.PipelineOutputs(100_001, dev)
        scr = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device=dev)
        g = S.sirius_run_pipeline(desc, o, scr, stream, sync=True)
        S.profile_start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            S.sirius_run_pipeline(desc, o, scr, stream, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ph = {k: v[0] / max(v[1], 1) for k, v in S.profile_stop().items()}
        ms = e0.elapsed_time(e1) / 3
        pr = ph.get("pipe_probe", 0.0)
        sweep[f"lf_{lf}"] = {"groups": g, "ms_per_query": ms, "rows_per_s": spec.n / (ms / 1e3), "phase_ms": ph,
                             "probe_roofline_frac": (spec.n * 16 / (pr / 1e3) / 1e9 / peak) if pr > 0 else None,
                             "table_mb": S.lib().sirius_join_table_bytes(
                                 S.lib().sirius_join_table_capacity(spec.m, lf), 4) / 1e6}
        del desc, o, scr
    best = min(sweep, key=lambda k: sweep[k]["ms_per_query"])
    out["plain_600M_hash_join"] = {"rows": spec.n, "join": "hash table forced (join_mode 1), one-column keys",
                                   "load_factor_sweep": sweep, "best": best,
                                   "roofline": {"bound": "hbm", "kernel": "probe_kernel (hash-table join)",
                                                "frac": sweep[best]["probe_roofline_frac"], "peak": peak,
                                                "unit": "GB/s", "bytes_per_row": 16}}
    del fact, dim
    torch.cuda.empty_cache()

    # ---- the 600M-row query with a dim-side predicate (dattr < 10: a tenth of the dim rows take
    # part): direct array; hash table with and without the Bloom pre-filter; hash table without
    # the predicate for reference
    spec = dg.plain_scale(seed=rank, dt=10)
    dim = dg.gen_dim_device(spec, dev)
    fact = dg.gen_fact_device(spec, dim, dev)
    runs = {}
    for name, kw in (("direct", {"dim_op": "lt", "dim_literal": 10}),
                     ("hash_bloom", {"dim_op": "lt", "dim_literal": 10, "join_mode": "hash", "bloom": "on"}),
                     ("hash_no_bloom", {"dim_op": "lt", "dim_literal": 10, "join_mode": "hash", "bloom": "off"}),
                     ("hash_no_predicate", {"join_mode": "hash"})):
        desc = S.make_desc(fact, dim, "lt", spec.t, spec.aggs, 100_000, **kw)
        o = S.PipelineOutputs(100_001, dev)
        scr = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device=dev)
        g = S.sirius_run_pipeline(desc, o, scr, stream, sync=True)
        S.profile_start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            S.sirius_run_pipeline(desc, o, scr, stream, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ph = {k: v[0] / max(v[1], 1) for k, v in S.profile_stop().items()}
        ms = e0.elapsed_time(e1) / 3
        runs[name] = {"groups": g, "ms_per_query": ms, "rows_per_s": spec.n / (ms / 1e3), "phase_ms": ph}
        del desc, o, scr
    out["plain_600M_dim_predicate"] = {"rows": spec.n, "dim_predicate": "dattr < 10 (10 % of dim rows)",
                                       "runs": runs}
    del fact, dim
    torch.cuda.empty_cache()

    # ---- star query: the 600M-row query joined to two 1.5M-row dims as filters (attr < 50 each)
    spec = dg.star(seed=rank)
    dim = dg.gen_dim_device(spec, dev)
    fact = dg.gen_fact_device(spec, dim, dev)
    sdims = dg.gen_semi_dims_device(spec, dev)
    desc = S.make_desc(fact, dim, "lt", spec.t, spec.aggs, 100_000, semi=dg.semi_args(spec, fact, sdims))
    o = S.PipelineOutputs(100_001, dev)
    scr = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device=dev)
    g = S.sirius_run_pipeline(desc, o, scr, stream, sync=True)
    S.profile_start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        S.sirius_run_pipeline(desc, o, scr, stream, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ph = {k: v[0] / max(v[1], 1) for k, v in S.profile_stop().items()}
    ms = e0.elapsed_time(e1) / 3
    out["star_600M"] = {"rows": spec.n, "groups": g, "ms_per_query": ms, "rows_per_s": spec.n / (ms / 1e3),
                        "phase_ms": ph, "filter_dims": f"2 x {spec.semi_m} rows, attr < {spec.semi_t} each",
                        "fact_bytes_per_row": 24}
    del fact, dim, sdims, desc, o, scr
    torch.cuda.empty_cache()

    # ---- group-by alone, hash table vs sort: 100M rows, int32 keys over 1e5 and 1e7 values
    n = 100_000_000
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234 + rank)
    vals = torch.randint(0, 10**8, (n,), dtype=torch.int64, device=dev, generator=gen)
    gb = {}
    for dom in (100_000, 10_000_000):
        keys = torch.randint(0, dom, (n,), dtype=torch.int32, device=dev, generator=gen)
        res = {}
        # the hash group-by through the C ABI with its outputs and scratch allocated once and no
        # host synchronisation inside the timed call (G stays on the device)
        gouts = S.groupby_outputs(S.lib().sirius_groupby_capacity(dom) + 1, dev)
        gscr = torch.empty(S.lib().sirius_groupby_scratch_bytes(dom), dtype=torch.uint8, device=dev)
        for name, fn in (("hash", lambda: S.sirius_groupby_agg(keys, vals, group_cap_hint=dom, stream=stream,
                                                               outputs=gouts, scratch=gscr, sync=False)),
                         ("sort", lambda: S.sirius_groupby_sort(keys, vals, out_cap=dom, stream=stream))):
            fn()
            torch.cuda.synchronize()
            g_ = int(gouts["groups"].item()) if name == "hash" else int(fn()["key"].numel())
            res[name] = {"ms": median_us(fn, 2, 5) / 1e3, "groups": g_}
        res["hash"]["rows_per_s"] = n / (res["hash"]["ms"] / 1e3)
        res["hash"]["hbm_frac_12B_per_row"] = n * 12 / (res["hash"]["ms"] / 1e3) / 1e9 / float(
            measured_peaks()[0].get("hbm_gbs", 6800.0))
        gb[f"keys_{dom}"] = res
        del keys, gouts, gscr
    out["groupby_hash_vs_sort_100M"] = gb
    del vals
    torch.cuda.empty_cache()

    # ---- string keys: 50M rows over 1e5 and 1e6 distinct strings (2..20 bytes, mean ~12)
    sg = {}
    for d in (100_000, 1_000_000):
        col = dg.gen_strings_device(dg.StringSpec(n=50_000_000, d=d, seed=rank), dev)
        off, ch, v = col["offsets"], col["chars"], col["vals"]
        ids32 = col["ids"].to(torch.int32)
        res = {"rows": int(v.numel()), "chars_bytes": int(ch.numel())}
        for name, fn in (
                ("dict_encode", lambda: S.sirius_dict_encode(off, ch, distinct_hint=d, stream=stream)),
                ("groupby_string", lambda: S.sirius_groupby_string(off, ch, v, distinct_hint=d, stream=stream)),
                ("groupby_int_hash_same_ids", lambda: S.sirius_groupby_agg(ids32, v, group_cap_hint=d, stream=stream)),
                ("groupby_int_sort_same_ids", lambda: S.sirius_groupby_sort(ids32, v, out_cap=d, stream=stream))):
            res[name + "_ms"] = median_us(fn, 1, 3) / 1e3
        res["groupby_string_rows_per_s"] = res["rows"] / (res["groupby_string_ms"] / 1e3)
        res["groups"] = int(S.sirius_groupby_string(off, ch, v, distinct_hint=d, stream=stream)["row"].numel())
        sg[f"distinct_{d}"] = res
        del col, off, ch, v, ids32
        torch.cuda.empty_cache()
    out["groupby_string_50M"] = sg

    # ---- 300M-row Zipf query, 10M group keys
    spec = dg.skewed(seed=rank)
    dim = dg.gen_dim_device(spec, dev)
    fact = dg.gen_fact_device(spec, dim, dev)
    need = spec.m
    desc = S.make_desc(fact, dim, "lt", spec.t, spec.aggs, need)
    o = S.PipelineOutputs(need + 1, dev)
    scr = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device=dev)
    g = S.sirius_run_pipeline(desc, o, scr, stream, sync=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        S.sirius_run_pipeline(desc, o, scr, stream, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    small = need // 4
    desc_s = S.make_desc(fact, dim, "lt", spec.t, spec.aggs, small)
    scr_s = torch.empty(S.pipeline_scratch_bytes(desc_s), dtype=torch.uint8, device=dev)
    o_s = S.PipelineOutputs(small + 1, dev)
    t0 = time.perf_counter()
    try:
        S.sirius_run_pipeline(desc_s, o_s, scr_s, stream, sync=True)
        first = "OK"
    except S.SiriusError as e:
        first = S.STATUS_NAMES.get(e.status, str(e.status))
    g_retry = S.sirius_run_pipeline(desc, o, scr, stream, sync=True)
    t_retry = time.perf_counter() - t0
    # ORDER BY COUNT DESC, key LIMIT 100 over the 5.9M groups
    keys_t, cnt_t = o.t["key"][:g_retry], o.t["count"][:g_retry]
    tscr = torch.empty(S.lib().sirius_topn_scratch_bytes(100), dtype=torch.uint8, device=dev)
    us_top = median_us(lambda: S.sirius_topn_groups(keys_t, cnt_t, 100, True, scratch=tscr, stream=stream), 3, 10)
    out["skewed_300M"] = {"rows": spec.n, "groups": g, "ms_per_query": ms, "rows_per_s": spec.n / (ms / 1e3),
                          "aggregates": spec.aggs, "group_keys_in_dim": need,
                          "undersized_hint": {"group_cap_hint": small, "first_status": first, "retries": 1,
                                              "groups_after_retry": g_retry,
                                              "ms_failed_run_plus_retry": t_retry * 1e3},
                          "top100_by_count_us": us_top}
    del fact, dim, desc, desc_s, scr, scr_s, o, o_s
    return out


def run_e2e(S, torch, spec, fact, dim, hint, aggs, args, dev, stream, world):
    """The same query through sirius_run_pipeline_host: fact and dim columns in pinned host
    memory; every step moves them to the device inside the call and copies the result rows
    back.  Two ways are timed -- staged copies (chunks, one copy stream per column, overlapped
    with the probe pass) and in-place reads of the pinned columns by the probe pass -- and the
    faster one is reported."""
    hf = S.pinned_copy(fact)
    hd = S.pinned_copy(dim)
    desc = S.make_desc(hf, hd, "lt", spec.t, aggs, hint, args.load_factor, args.agg_mode,
                       args.block_threads, args.blocks_per_sm, host=True,
                       probe_variant=args.probe_variant)
    outs = S.HostOutputs(hint + 1)
    modes = {}
    g = 0
    for name, chunk in (("staged_copies", 0), ("in_place", -1)):
        scratch = torch.empty(S.pipeline_host_scratch_bytes(desc, chunk, outs.cap), dtype=torch.uint8,
                              device=dev)
        g = S.sirius_run_pipeline_host(desc, outs, chunk, scratch, stream, dev)   # warm-up
        times = []
        for _ in range(args.e2e_steps):
            if world > 1:
                import torch.distributed as dist
                dist.barrier()
            t0 = time.perf_counter()
            g = S.sirius_run_pipeline_host(desc, outs, chunk, scratch, stream, dev)
            times.append(time.perf_counter() - t0)
        modes[name] = max_over_ranks(sum(times) / len(times), world, dev)
        del scratch
    best = min(modes, key=modes.get)
    t = modes[best]
    h2d = sum(v.numel() * v.element_size() for v in hf.values()) + \
        sum(v.numel() * v.element_size() for v in hd.values())
    d2h = g * 8 * 5 + 256
    # the link's ceiling on this machine: plain copies of the same pinned columns to the device,
    # each column in 16M-element pieces on a stream of its own (all columns in flight together,
    # as the library's staged chunks are), by cudaMemcpyAsync from the CUDA runtime itself (torch's
    # copy_ of pinned views has measured well below the link on some boxes), timed with CUDA events
    # from the launching stream
    dst = {k: torch.empty_like(v, device=dev) for k, v in list(hf.items()) + [("d_" + k, v) for k, v in hd.items()]}
    src = dict(list(hf.items()) + [("d_" + k, v) for k, v in hd.items()])
    side = {k: torch.cuda.Stream(device=dev) for k in src}
    main = torch.cuda.current_stream(dev)
    rt = cudart()
    piece = 1 << 24

    def copy_all():
        start = torch.cuda.Event()
        start.record(main)
        for k, v in src.items():
            side[k].wait_event(start)
            es = v.element_size()
            for i in range(0, v.numel(), piece):
                m = min(piece, v.numel() - i)
                if rt is not None:
                    rc = rt.cudaMemcpyAsync(ctypes.c_void_p(dst[k].data_ptr() + i * es),
                                            ctypes.c_void_p(v.data_ptr() + i * es), ctypes.c_size_t(m * es),
                                            1, ctypes.c_void_p(side[k].cuda_stream))
                    if rc != 0:
                        raise RuntimeError(f"cudaMemcpyAsync failed: {rc}")
                else:
                    with torch.cuda.stream(side[k]):
                        dst[k][i:i + m].copy_(v[i:i + m], non_blocking=True)
        for k in src:
            done = torch.cuda.Event()
            done.record(side[k])
            main.wait_event(done)
    copy_all()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for _ in range(3):
        copy_all()
    e1.record(main)
    torch.cuda.synchronize()
    copy_gbs = h2d / (e0.elapsed_time(e1) / 3 / 1e3) / 1e9
    del dst
    return {"value": job_rows_per_s(world, spec.n, t), "unit": "rows/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": t * 1e3, "steps": args.e2e_steps,
            "h2d_gbs": h2d / t / 1e9, "mode": best,
            "ms_per_step_by_mode": {k: v * 1e3 for k, v in modes.items()},
            "link_copy_gbs": copy_gbs, "link_frac": (h2d / t / 1e9) / copy_gbs,
            "call": "sirius_run_pipeline_host (pinned host columns)"}


if __name__ == "__main__":
    main()
