"""A small, fixed pipeline case for profiling one probe kernel under ncu.

    python -m paper_2508_04701_gb300.profile_case [--n ROWS] [--m DIM_ROWS]
                                                  [--variant auto|direct|staged|single]
                                                  [--load-factor LF] [--runs R]
    python -m paper_2508_04701_gb300.profile_case --workload plain_1M --variant single
    python -m paper_2508_04701_gb300.profile_case --op sort --n ROWS --m DISTINCT_KEYS
    python -m paper_2508_04701_gb300.profile_case --op groupby --n ROWS --m DISTINCT_KEYS
    python -m paper_2508_04701_gb300.profile_case --op strings --n ROWS --m DISTINCT_STRINGS
    python -m paper_2508_04701_gb300.profile_case --op operators [--n ROWS] [--m DIM_ROWS]

--op sort runs the sort-based group-by on int32 keys U[0, m) with int64 values; --op groupby the
hash group-by (SUM, COUNT, MIN, MAX) on the same inputs; --op strings
dictionary-encodes a seeded string column of n rows over m distinct strings; --op operators
runs the query's unfused C-ABI operators on the 600M-row query's distributions at n rows:
filter (pred < 30), join build over the dim keys, probe of the selected rows, gathers of their
values and group keys, hash group-by.

Builds the 600M-row query's distributions at a reduced fact size (default 100M rows, 1.6 GB of
columns, above the L2 size) against the full 15M-row dim table, and runs the pipeline R times.
--workload plain_1M runs the 1M-row fact / 65 536-row dim / 1 000-group query instead (its sizes
are fixed).
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=100_000_000)
    p.add_argument("--m", type=int, default=15_000_000)
    p.add_argument("--variant", default="direct", choices=["auto", "direct", "staged", "single"])
    p.add_argument("--load-factor", type=float, default=0.0)
    p.add_argument("--runs", type=int, default=2)
    p.add_argument("--workload", default="plain", choices=["plain", "composite", "skewed", "star", "plain_1M"])
    p.add_argument("--join-mode", default="auto", choices=["auto", "hash"])
    p.add_argument("--agg-mode", default="auto", choices=["auto", "smem", "global", "part", "hot", "routed"])
    p.add_argument("--batch", type=int, default=0, help="run a batch of this many queries instead")
    p.add_argument("--op", default="pipeline", choices=["pipeline", "sort", "groupby", "strings", "operators"])
    a = p.parse_args()
    import torch

    from paper_2508_04701_gb300 import datagen as dg
    from paper_2508_04701_gb300 import sirius as S
    if a.op == "groupby":
        gen = torch.Generator(device="cuda")
        gen.manual_seed(1)
        vals = torch.randint(0, 10**8, (a.n,), dtype=torch.int64, device="cuda", generator=gen)
        keys = torch.randint(0, a.m, (a.n,), dtype=torch.int32, device="cuda", generator=gen)
        outs = S.groupby_outputs(S.lib().sirius_groupby_capacity(a.m) + 1, "cuda")
        scr = torch.empty(S.lib().sirius_groupby_scratch_bytes(a.m), dtype=torch.uint8, device="cuda")
        for _ in range(a.runs):
            S.sirius_groupby_agg(keys, vals, "sum,count,min,max", a.m, outputs=outs, scratch=scr, sync=False)
        torch.cuda.synchronize()
        print(f"profile case ok: hash group-by of {a.n} rows, {int(outs['groups'].item())} groups")
        return
    if a.op == "sort":
        gen = torch.Generator(device="cuda")
        gen.manual_seed(1)
        vals = torch.randint(0, 10**8, (a.n,), dtype=torch.int64, device="cuda", generator=gen)
        keys = torch.randint(0, a.m, (a.n,), dtype=torch.int32, device="cuda", generator=gen)
        for _ in range(a.runs):
            g = S.sirius_groupby_sort(keys, vals, out_cap=a.m)
        torch.cuda.synchronize()
        print(f"profile case ok: sort group-by of {a.n} rows, {g['key'].numel()} groups")
        return
    if a.op == "strings":
        col = dg.gen_strings_device(dg.StringSpec(n=a.n, d=a.m, seed=1))
        for _ in range(a.runs):
            codes, rows = S.sirius_dict_encode(col["offsets"], col["chars"], distinct_hint=a.m)
        torch.cuda.synchronize()
        print(f"profile case ok: dictionary of {a.n} strings ({col['chars'].numel()} bytes), {rows.numel()} distinct")
        return
    if a.op == "operators":
        spec = dg.plain_scale(n=a.n, m=a.m)
        dim = dg.gen_dim_device(spec)
        fact = dg.gen_fact_device(spec, dim)
        for _ in range(a.runs):
            ids = S.sirius_filter(fact["pred"], "lt", spec.t)
            tab = S.sirius_hash_join_build(dim["pk"], load_factor=0.5)
            pp, pb = S.sirius_hash_join_probe(tab, fact["fk"], sel=ids)
            vals = S.sirius_gather(fact["val"], pp)
            keys = S.sirius_gather_group_key(dim["grp"], None, pb)
            g = S.sirius_groupby_agg(keys, vals, group_cap_hint=100_000)
        torch.cuda.synchronize()
        print(f"profile case ok: operators over n={spec.n} m={spec.m}: {ids.numel()} selected, "
              f"{pp.numel()} pairs, {g['key'].numel()} groups")
        return
    if a.batch > 0:
        specs = [dg.batch_query(q) for q in range(a.batch)]
        keep, descs = [], []
        for sp in specs:
            dim = dg.gen_dim_device(sp)
            fact = dg.gen_fact_device(sp, dim)
            keep.append((dim, fact))
            descs.append(S.make_desc(fact, dim, "lt", sp.t, group_cap_hint=1000))
        cap = S.lib().sirius_groupby_capacity(1000) + 1
        outs = [S.PipelineOutputs(cap) for _ in specs]
        plan = S.BatchPlan(a.batch)
        scratch = torch.empty(S.batch_scratch_bytes(descs), dtype=torch.uint8, device="cuda")
        for _ in range(a.runs):
            g = plan.run(descs, outs, scratch=scratch)
        torch.cuda.synchronize()
        print(f"profile case ok: batch of {a.batch} queries, {sum(s.n for s in specs)} fact rows, "
              f"{sum(g)} groups")
        return
    if a.workload == "plain_1M":   # the 1M-row / 65 536-row / 1 000-group query (sizes fixed)
        spec, hint = dg.plain_small(), 1000
    elif a.workload == "skewed":
        spec, hint = dg.skewed(n=a.n, m=a.m), a.m
    elif a.workload == "star":
        spec, hint = dg.star(n=a.n, m=a.m), 100_000
    else:
        spec, hint = dg.plain_scale(n=a.n, m=a.m, composite=a.workload == "composite"), 100_000
    dim = dg.gen_dim_device(spec)
    fact = dg.gen_fact_device(spec, dim)
    semi = dg.semi_args(spec, fact, dg.gen_semi_dims_device(spec)) if a.workload == "star" else None
    desc = S.make_desc(fact, dim, "lt", spec.t, spec.aggs, hint, a.load_factor, agg_mode=a.agg_mode,
                       probe_variant=a.variant, join_mode=a.join_mode, semi=semi)
    outs = S.PipelineOutputs(hint + 1)
    scratch = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device="cuda")
    for _ in range(a.runs):
        g = S.sirius_run_pipeline(desc, outs, scratch)
    torch.cuda.synchronize()
    print(f"profile case ok: n={spec.n} m={spec.m} variant={a.variant} groups={g}")


if __name__ == "__main__":
    main()
