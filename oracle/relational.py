"""Plain, slow, obviously correct CPU definition of the relational pipeline.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product path.

What it computes follows the paper's statement of the engine (Sec. 3.2.2): a query plan is a
pipeline of stateless physical operators -- a predicate filter, a hash join and a hash
group-by -- that the executor pushes columns through; filter and join outputs are row ids that
are materialised into columns only when a later operator needs them (the materialisation
kernel, Sec. 3.2.2; row ids as a distinct type, Sec. 3.2.3).  Sec. 4.2 names the same three
operators as where query time goes.  The paper prints no algorithm for any of them, so the
oracle is the plain relational definition, written out:

    R      = { (g(d), f.val) : f in fact, d in dim, f.pred <op> t, f.fk = d.pk }
    result = { (k, SUM val, COUNT(*), MIN val, MAX val) : k a group key with >= 1 row in R }

with SQL inner-join semantics (duplicate build keys multiply), groups without rows omitted,
and exact integer arithmetic (values are fixed-point decimals stored as int64).  Results are
returned sorted by key, the canonical order used for comparison; the operators themselves
promise no order except the filter, whose row ids ascend.

Library primitives used as steps: numpy comparison, nonzero, a stable sort, searchsorted and
ufunc reductions.  Python-loop versions (``*_loop``) exist for tiny inputs only.

Pins (tests/test_oracle_pins.py): brute-force loops, closed-form arithmetic series,
cardinality and sum invariants, special cases (empty, single group, no match) and planted
mistakes that the pins must catch.
"""
from __future__ import annotations

import operator
from typing import Dict, Optional, Tuple

import numpy as np

# comparison operators of the filter, by the C-ABI's enum order
OPS = ("lt", "le", "gt", "ge", "eq", "ne")
_NP_OPS = {"lt": np.less, "le": np.less_equal, "gt": np.greater, "ge": np.greater_equal,
           "eq": np.equal, "ne": np.not_equal}
_PY_OPS = {"lt": operator.lt, "le": operator.le, "gt": operator.gt, "ge": operator.ge,
           "eq": operator.eq, "ne": operator.ne}

INT64_MIN = -(1 << 63)
INT64_MAX = (1 << 63) - 1


# ------------------------------------------------------------------------------- filter
def filter_rows(col: np.ndarray, op: str, literal: int) -> np.ndarray:
    """Predicate filter (Sec. 3.2.2 predicate pushdown; Sec. 4.2 filter operator).

    Returns the ascending row ids i with ``col[i] <op> literal`` as uint32 (row ids are their
    own type, Sec. 3.2.3; this build narrows them to 32 bits and requires n < 2**32)."""
    col = np.asarray(col)
    assert col.shape[0] < (1 << 32)
    mask = _NP_OPS[op](col.astype(np.int64), np.int64(literal))
    return np.nonzero(mask)[0].astype(np.uint32)


def filter_rows_loop(col, op: str, literal: int) -> np.ndarray:
    """Tiny-input version of filter_rows: one Python comparison per row."""
    f = _PY_OPS[op]
    return np.array([i for i, v in enumerate(col) if f(int(v), int(literal))], dtype=np.uint32)


# ------------------------------------------------------------------------------- keys
def pack_composite(hi: np.ndarray, lo: np.ndarray) -> np.ndarray:
    """A two-column join key (hi, lo) of int32 words as one uint64: hi in the upper 32 bits."""
    hi = np.asarray(hi, dtype=np.int32).view(np.uint32).astype(np.uint64)
    lo = np.asarray(lo, dtype=np.int32).view(np.uint32).astype(np.uint64)
    return (hi << np.uint64(32)) | lo


def pack_group(grp: np.ndarray, flag: Optional[np.ndarray] = None) -> np.ndarray:
    """Group key as int64: grp itself, or (grp, flag) as grp * 256 + (flag as unsigned byte)."""
    g = np.asarray(grp, dtype=np.int32).astype(np.int64)
    if flag is None:
        return g
    f = np.asarray(flag, dtype=np.int8).view(np.uint8).astype(np.int64)
    return g * 256 + f


def join_key(cols: Dict[str, np.ndarray], lo: str, hi: str) -> np.ndarray:
    """The join key column of a table: one int32 column, or an (hi, lo) pair packed."""
    if cols.get(hi) is not None:
        return pack_composite(cols[hi], cols[lo])
    return np.asarray(cols[lo], dtype=np.int32).astype(np.int64)


# ------------------------------------------------------------------------------- join
def join_sorted(probe_keys: np.ndarray, build_keys: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Inner equi-join (Sec. 3.2.2 join operator; Sec. 4.2): every pair (i, j) with
    probe_keys[i] == build_keys[j], as (probe row ids, build row ids), sorted by (i, j).

    Realised with a stable sort of the build keys and a binary search of each probe key."""
    pk = np.asarray(probe_keys)
    bk = np.asarray(build_keys)
    if pk.shape[0] == 0 or bk.shape[0] == 0:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    order = np.argsort(bk, kind="stable")
    sb = bk[order]
    lo = np.searchsorted(sb, pk, side="left")
    hi = np.searchsorted(sb, pk, side="right")
    cnt = hi - lo
    probe_ids = np.repeat(np.arange(pk.shape[0], dtype=np.int64), cnt)
    # position of each output pair inside its probe row's run of matches
    starts = np.repeat(lo, cnt)
    offs = np.arange(probe_ids.shape[0], dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    build_ids = order[starts + offs]
    # canonical order: (probe row, build row)
    o = np.lexsort((build_ids, probe_ids))
    return probe_ids[o].astype(np.uint32), build_ids[o].astype(np.uint32)


def join_loop(probe_keys, build_keys) -> Tuple[np.ndarray, np.ndarray]:
    """Tiny-input inner equi-join: the nested loop over all (i, j)."""
    pi, bj = [], []
    for i, a in enumerate(probe_keys):
        for j, b in enumerate(build_keys):
            if int(a) == int(b):
                pi.append(i)
                bj.append(j)
    return np.array(pi, dtype=np.uint32), np.array(bj, dtype=np.uint32)


# ------------------------------------------------------------------------------- group-by
def groupby_agg(keys: np.ndarray, vals: np.ndarray) -> Dict[str, np.ndarray]:
    """Hash group-by aggregation (Sec. 3.2.2; Sec. 4.2 group-by): per distinct key the
    exact SUM, COUNT(*), MIN and MAX of vals, as int64 arrays sorted by key.

    Sums are exact: when n * max|val| could pass 2**63 they are formed in Python integers,
    and a sum that does not fit int64 raises OverflowError (precondition of the operator)."""
    keys = np.asarray(keys)
    if keys.dtype != np.uint64:
        keys = keys.astype(np.int64)
    vals = np.asarray(vals, dtype=np.int64)
    n = keys.shape[0]
    if n == 0:
        z = np.zeros(0, np.int64)
        return {"key": keys[:0].copy(), "sum": z, "count": z.copy(), "min": z.copy(),
                "max": z.copy()}
    order = np.argsort(keys, kind="stable")
    k = keys[order]
    v = vals[order]
    uniq, start = np.unique(k, return_index=True)
    count = np.diff(np.append(start, n)).astype(np.int64)
    vmax = max(abs(int(v.max())), abs(int(v.min())))
    if n * vmax < (1 << 63):
        s = np.add.reduceat(v, start)
    else:
        s_obj = [sum(int(x) for x in v[a:b]) for a, b in zip(start, np.append(start[1:], n))]
        if any(x < INT64_MIN or x > INT64_MAX for x in s_obj):
            raise OverflowError("a group's SUM does not fit int64")
        s = np.array(s_obj, dtype=np.int64)
    return {"key": uniq, "sum": s.astype(np.int64), "count": count,
            "min": np.minimum.reduceat(v, start).astype(np.int64),
            "max": np.maximum.reduceat(v, start).astype(np.int64)}


def groupby_loop(keys, vals) -> Dict[str, np.ndarray]:
    """Tiny-input group-by: a dict of running (sum, count, min, max) per key."""
    acc = {}
    for k, v in zip(keys, vals):
        k, v = int(k), int(v)
        if k not in acc:
            acc[k] = [0, 0, v, v]
        a = acc[k]
        a[0] += v
        a[1] += 1
        a[2] = min(a[2], v)
        a[3] = max(a[3], v)
    ks = sorted(acc)
    return {"key": np.array(ks, dtype=np.int64),
            "sum": np.array([acc[k][0] for k in ks], dtype=np.int64),
            "count": np.array([acc[k][1] for k in ks], dtype=np.int64),
            "min": np.array([acc[k][2] for k in ks], dtype=np.int64),
            "max": np.array([acc[k][3] for k in ks], dtype=np.int64)}


# ------------------------------------------------------------------------------- pipeline
def semi_keep(fact_keys: np.ndarray, dim: Dict[str, np.ndarray], op: Optional[str],
              literal: int) -> np.ndarray:
    """Semi-join: which fact keys equal the key of some dim row that passes attr <op> literal
    (every dim row when op is None)."""
    pk = join_key(dim, "pk", "pk_hi")
    if op is not None:
        pk = pk[filter_rows(dim["attr"], op, literal).astype(np.int64)]
    return np.isin(fact_keys, pk)


def pipeline(fact: Dict[str, np.ndarray], dim: Dict[str, np.ndarray], op: str = "lt",
             literal: int = 50, join: str = "sorted", dim_op: Optional[str] = None,
             dim_literal: int = 0, semi=None) -> Dict[str, np.ndarray]:
    """One pipeline of the push-based executor (Sec. 3.2.2): filter the fact rows, join the
    survivors to the dim on fk = pk, materialise the value and group key of each joined pair
    by row id (late materialisation), then group-by aggregate.

    fact: fk (int32, low word), fk_hi (optional high word), pred int32, val int64.
    dim:  pk (int32, low word), pk_hi (optional), grp int32, flag (optional int8), and dattr
          (int32) when dim_op is given: the dim-side predicate dattr <dim_op> dim_literal keeps
          the dim rows that take part in the join (a filter on the build side; moving it there
          from above the join is the predicate transfer of Sec. 3.4).
    semi: further dims joined as filters (a star query): a list of dicts {"fk": the fact's key
          column into the dim, "fk_hi"?, "dim": {"pk", "pk_hi"?, "attr"?}, "op", "literal"};
          a fact row takes part only if each of these keys has a partner (semi_keep).
    Group key: grp, or (grp, flag) packed by pack_group."""
    if dim_op is not None:
        keep = filter_rows(dim["dattr"], dim_op, dim_literal).astype(np.int64)
        dim = {k: (np.asarray(v)[keep] if v is not None else None) for k, v in dim.items()}
    sel = filter_rows(fact["pred"], op, literal).astype(np.int64)
    for sj in semi or []:
        keys = join_key({"fk": sj["fk"], "fk_hi": sj.get("fk_hi")}, "fk", "fk_hi")[sel]
        sel = sel[semi_keep(keys, sj["dim"], sj.get("op") if sj["dim"].get("attr") is not None else None,
                            sj.get("literal", 0))]
    fk = join_key(fact, "fk", "fk_hi")[sel]
    pk = join_key(dim, "pk", "pk_hi")
    jf = join_loop if join == "loop" else join_sorted
    p, b = jf(fk, pk)
    rows = sel[p.astype(np.int64)]
    gkey = pack_group(dim["grp"], dim.get("flag"))[b.astype(np.int64)]
    val = np.asarray(fact["val"], dtype=np.int64)[rows]
    gb = groupby_loop if join == "loop" else groupby_agg
    return gb(gkey, val)


# ------------------------------------------------------------------------------- top N
def topn(keys: np.ndarray, order: np.ndarray, n: int, descending: bool = True) -> np.ndarray:
    """ORDER BY order DESC|ASC, key ASC LIMIT n over group-by outputs: the positions of the
    first n groups (Python's sort on exact integers)."""
    sign = -1 if descending else 1
    idx = sorted(range(len(keys)), key=lambda i: (sign * int(order[i]), int(keys[i])))
    return np.asarray(idx[:n], dtype=np.int64)


def merge_partials(parts) -> Dict[str, np.ndarray]:
    """Combine group-by results of disjoint row chunks: SUM and COUNT add, MIN and MAX take
    the extreme (all four aggregates are distributive)."""
    acc: Dict[int, list] = {}
    for r in parts:
        for k, s, c, mn, mx in zip(r["key"].tolist(), r["sum"].tolist(), r["count"].tolist(),
                                   r["min"].tolist(), r["max"].tolist()):
            a = acc.get(k)
            if a is None:
                acc[k] = [s, c, mn, mx]
            else:
                a[0] += s
                a[1] += c
                a[2] = min(a[2], mn)
                a[3] = max(a[3], mx)
    ks = sorted(acc)
    return {"key": np.array(ks, dtype=np.int64),
            "sum": np.array([acc[k][0] for k in ks], dtype=np.int64),
            "count": np.array([acc[k][1] for k in ks], dtype=np.int64),
            "min": np.array([acc[k][2] for k in ks], dtype=np.int64),
            "max": np.array([acc[k][3] for k in ks], dtype=np.int64)}


def restrict_dim(dim: Dict[str, np.ndarray], group_keys) -> Dict[str, np.ndarray]:
    """The dim rows whose group key is in group_keys.  Selecting groups before the join gives
    exactly those groups' rows of the full result (the join and the group-by act row by row),
    which lets a full-size result be checked one sampled group at a time."""
    gk = pack_group(dim["grp"], dim.get("flag"))
    keep = np.isin(gk, np.asarray(list(group_keys), dtype=np.int64))
    return {k: (v[keep] if v is not None else None) for k, v in dim.items()}


def sort_pairs(probe_ids, build_ids) -> Tuple[np.ndarray, np.ndarray]:
    """Canonical (probe row, build row) order for comparing unordered join outputs."""
    p = np.asarray(probe_ids).astype(np.int64)
    b = np.asarray(build_ids).astype(np.int64)
    o = np.lexsort((b, p))
    return p[o].astype(np.uint32), b[o].astype(np.uint32)


def sort_groups(res: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
    """Canonical order (by key) for comparing unordered group-by outputs."""
    o = np.argsort(np.asarray(res["key"]), kind="stable")
    return {k: np.asarray(v)[o] for k, v in res.items()}


__all__ = ["OPS", "filter_rows", "filter_rows_loop", "pack_composite", "pack_group", "semi_keep", "topn",
           "join_key", "join_sorted", "join_loop", "groupby_agg", "groupby_loop", "pipeline",
           "merge_partials", "restrict_dim", "sort_pairs", "sort_groups"]
