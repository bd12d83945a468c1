"""Python binding of libsirius (include/sirius.h): the same entry points, argument marshalling
only.  Device memory and streams come from PyTorch; every step of the work runs in the
library's CUDA kernels.  Loading fails loudly when the library is missing -- there is no CPU
path.

Entry points take torch tensors (device memory) and return Python values; a non-OK status
raises SiriusError carrying the status code and the library's message.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsirius.so")

OK, ERR_INVALID, ERR_OOM, ERR_CAPACITY, ERR_TABLE_FULL, ERR_TIMEOUT, ERR_CUDA, ERR_SCRATCH = range(8)
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CAPACITY", 4: "TABLE_FULL", 5: "TIMEOUT",
                6: "CUDA", 7: "SCRATCH"}
LT, LE, GT, GE, EQ, NE = range(6)
OPS = {"lt": LT, "le": LE, "gt": GT, "ge": GE, "eq": EQ, "ne": NE}
AGG_SUM, AGG_COUNT, AGG_MIN, AGG_MAX, AGG_ALL = 1, 2, 4, 8, 15
AGG_MODES = {"auto": 0, "smem": 1, "global": 2, "part": 3, "hot": 4, "routed": 5}
PROBE_VARIANTS = {"auto": 0, "direct": 1, "staged": 2, "single": 3}
BLOOM_MODES = {"auto": 0, "off": 1, "on": 2}
JOIN_MODES = {"auto": 0, "hash": 1}
SPLIT_MODES = {"auto": 0, "off": 1, "on": 2}


class SiriusError(RuntimeError):
    def __init__(self, status: int, msg: str, needed: Optional[int] = None):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
        self.needed = needed


class Semijoin(ctypes.Structure):
    _fields_ = [("fk", ctypes.c_void_p), ("fk_hi", ctypes.c_void_p), ("pk", ctypes.c_void_p),
                ("pk_hi", ctypes.c_void_p), ("attr", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("op", ctypes.c_int32), ("literal", ctypes.c_int32)]


MAX_SEMIJOINS = 3


class PipelineDesc(ctypes.Structure):
    _fields_ = [("fk", ctypes.c_void_p), ("fk_hi", ctypes.c_void_p), ("pred", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("pk", ctypes.c_void_p), ("pk_hi", ctypes.c_void_p), ("grp", ctypes.c_void_p),
                ("flag", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("op", ctypes.c_int32), ("literal", ctypes.c_int32), ("aggs", ctypes.c_uint32),
                ("agg_mode", ctypes.c_int32), ("group_cap_hint", ctypes.c_int64),
                ("load_factor", ctypes.c_float), ("block_threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("probe_variant", ctypes.c_int32),
                ("join_mode", ctypes.c_int32), ("split_probe", ctypes.c_int32),
                ("dpred", ctypes.c_void_p), ("dop", ctypes.c_int32), ("dliteral", ctypes.c_int32),
                ("bloom", ctypes.c_int32), ("nsemi", ctypes.c_int32),
                ("semi", Semijoin * MAX_SEMIJOINS)]


class Result(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("sum", ctypes.c_void_p), ("count", ctypes.c_void_p),
                ("min", ctypes.c_void_p), ("max", ctypes.c_void_p), ("out_cap", ctypes.c_int64),
                ("d_groups", ctypes.c_void_p), ("d_status", ctypes.c_void_p),
                ("sync", ctypes.c_int32), ("status", ctypes.c_int32), ("groups", ctypes.c_int64)]


class JoinTable(ctypes.Structure):
    _fields_ = [("d_mem", ctypes.c_void_p), ("capacity", ctypes.c_int64),
                ("key_width", ctypes.c_int32), ("probe_variant", ctypes.c_int32)]


class DimIndex(ctypes.Structure):
    _fields_ = [("d_mem", ctypes.c_void_p), ("bytes", ctypes.c_size_t),
                ("join_capacity", ctypes.c_int64), ("group_capacity", ctypes.c_int64),
                ("direct_capacity", ctypes.c_int64),
                ("key_width", ctypes.c_int32), ("bloom_log2", ctypes.c_int32)]


# (name, restype, argtypes) of every exported function
_VP, _I32, _I64, _U32, _U64, _SZ, _F64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                          ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t,
                                          ctypes.c_double)
SIGNATURES = {
    "sirius_version": (_I32, []),
    "sirius_last_error": (ctypes.c_char_p, []),
    "sirius_launch_count": (_U64, []),
    "sirius_device_sm_count": (_I32, []),
    "sirius_profile_start": (None, []),
    "sirius_profile_stop": (_I32, [_VP, _VP, _I32]),
    "sirius_filter_scratch_bytes": (_SZ, [_I64]),
    "sirius_filter": (_I32, [_VP, _I64, _I32, _I32, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "sirius_filter_static_max_rows": (_I64, []),
    "sirius_inject_alloc_failures": (_I32, [_I32]),
    "sirius_filter_static": (_I32, [_VP, _I64, _I32, _I32, _VP, _VP, _VP, _VP]),
    "sirius_join_table_capacity": (_I64, [_I64, _F64]),
    "sirius_join_table_bytes": (_SZ, [_I64, _I32]),
    "sirius_hash_join_build": (_I32, [_VP, _VP, _I64, ctypes.POINTER(JoinTable), _VP, _VP]),
    "sirius_hash_join_probe": (_I32, [ctypes.POINTER(JoinTable), _VP, _VP, _VP, _I64, _VP, _VP,
                                      _I64, _VP, _VP, _VP]),
    "sirius_gather_i32": (_I32, [_VP, _VP, _I64, _VP, _VP]),
    "sirius_gather_i64": (_I32, [_VP, _VP, _I64, _VP, _VP]),
    "sirius_gather_group_key": (_I32, [_VP, _VP, _VP, _I64, _VP, _VP]),
    "sirius_groupby_capacity": (_I64, [_I64]),
    "sirius_topn_scratch_bytes": (_SZ, [_I64]),
    "sirius_groupby_sort_scratch_bytes": (_SZ, [_I64]),
    "sirius_groupby_sort": (_I32, [_VP, _I32, _VP, _I64, _U32, _VP, _VP, _VP, _VP, _VP, _I64, _VP, _VP,
                                   _VP, _SZ, _VP]),
    "sirius_topn_groups": (_I32, [_VP, _VP, _I64, _I32, _I64, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "sirius_dict_capacity": (_I64, [_I64]),
    "sirius_dict_scratch_bytes": (_SZ, [_I64, _I64]),
    "sirius_dict_encode": (_I32, [_VP, _VP, _I64, _I64, _I64, _U32, _VP, _VP, _I64, _VP, _VP, _VP, _SZ,
                                  _VP]),
    "sirius_groupby_string_scratch_bytes": (_SZ, [_I64, _I64]),
    "sirius_groupby_string": (_I32, [_VP, _VP, _I64, _VP, _I64, _I64, _U32, _U32, _VP, _VP, _VP, _VP, _VP,
                                     _I64, _VP, _VP, _VP, _SZ, _VP]),
    "sirius_groupby_scratch_bytes": (_SZ, [_I64]),
    "sirius_groupby_agg": (_I32, [_VP, _I32, _VP, _I64, _U32, _I64, _VP, _VP, _VP, _VP, _VP,
                                  _I64, _VP, _VP, _VP, _SZ, _VP]),
    "sirius_pipeline_scratch_bytes": (_SZ, [ctypes.POINTER(PipelineDesc)]),
    "sirius_run_pipeline": (_I32, [ctypes.POINTER(PipelineDesc), ctypes.POINTER(Result), _VP, _SZ,
                                   _VP]),
    "sirius_dim_index_bytes": (_SZ, [ctypes.POINTER(PipelineDesc)]),
    "sirius_dim_index_build": (_I32, [ctypes.POINTER(PipelineDesc), ctypes.POINTER(DimIndex), _VP,
                                      _VP]),
    "sirius_probe_scratch_bytes": (_SZ, [ctypes.POINTER(PipelineDesc), ctypes.POINTER(DimIndex)]),
    "sirius_run_probe": (_I32, [ctypes.POINTER(PipelineDesc), ctypes.POINTER(DimIndex),
                                ctypes.POINTER(Result), _VP, _SZ, _VP]),
    "sirius_pipeline_host_scratch_bytes": (_SZ, [ctypes.POINTER(PipelineDesc), _I64, _I64]),
    "sirius_run_pipeline_host": (_I32, [ctypes.POINTER(PipelineDesc), ctypes.POINTER(Result), _I64,
                                        _VP, _SZ, _VP]),
    "sirius_pipeline_batch_scratch_bytes": (_SZ, [ctypes.POINTER(PipelineDesc), _I32,
                                                  ctypes.POINTER(DimIndex)]),
    "sirius_batch_plan_create": (_I32, [_I32, ctypes.POINTER(ctypes.c_void_p)]),
    "sirius_batch_plan_run": (_I32, [_VP, ctypes.POINTER(PipelineDesc), _I32, ctypes.POINTER(DimIndex),
                                     ctypes.POINTER(Result), _I64, _I32, _VP, _SZ, _VP]),
    "sirius_batch_plan_destroy": (None, [_VP]),
    "sirius_run_pipeline_batch": (_I32, [ctypes.POINTER(PipelineDesc), _I32, ctypes.POINTER(DimIndex),
                                         ctypes.POINTER(Result), _VP, _SZ, _VP]),
    "sirius_selftest_lookback_timeout": (_I32, [_VP, _SZ, _VP, _VP]),
    "sirius_selftest_grid_barrier": (_I32, [_I32, _I32, _U32, _VP, _SZ, _VP, _VP, _VP]),
}

_LIB = None


def lib() -> ctypes.CDLL:
    """The loaded libsirius.so; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no fallback path)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def last_error() -> str:
    return lib().sirius_last_error().decode()


def _check(st: int, needed: Optional[int] = None):
    if st != OK:
        raise SiriusError(st, last_error(), needed)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libsirius takes device tensors")
    if not t.is_contiguous():
        raise ValueError("libsirius takes contiguous columns")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _scratch(nbytes: int, device) -> torch.Tensor:
    # torch allocations are 512-byte aligned; one extra page keeps the size non-zero
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def launch_count() -> int:
    return int(lib().sirius_launch_count())


PHASES = ["filter", "join_build", "join_probe", "gather", "groupby", "pipe_init", "pipe_build",
          "pipe_probe", "pipe_finalize", "batch_graph", "batch_build", "batch_probe",
          "batch_finalize", "copy", "pipe_aggregate", "pipe_single"]


def profile_start():
    lib().sirius_profile_start()


def profile_stop() -> Dict[str, tuple]:
    """{phase: (total ms, launches)} for the phases that ran since profile_start()."""
    ms = (ctypes.c_double * 16)()
    n = (ctypes.c_int64 * 16)()
    _check(lib().sirius_profile_stop(ms, n, 16))
    return {PHASES[i]: (ms[i], n[i]) for i in range(16) if n[i]}


# ---------------------------------------------------------------------------- A2: filter
def sirius_filter(col: torch.Tensor, op="lt", literal: int = 0, out: Optional[torch.Tensor] = None,
                  stream=None, scratch: Optional[torch.Tensor] = None, sync: bool = True):
    """Ascending row ids of col <op> literal.  Returns the row-id tensor trimmed to the count
    (sync=True), or (out, d_count) without synchronising."""
    n = col.numel()
    if col.dtype != torch.int32:
        raise TypeError("filter column must be int32")
    op = OPS[op] if isinstance(op, str) else int(op)
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.int32, device=col.device)
    d_count = torch.zeros(1, dtype=torch.int64, device=col.device)
    if scratch is None:
        scratch = _scratch(lib().sirius_filter_scratch_bytes(n), col.device)
    h = ctypes.c_int64(0)
    st = lib().sirius_filter(_ptr(col), n, op, int(literal), _ptr(out), _ptr(d_count),
                             ctypes.byref(h) if sync else None, _ptr(scratch), scratch.numel(),
                             _stream(stream))
    _check(st)
    if sync:
        return out[:h.value]
    return out, d_count


# ---------------------------------------------------------------------------- A1/A3: join
class HashJoinTable:
    """A join table in a torch-owned device buffer."""

    def __init__(self, m: int, key_width: int = 4, load_factor: float = 0.5, device="cuda",
                 probe_variant: int = 0):
        cap = lib().sirius_join_table_capacity(m, load_factor)
        nbytes = lib().sirius_join_table_bytes(cap, key_width)
        self.mem = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.struct = JoinTable(self.mem.data_ptr(), cap, key_width, int(probe_variant))
        self.has_dups = None

    @property
    def capacity(self) -> int:
        return self.struct.capacity


def sirius_hash_join_build(keys: torch.Tensor, keys_hi: Optional[torch.Tensor] = None,
                           load_factor: float = 0.5, table: Optional[HashJoinTable] = None,
                           stream=None) -> HashJoinTable:
    m = keys.numel()
    if table is None:
        table = HashJoinTable(m, 8 if keys_hi is not None else 4, load_factor, keys.device)
    d = ctypes.c_int32(0)
    st = lib().sirius_hash_join_build(_ptr(keys), _ptr(keys_hi), m, ctypes.byref(table.struct),
                                      ctypes.byref(d), _stream(stream))
    _check(st)
    table.has_dups = bool(d.value)
    return table


def sirius_hash_join_probe(table: HashJoinTable, keys: torch.Tensor,
                           keys_hi: Optional[torch.Tensor] = None,
                           sel: Optional[torch.Tensor] = None, out_cap: Optional[int] = None,
                           stream=None):
    """All (probe row, build row) pairs with equal keys, unordered, as two int32 tensors
    (uint32 bit patterns).  Retries once with the exact size when out_cap is too small."""
    n = sel.numel() if sel is not None else keys.numel()
    if out_cap is None:
        out_cap = n
    while True:
        op_ = torch.empty(max(out_cap, 1), dtype=torch.int32, device=keys.device)
        ob = torch.empty(max(out_cap, 1), dtype=torch.int32, device=keys.device)
        h = ctypes.c_int64(0)
        st = lib().sirius_hash_join_probe(ctypes.byref(table.struct), _ptr(keys), _ptr(keys_hi),
                                          _ptr(sel), n, _ptr(op_), _ptr(ob), out_cap, None,
                                          ctypes.byref(h), _stream(stream))
        if st == ERR_CAPACITY:
            out_cap = h.value
            continue
        _check(st)
        return op_[:h.value], ob[:h.value]


# ---------------------------------------------------------------------------- A4: gather
def sirius_gather(src: torch.Tensor, idx: torch.Tensor, stream=None) -> torch.Tensor:
    n = idx.numel()
    dst = torch.empty(n, dtype=src.dtype, device=src.device)
    if src.dtype == torch.int32:
        st = lib().sirius_gather_i32(_ptr(src), _ptr(idx), n, _ptr(dst), _stream(stream))
    elif src.dtype == torch.int64:
        st = lib().sirius_gather_i64(_ptr(src), _ptr(idx), n, _ptr(dst), _stream(stream))
    else:
        raise TypeError("gather supports int32 and int64 columns")
    _check(st)
    return dst


def sirius_topn_groups(keys: torch.Tensor, order: torch.Tensor, n_top: int, descending: bool = True,
                       scratch: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Positions (int32 tensor, best first) of the n_top groups by (order, key): ORDER BY order
    DESC|ASC, key ASC LIMIT n_top over group-by outputs; gather columns with sirius_gather."""
    g = keys.numel()
    out = torch.empty(max(min(n_top, g), 1), dtype=torch.int32, device=keys.device)
    if scratch is None:
        scratch = _scratch(int(lib().sirius_topn_scratch_bytes(n_top)), keys.device)
    cnt = ctypes.c_int64(0)
    _check(lib().sirius_topn_groups(_ptr(keys) if g else None, _ptr(order) if g else None, g,
                                    1 if descending else 0, int(n_top), _ptr(out), None, ctypes.byref(cnt),
                                    _ptr(scratch), scratch.numel(), _stream(stream)))
    return out[:cnt.value]


def sirius_gather_group_key(grp: torch.Tensor, flag: Optional[torch.Tensor], idx: torch.Tensor,
                            stream=None) -> torch.Tensor:
    n = idx.numel()
    dst = torch.empty(n, dtype=torch.int64, device=grp.device)
    _check(lib().sirius_gather_group_key(_ptr(grp), _ptr(flag), _ptr(idx), n, _ptr(dst),
                                         _stream(stream)))
    return dst


# ---------------------------------------------------------------------------- A5/A6: group-by
def _agg_mask(aggs) -> int:
    if isinstance(aggs, int):
        return aggs
    m = 0
    for a in aggs.split(","):
        m |= {"sum": AGG_SUM, "count": AGG_COUNT, "min": AGG_MIN, "max": AGG_MAX}[a.strip()]
    return m


def groupby_outputs(out_cap: int, device="cuda") -> Dict[str, torch.Tensor]:
    """Output arrays for sirius_groupby_agg / sirius_groupby_sort (out_cap groups each) and the
    device group count ("groups", one int64)."""
    outs = {c: torch.empty(max(out_cap, 1), dtype=torch.int64, device=device)
            for c in ("key", "sum", "count", "min", "max")}
    outs["groups"] = torch.zeros(1, dtype=torch.int64, device=device)
    return outs


def sirius_groupby_agg(keys: torch.Tensor, vals: torch.Tensor, aggs="sum,count,min,max",
                       group_cap_hint: int = 1024, out_cap: Optional[int] = None,
                       stream=None, outputs: Optional[Dict[str, torch.Tensor]] = None,
                       scratch: Optional[torch.Tensor] = None, sync: bool = True):
    """Hash group-by.  sync=True: returns the trimmed group arrays (reads G back); sync=False:
    returns nothing and leaves G in outputs["groups"] (no host synchronisation).  outputs /
    scratch: preallocated (groupby_outputs, sirius_groupby_scratch_bytes) to avoid allocating
    per call."""
    n = keys.numel()
    kw = {torch.int32: 4, torch.int64: 8}[keys.dtype]
    mask = _agg_mask(aggs)
    dev = keys.device
    if outputs is None:
        if out_cap is None:
            out_cap = lib().sirius_groupby_capacity(group_cap_hint) + 1
        outputs = groupby_outputs(out_cap, dev)
    outs = outputs
    out_cap = outs["key"].numel()
    if scratch is None:
        scratch = _scratch(lib().sirius_groupby_scratch_bytes(group_cap_hint), dev)
    h = ctypes.c_int64(0)
    st = lib().sirius_groupby_agg(
        _ptr(keys), kw, _ptr(vals), n, mask, group_cap_hint, _ptr(outs["key"]),
        _ptr(outs["sum"]) if mask & AGG_SUM else None, _ptr(outs["count"]),
        _ptr(outs["min"]) if mask & AGG_MIN else None,
        _ptr(outs["max"]) if mask & AGG_MAX else None, out_cap, _ptr(outs.get("groups")),
        ctypes.byref(h) if sync else None, _ptr(scratch), scratch.numel(), _stream(stream))
    _check(st, h.value)
    if not sync:
        return None
    g = h.value
    return {c: outs[c][:g] for c in ("key", "sum", "count", "min", "max")}


def sirius_groupby_sort(keys: torch.Tensor, vals: torch.Tensor, aggs="sum,count,min,max",
                        out_cap: Optional[int] = None, stream=None) -> Dict[str, torch.Tensor]:
    """The sort-based group-by: the same results as sirius_groupby_agg, groups in ascending
    key order.  out_cap defaults to the row count (every key distinct at worst)."""
    n = keys.numel()
    kw = {torch.int32: 4, torch.int64: 8}[keys.dtype]
    mask = _agg_mask(aggs)
    if out_cap is None:
        out_cap = max(n, 1)
    dev = keys.device
    outs = {c: torch.empty(max(out_cap, 1), dtype=torch.int64, device=dev)
            for c in ("key", "sum", "count", "min", "max")}
    scratch = _scratch(lib().sirius_groupby_sort_scratch_bytes(n), dev)
    h = ctypes.c_int64(0)
    st = lib().sirius_groupby_sort(
        _ptr(keys) if n else None, kw, _ptr(vals) if n else None, n, mask, _ptr(outs["key"]),
        _ptr(outs["sum"]) if mask & AGG_SUM else None, _ptr(outs["count"]),
        _ptr(outs["min"]) if mask & AGG_MIN else None,
        _ptr(outs["max"]) if mask & AGG_MAX else None, out_cap, None, ctypes.byref(h),
        _ptr(scratch), scratch.numel(), _stream(stream))
    _check(st, h.value)
    g = h.value
    return {c: t[:g] for c, t in outs.items()}


# ---------------------------------------------------------------------------- string keys
DICT_WEAK_HASH = 1


def _strcol(offsets: torch.Tensor, chars: torch.Tensor):
    if offsets.dtype != torch.int32 or chars.dtype != torch.uint8:
        raise ValueError("a string column is int32 offsets (n + 1) and uint8 chars")
    if offsets.numel() < 1:
        raise ValueError("offsets hold n + 1 entries")
    return offsets.numel() - 1, chars.numel()


def sirius_dict_encode(offsets: torch.Tensor, chars: torch.Tensor, distinct_hint: int = 1024,
                       weak_hash: bool = False, dict_cap: Optional[int] = None, stream=None):
    """Codes of a string column in order of first occurrence: (codes int32[n], dict_rows
    int64[D]) with dict_rows[c] the first row holding string c."""
    n, n_chars = _strcol(offsets, chars)
    dev = offsets.device
    if dict_cap is None:
        dict_cap = int(lib().sirius_dict_capacity(distinct_hint))
    codes = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    rows = torch.empty(max(dict_cap, 1), dtype=torch.int64, device=dev)
    scratch = _scratch(lib().sirius_dict_scratch_bytes(n, distinct_hint), dev)
    h = ctypes.c_int64(0)
    st = lib().sirius_dict_encode(_ptr(offsets), _ptr(chars) if n_chars else None, n_chars, n, distinct_hint,
                                  DICT_WEAK_HASH if weak_hash else 0, _ptr(codes), _ptr(rows), dict_cap, None,
                                  ctypes.byref(h), _ptr(scratch), scratch.numel(), _stream(stream))
    _check(st, h.value)
    return codes[:n], rows[:h.value]


def sirius_groupby_string(offsets: torch.Tensor, chars: torch.Tensor, vals: torch.Tensor,
                          aggs="sum,count,min,max", distinct_hint: int = 1024, weak_hash: bool = False,
                          out_cap: Optional[int] = None, stream=None) -> Dict[str, torch.Tensor]:
    """GROUP BY a string column, groups in order of first occurrence: 'row' (the first row
    holding the group's string), 'sum', 'count', 'min', 'max'."""
    n, n_chars = _strcol(offsets, chars)
    mask = _agg_mask(aggs)
    dev = offsets.device
    if out_cap is None:
        out_cap = int(lib().sirius_dict_capacity(distinct_hint))
    outs = {c: torch.empty(max(out_cap, 1), dtype=torch.int64, device=dev)
            for c in ("row", "sum", "count", "min", "max")}
    scratch = _scratch(lib().sirius_groupby_string_scratch_bytes(n, distinct_hint), dev)
    h = ctypes.c_int64(0)
    st = lib().sirius_groupby_string(
        _ptr(offsets), _ptr(chars) if n_chars else None, n_chars, _ptr(vals) if n else None, n, distinct_hint,
        DICT_WEAK_HASH if weak_hash else 0, mask, _ptr(outs["row"]),
        _ptr(outs["sum"]) if mask & AGG_SUM else None, _ptr(outs["count"]),
        _ptr(outs["min"]) if mask & AGG_MIN else None, _ptr(outs["max"]) if mask & AGG_MAX else None,
        out_cap, None, ctypes.byref(h), _ptr(scratch), scratch.numel(), _stream(stream))
    _check(st, h.value)
    return {c: t[:h.value] for c, t in outs.items()}


# ---------------------------------------------------------------------------- A7: pipeline
def _host_ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("host columns must be contiguous CPU tensors (pinned for full speed)")
    return t.data_ptr()


def make_desc(fact: Dict[str, torch.Tensor], dim: Dict[str, torch.Tensor], op="lt",
              literal: int = 50, aggs="sum,count,min,max", group_cap_hint: int = 0,
              load_factor: float = 0.0, agg_mode="auto", block_threads: int = 0,
              blocks_per_sm: int = 0, host: bool = False, probe_variant="auto",
              join_mode="auto", dim_op=None, dim_literal: int = 0, bloom="auto",
              semi=None, split_probe="auto") -> PipelineDesc:
    """A pipeline descriptor over device columns (host=True: over host columns, for
    sirius_run_pipeline_host).  fact: fk, fk_hi?, pred, val; dim: pk, pk_hi?, grp, flag?, and
    dattr when dim_op is given (the dim-side predicate dattr <dim_op> dim_literal).
    semi: up to MAX_SEMIJOINS further dims joined as filters (a star query), each a dict
    {"fk": fact key column, "fk_hi"?, "dim": {"pk", "pk_hi"?, "attr"?}, "op", "literal"}."""
    P = _host_ptr if host else _ptr
    g = lambda d, k: P(d.get(k)) if d.get(k) is not None else None  # noqa: E731
    d = PipelineDesc(
        g(fact, "fk"), g(fact, "fk_hi"), g(fact, "pred"), g(fact, "val"), fact["pred"].numel(),
        g(dim, "pk"), g(dim, "pk_hi"), g(dim, "grp"), g(dim, "flag"), dim["pk"].numel(),
        OPS[op] if isinstance(op, str) else int(op), int(literal), _agg_mask(aggs),
        AGG_MODES[agg_mode] if isinstance(agg_mode, str) else int(agg_mode), int(group_cap_hint),
        float(load_factor), int(block_threads), int(blocks_per_sm),
        PROBE_VARIANTS[probe_variant] if isinstance(probe_variant, str) else int(probe_variant),
        JOIN_MODES[join_mode] if isinstance(join_mode, str) else int(join_mode),
        SPLIT_MODES[split_probe] if isinstance(split_probe, str) else int(split_probe),
        g(dim, "dattr") if dim_op is not None else None,
        (OPS[dim_op] if isinstance(dim_op, str) else int(dim_op)) if dim_op is not None else 0,
        int(dim_literal), BLOOM_MODES[bloom] if isinstance(bloom, str) else int(bloom), 0)
    semi = list(semi or [])
    if len(semi) > MAX_SEMIJOINS:
        raise ValueError(f"at most {MAX_SEMIJOINS} semi-join dims")
    keep = []
    for i, sj in enumerate(semi):
        sd = sj["dim"]
        d.semi[i] = Semijoin(P(sj["fk"]), P(sj.get("fk_hi")) if sj.get("fk_hi") is not None else None,
                             g(sd, "pk"), g(sd, "pk_hi"), g(sd, "attr"), sd["pk"].numel(),
                             OPS[sj.get("op", "lt")], int(sj.get("literal", 0)))
        keep.append((sj["fk"], sj.get("fk_hi"), dict(sd)))
    d.nsemi = len(semi)
    # the descriptor holds raw pointers: keep the tensors they point into alive with it
    d._columns = (dict(fact), dict(dim), keep)
    return d


def pipeline_scratch_bytes(desc: PipelineDesc) -> int:
    return int(lib().sirius_pipeline_scratch_bytes(ctypes.byref(desc)))


class PipelineOutputs:
    """Device output arrays for one pipeline result."""

    def __init__(self, out_cap: int, device="cuda"):
        self.cap = out_cap
        self.t = {c: torch.empty(max(out_cap, 1), dtype=torch.int64, device=device)
                  for c in ("key", "sum", "count", "min", "max")}
        self.d_groups = torch.zeros(1, dtype=torch.int64, device=device)
        self.d_status = torch.zeros(1, dtype=torch.int32, device=device)

    def result(self, sync: bool) -> Result:
        t = self.t
        return Result(t["key"].data_ptr(), t["sum"].data_ptr(), t["count"].data_ptr(),
                      t["min"].data_ptr(), t["max"].data_ptr(), self.cap,
                      self.d_groups.data_ptr(), self.d_status.data_ptr(), 1 if sync else 0, 0, 0)

    def trimmed(self, g: int) -> Dict[str, torch.Tensor]:
        return {c: v[:g] for c, v in self.t.items()}


def sirius_run_pipeline(desc: PipelineDesc, outputs: PipelineOutputs,
                        scratch: Optional[torch.Tensor] = None, stream=None, sync: bool = True):
    """Runs one fused pipeline.  sync=True: returns G (raises on a device error); sync=False:
    returns None and leaves G / status in outputs.d_groups / outputs.d_status."""
    r = outputs.result(sync)
    if scratch is None:
        scratch = _scratch(pipeline_scratch_bytes(desc), outputs.d_groups.device)
    st = lib().sirius_run_pipeline(ctypes.byref(desc), ctypes.byref(r), _ptr(scratch),
                                   scratch.numel(), _stream(stream))
    _check(st, r.groups)
    return r.groups if sync else None


def run_pipeline(fact, dim, op="lt", literal=50, aggs="sum,count,min,max", group_cap_hint=0,
                 out_cap=None, **tuning) -> Dict[str, torch.Tensor]:
    """One query end to end on device tensors; returns the trimmed group arrays."""
    desc = make_desc(fact, dim, op, literal, aggs, group_cap_hint, **tuning)
    if out_cap is None:
        out_cap = max(1, group_cap_hint or dim["pk"].numel())
    outs = PipelineOutputs(out_cap, fact["pred"].device)
    g = sirius_run_pipeline(desc, outs)
    return outs.trimmed(g)


# ---------------------------------------------------------------------------- resident build side
class DimIndexBuffer:
    """A built dim index (join table + group keys) in a torch-owned device buffer."""

    def __init__(self, desc: PipelineDesc, device="cuda", stream=None):
        nbytes = int(lib().sirius_dim_index_bytes(ctypes.byref(desc)))
        self.mem = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        self.struct = DimIndex(self.mem.data_ptr(), self.mem.numel(), 0, 0, 0, 0, 0)
        st = ctypes.c_int32(0)
        _check(lib().sirius_dim_index_build(ctypes.byref(desc), ctypes.byref(self.struct),
                                            ctypes.byref(st), _stream(stream)))

    @property
    def nbytes(self) -> int:
        return self.mem.numel()

    def probe_scratch_bytes(self, desc: PipelineDesc) -> int:
        """Scratch of one probe pass of `desc` (its fact rows and aggregation mode) against
        this index."""
        return int(lib().sirius_probe_scratch_bytes(ctypes.byref(desc), ctypes.byref(self.struct)))

    def join_kind(self) -> str:
        """'direct' when the build took the direct-address array, else 'hash' (reads the
        index header: int32 status, uint32 direct at byte 4, uint32 direct_failed at byte 24)."""
        h = self.mem[:32].cpu().numpy().view("uint32")
        return "direct" if h[1] and not h[6] else "hash"


def sirius_dim_index_build(desc: PipelineDesc, device="cuda", stream=None) -> DimIndexBuffer:
    return DimIndexBuffer(desc, device, stream)


def sirius_run_probe(desc: PipelineDesc, index: DimIndexBuffer, outputs: PipelineOutputs,
                     scratch: Optional[torch.Tensor] = None, stream=None, sync: bool = True):
    r = outputs.result(sync)
    if scratch is None:
        scratch = _scratch(index.probe_scratch_bytes(desc), outputs.d_groups.device)
    st = lib().sirius_run_probe(ctypes.byref(desc), ctypes.byref(index.struct), ctypes.byref(r),
                                _ptr(scratch), scratch.numel(), _stream(stream))
    _check(st, r.groups)
    return r.groups if sync else None


# ---------------------------------------------------------------------------- host-resident columns
class HostOutputs:
    """Pinned host arrays receiving one pipeline result from sirius_run_pipeline_host."""

    def __init__(self, out_cap: int):
        self.cap = out_cap
        self.t = {c: torch.empty(max(out_cap, 1), dtype=torch.int64, pin_memory=True)
                  for c in ("key", "sum", "count", "min", "max")}

    def result(self) -> Result:
        t = self.t
        return Result(t["key"].data_ptr(), t["sum"].data_ptr(), t["count"].data_ptr(),
                      t["min"].data_ptr(), t["max"].data_ptr(), self.cap, None, None, 1, 0, 0)

    def trimmed(self, g: int) -> Dict[str, torch.Tensor]:
        return {c: v[:g] for c, v in self.t.items()}


def pipeline_host_scratch_bytes(desc: PipelineDesc, chunk_rows: int, out_cap: int) -> int:
    return int(lib().sirius_pipeline_host_scratch_bytes(ctypes.byref(desc), chunk_rows, out_cap))


def sirius_run_pipeline_host(desc: PipelineDesc, outputs: HostOutputs, chunk_rows: int = 0,
                             scratch: Optional[torch.Tensor] = None, stream=None,
                             device="cuda") -> int:
    """One query over host columns (desc made with host=True); synchronises; returns G."""
    r = outputs.result()
    if scratch is None:
        scratch = _scratch(pipeline_host_scratch_bytes(desc, chunk_rows, outputs.cap), device)
    st = lib().sirius_run_pipeline_host(ctypes.byref(desc), ctypes.byref(r), chunk_rows,
                                        _ptr(scratch), scratch.numel(), _stream(stream))
    _check(st, r.groups)
    return r.groups


def _index_array(indexes, nq):
    if indexes is None:
        return None
    arr = (DimIndex * nq)()
    for i, ix in enumerate(indexes):
        if ix is not None:
            arr[i] = ix.struct
    return arr


def batch_scratch_bytes(descs, indexes=None) -> int:
    nq = len(descs)
    d = (PipelineDesc * nq)(*descs)
    return int(lib().sirius_pipeline_batch_scratch_bytes(d, nq, _index_array(indexes, nq)))


class BatchPlan:
    """A reusable batch plan (sirius_batch_plan_*): task table, staging and CUDA graph."""

    def __init__(self, max_queries: int):
        h = ctypes.c_void_p()
        _check(lib().sirius_batch_plan_create(int(max_queries), ctypes.byref(h)))
        self.handle = h
        self.max_queries = max_queries

    def close(self):
        if self.handle:
            lib().sirius_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, descs, outputs, indexes=None, rows_per_unit: int = 0, use_graph: bool = False,
            scratch: Optional[torch.Tensor] = None, stream=None, sync: bool = True):
        """Runs len(descs) pipelines; outputs[i] is a PipelineOutputs.  sync=True returns the
        list of G (raises with the first failing status); sync=False returns None."""
        nq = len(descs)
        d = (PipelineDesc * nq)(*descs)
        res = (Result * nq)(*[o.result(sync) for o in outputs])
        idx = _index_array(indexes, nq)
        if scratch is None:
            scratch = _scratch(int(lib().sirius_pipeline_batch_scratch_bytes(d, nq, idx)),
                               outputs[0].d_groups.device)
        st = lib().sirius_batch_plan_run(self.handle, d, nq, idx, res, int(rows_per_unit),
                                         1 if use_graph else 0, _ptr(scratch), scratch.numel(),
                                         _stream(stream))
        self.last_status = [res[i].status for i in range(nq)]
        _check(st)
        return [res[i].groups for i in range(nq)] if sync else None


def sirius_run_pipeline_batch(descs, outputs, indexes=None, scratch=None, stream=None):
    """One-off batch (plan created and destroyed inside the call); returns the list of G."""
    nq = len(descs)
    d = (PipelineDesc * nq)(*descs)
    res = (Result * nq)(*[o.result(True) for o in outputs])
    idx = _index_array(indexes, nq)
    if scratch is None:
        scratch = _scratch(int(lib().sirius_pipeline_batch_scratch_bytes(d, nq, idx)),
                           outputs[0].d_groups.device)
    st = lib().sirius_run_pipeline_batch(d, nq, idx, res, _ptr(scratch), scratch.numel(),
                                         _stream(stream))
    _check(st)
    return [res[i].groups for i in range(nq)]


def pinned_copy(cols: Dict[str, torch.Tensor]) -> Dict[str, torch.Tensor]:
    """Pinned host copies of device columns (one allocation per column)."""
    out = {}
    for k, v in cols.items():
        h = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
        h.copy_(v)
        out[k] = h
    return out
