"""Seeded synthetic star-schema inputs (fact + dim tables) for the relational hot path.

This module holds the input recipe only: counter-based random streams and the table shapes.
It contains none of the filter / join / group-by arithmetic.  Both the CPU oracle (through the
numpy functions here) and the CUDA path (through the device functions here) take their inputs
from it; nothing else is shared between them.

Stream definition (SplitMix64, Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; constants of Vigna's reference implementation):

    mix64(z)           = the SplitMix64 output finalizer (xor-shift 30/27/31, two multiplies)
    splitmix64(z)      = mix64(z + GAMMA),  GAMMA = 0x9E3779B97F4A7C15
    base(seed, T, c)   = splitmix64(seed ^ (T << 40) ^ (c << 32))
    elem(seed,T,c,i)   = splitmix64(base + i * GAMMA)       (= output i of SplitMix64 at state base)
    bounded(r, n)      = floor(r * n / 2**64)                (uniform integer in [0, n), n < 2**32)

Permutations ("pk = shuffled 0..M-1") are the stable argsort of a stream's elements.
Zipf(s) draws: u = (r >> 11) * 2**-53, rank0 = first k with cdf[k] > u, where
cdf = cumsum(k**-s, k = 1..M) / total, computed once on the host in float64 and shared as data.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
from typing import Dict, Optional

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1

# table ids (the T of base(seed, T, c))
FACT = 1
DIM = 2
BATCH_TABLE0 = 0x100  # query q of a batch: fact 0x100 + 2q, dim 0x101 + 2q

# fact columns
C_FK, C_PRED, C_VAL, C_FK_ROW = 0, 1, 2, 3
C_SEMI0 = 8          # fact column tag of the key into semi-join dim s: C_SEMI0 + s
SEMI_TABLE_STEP = 0x10  # semi-join dim s of a query: table dim_table + SEMI_TABLE_STEP * (s + 1)
# dim columns
C_PK_TAG, C_GRP, C_FLAG_TAG, C_KEY_SALT, C_DATTR = 0, 1, 2, 3, 4


# ----------------------------------------------------------------------------- scalar streams
def mix64_int(z: int) -> int:
    """SplitMix64 finalizer on a Python int (mod 2**64)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_int(z: int) -> int:
    return mix64_int((z + GAMMA) & MASK64)


def stream_base(seed: int, table: int, col: int) -> int:
    return splitmix64_int((seed ^ (table << 40) ^ (col << 32)) & MASK64)


# ----------------------------------------------------------------------------- numpy streams
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finalizer, elementwise on a uint64 array (numpy wraps mod 2**64)."""
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _C1
    z ^= z >> np.uint64(27)
    z *= _C2
    z ^= z >> np.uint64(31)
    return z


def stream_from_state(state: int, i0: int, i1: int) -> np.ndarray:
    """Outputs i0..i1-1 (0-based) of a SplitMix64 generator whose state starts at `state`."""
    i = np.arange(i0, i1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state & MASK64) + (i + np.uint64(1)) * np.uint64(GAMMA)
    return mix64(z)


def stream(seed: int, table: int, col: int, i0: int, i1: int) -> np.ndarray:
    """Elements i0..i1-1 of stream (seed, table, col) as uint64."""
    return stream_from_state(stream_base(seed, table, col), i0, i1)


def bounded(r: np.ndarray, n: int) -> np.ndarray:
    """floor(r * n / 2**64) for uint64 r and 0 < n < 2**32, as int64."""
    assert 0 < n < (1 << 32)
    nn = np.uint64(n)
    lo = r & np.uint64(0xFFFFFFFF)
    hi = r >> np.uint64(32)
    t = hi * nn + ((lo * nn) >> np.uint64(32))
    return (t >> np.uint64(32)).astype(np.int64)


def permutation(seed: int, table: int, col: int, m: int) -> np.ndarray:
    """Seeded permutation of 0..m-1: stable argsort of the stream's elements."""
    return np.argsort(stream(seed, table, col, 0, m), kind="stable").astype(np.int64)


def zipf_cdf(m: int, s: float) -> np.ndarray:
    """cdf[k] = P(rank <= k+1) for P(rank = k) proportional to k**-s, k = 1..m (float64)."""
    w = np.arange(1, m + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    c /= c[-1]
    c[-1] = 1.0
    return c


def zipf_rank0(r: np.ndarray, cdf: np.ndarray) -> np.ndarray:
    u = (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return np.searchsorted(cdf, u, side="right").astype(np.int64)


def composite_key(v: np.ndarray, salt: int):
    """Unique 64-bit key for each v (mix64 is a bijection), split into (hi, lo) int32 words."""
    k = mix64(v.astype(np.uint64) ^ np.uint64(salt))
    hi = (k >> np.uint64(32)).astype(np.uint32).view(np.int32)
    lo = (k & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)
    return hi, lo


# ----------------------------------------------------------------------------- workloads
@dataclasses.dataclass(frozen=True)
class StarSpec:
    """One star-schema query: SELECT key, SUM(val), COUNT(*), MIN(val), MAX(val)
    FROM fact JOIN dim ON fk = pk WHERE pred < t GROUP BY key."""
    name: str
    n: int                      # fact rows
    m: int                      # dim rows
    fk_domain: int              # fk uniform in [0, fk_domain) (ignored for zipf)
    pred_bound: int = 100       # pred uniform in [0, pred_bound)
    val_bound: int = 100_000_000  # raw decimal(x100) in [0, val_bound): decimal value in [0, 1e6)
    grp_bound: int = 1000       # grp uniform in [0, grp_bound) (ignored with group_flag)
    t: int = 50                 # WHERE pred < t
    zipf_s: float = 0.0         # > 0: fk = pk[Zipf rank]
    composite: bool = False     # 64-bit join keys as (hi, lo) int32 pairs
    group_flag: bool = False    # group key (grp, flag) = bijection of dim row onto [0, m/2) x {0,1}
    dim_attr_bound: int = 0     # > 0: dim column dattr uniform in [0, dim_attr_bound)
    dt: int = 0                 # with dattr: the dim-side predicate dattr < dt
    semi: int = 0               # further dims joined as filters (star query), 0..3
    semi_m: int = 0             # rows of each: pk a permutation of [0, semi_m), attr in [0, 100)
    semi_t: int = 50            # the filter dims' predicate attr < semi_t
    aggs: str = "sum,count,min,max"
    seed: int = 0
    fact_table: int = FACT
    dim_table: int = DIM

    @property
    def fact_bytes_per_row(self) -> int:
        return 4 + 4 + 8 + (4 if self.composite else 0)


def plain_small(seed: int = 0) -> StarSpec:
    """1M-row fact, 65 536-row dim, 1 000 groups, pred < 50."""
    return StarSpec("plain_1M", n=1_000_000, m=65_536, fk_domain=65_536, grp_bound=1000, t=50,
                    seed=seed)


def plain_scale(n: int = 600_000_000, m: int = 15_000_000, composite: bool = False,
                seed: int = 0, dt: int = 0) -> StarSpec:
    """600M-row fact, 15M-row dim, grp in [0, 100 000), pred < 30 (30 % selectivity).
    dt > 0: the dim also has dattr uniform in [0, 100) and the query the dim-side predicate
    dattr < dt (dt % of the dim rows, and so of the fact rows, take part in the join)."""
    name = "plain_600M" + ("_composite" if composite else "") + (f"_dim{dt}" if dt else "")
    return StarSpec(name, n=n, m=m, fk_domain=m, grp_bound=100_000, t=30, composite=composite,
                    seed=seed, dim_attr_bound=100 if dt else 0, dt=dt)


def star(n: int = 600_000_000, m: int = 15_000_000, seed: int = 0) -> StarSpec:
    """The 600M-row query joined to two more dims as filters (a star query of three dims): two
    1.5M-row dims, each keeping the rows with attr < 50, so a quarter of the fact rows join."""
    return StarSpec("star_600M", n=n, m=m, fk_domain=m, grp_bound=100_000, t=30, seed=seed,
                    semi=2, semi_m=1_500_000, semi_t=50)


def skewed(n: int = 300_000_000, m: int = 10_000_000, seed: int = 0) -> StarSpec:
    """300M-row fact, fk Zipf(1.1) over 10M dim keys, group key (grp, flag) with 10M values."""
    return StarSpec("skewed_300M", n=n, m=m, fk_domain=m, t=50, zipf_s=1.1, group_flag=True,
                    aggs="sum,count", seed=seed)


def batch_query(q: int, seed: int = 0, n_lo: int = 10_000, n_hi: int = 20_000_000,
                m_lo: int = 1_000, m_hi: int = 2_000_000) -> StarSpec:
    """Query q of the 512-query batch: sizes log-uniform, t uniform in {5..90}."""
    r = stream(seed, BATCH_TABLE0 - 1, 0, 3 * q, 3 * q + 3)
    u = (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    n = int(math.floor(n_lo * math.exp(float(u[0]) * math.log(n_hi / n_lo))))
    m = int(math.floor(m_lo * math.exp(float(u[1]) * math.log(m_hi / m_lo))))
    t = 5 + int(bounded(r[2:3], 86)[0])
    return StarSpec(f"batch_q{q}", n=n, m=m, fk_domain=m, grp_bound=1000, t=t, seed=seed,
                    fact_table=BATCH_TABLE0 + 2 * q, dim_table=BATCH_TABLE0 + 2 * q + 1)


# ----------------------------------------------------------------------------- host tables
def gen_dim_host(spec: StarSpec) -> Dict[str, np.ndarray]:
    """Dim columns as numpy arrays: pk (int32, or pk/pk_hi words), grp int32, flag int8."""
    s, T, m = spec.seed, spec.dim_table, spec.m
    perm = permutation(s, T, C_PK_TAG, m)
    out: Dict[str, np.ndarray] = {}
    if spec.composite:
        hi, lo = composite_key(perm, stream_base(s, T, C_KEY_SALT))
        out["pk"], out["pk_hi"] = lo, hi
    else:
        out["pk"] = perm.astype(np.int32)
    if spec.group_flag:
        v = permutation(s, T, C_FLAG_TAG, m)
        out["grp"] = (v >> 1).astype(np.int32)
        out["flag"] = (v & 1).astype(np.int8)
    else:
        out["grp"] = bounded(stream(s, T, C_GRP, 0, m), spec.grp_bound).astype(np.int32)
    if spec.dim_attr_bound > 0:
        out["dattr"] = bounded(stream(s, T, C_DATTR, 0, m), spec.dim_attr_bound).astype(np.int32)
    return out


def gen_fact_host(spec: StarSpec, i0: int = 0, i1: Optional[int] = None,
                  dim: Optional[Dict[str, np.ndarray]] = None,
                  cdf: Optional[np.ndarray] = None) -> Dict[str, np.ndarray]:
    """Fact rows i0..i1-1 as numpy arrays: fk (or fk/fk_hi words), pred int32, val int64."""
    s, T = spec.seed, spec.fact_table
    i1 = spec.n if i1 is None else i1
    out: Dict[str, np.ndarray] = {}
    r_fk = stream(s, T, C_FK, i0, i1)
    if spec.zipf_s > 0:
        if dim is None:
            dim = gen_dim_host(spec)
        if cdf is None:
            cdf = zipf_cdf(spec.m, spec.zipf_s)
        out["fk"] = dim["pk"][zipf_rank0(r_fk, cdf)].astype(np.int32)
        if spec.composite:
            out["fk_hi"] = dim["pk_hi"][zipf_rank0(r_fk, cdf)]
    elif spec.composite:
        v = bounded(r_fk, spec.fk_domain)
        hi, lo = composite_key(v, stream_base(s, spec.dim_table, C_KEY_SALT))
        out["fk"], out["fk_hi"] = lo, hi
    else:
        out["fk"] = bounded(r_fk, spec.fk_domain).astype(np.int32)
    out["pred"] = bounded(stream(s, T, C_PRED, i0, i1), spec.pred_bound).astype(np.int32)
    out["val"] = bounded(stream(s, T, C_VAL, i0, i1), spec.val_bound)
    for k in range(spec.semi):
        out[f"sk{k}"] = bounded(stream(s, T, C_SEMI0 + k, i0, i1), spec.semi_m).astype(np.int32)
    return out


def gen_semi_dims_host(spec: StarSpec):
    """The star query's filter dims as numpy arrays: pk int32 (a permutation), attr int32."""
    out = []
    for k in range(spec.semi):
        T = spec.dim_table + SEMI_TABLE_STEP * (k + 1)
        out.append({"pk": permutation(spec.seed, T, C_PK_TAG, spec.semi_m).astype(np.int32),
                    "attr": bounded(stream(spec.seed, T, C_DATTR, 0, spec.semi_m), 100).astype(np.int32)})
    return out


def semi_args(spec: StarSpec, fact, semi_dims):
    """The `semi` argument (filter dims of a star query) of the oracle's pipeline and of the
    binding's make_desc: fact column sk<k> against filter dim k, attr < semi_t."""
    return [{"fk": fact[f"sk{k}"], "dim": semi_dims[k], "op": "lt", "literal": spec.semi_t}
            for k in range(spec.semi)]


# ----------------------------------------------------------------------------- device tables
_DG_LIB = None


def _dg_lib():
    """The CUDA twin of the streams above (libsirius_datagen.so, built by the package build)."""
    global _DG_LIB
    if _DG_LIB is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsirius_datagen.so")
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA data generator not built: {path} is missing "
                               "(run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        u64, i64, vp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
        lib.dg_stream_u64.argtypes = [u64, i64, i64, vp, vp]
        lib.dg_bounded_i32.argtypes = [u64, i64, i64, u64, vp, vp]
        lib.dg_bounded_i64.argtypes = [u64, i64, i64, u64, vp, vp]
        lib.dg_zipf_gather_i32.argtypes = [u64, i64, i64, vp, i64, vp, vp, vp]
        lib.dg_composite_bounded.argtypes = [u64, i64, i64, u64, u64, vp, vp, vp]
        lib.dg_composite_of.argtypes = [vp, i64, u64, vp, vp, vp]
        for f in (lib.dg_stream_u64, lib.dg_bounded_i32, lib.dg_bounded_i64,
                  lib.dg_zipf_gather_i32, lib.dg_composite_bounded, lib.dg_composite_of):
            f.restype = ctypes.c_int
        _DG_LIB = lib
    return _DG_LIB


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"datagen {what} failed with CUDA error {rc}")


def _dstream_u64(base, i0, n, device):
    import torch
    out = torch.empty(n, dtype=torch.int64, device=device)
    if n:
        _check(_dg_lib().dg_stream_u64(base, i0, n, out.data_ptr(),
                                       torch.cuda.current_stream(device).cuda_stream), "stream")
    return out


def _dbounded(base, i0, n, bound, device, dtype):
    import torch
    out = torch.empty(n, dtype=dtype, device=device)
    if n:
        f = _dg_lib().dg_bounded_i32 if dtype == torch.int32 else _dg_lib().dg_bounded_i64
        _check(f(base, i0, n, bound, out.data_ptr(),
                 torch.cuda.current_stream(device).cuda_stream), "bounded")
    return out


def _dpermutation(seed, table, col, m, device):
    import torch
    tags = _dstream_u64(stream_base(seed, table, col), 0, m, device)
    # unsigned order == signed order after flipping the sign bit
    tags ^= torch.iinfo(torch.int64).min
    return torch.sort(tags, stable=True).indices


def gen_dim_device(spec: StarSpec, device="cuda"):
    """Dim columns as device tensors, bit-identical to gen_dim_host."""
    import torch
    s, T, m = spec.seed, spec.dim_table, spec.m
    stream_ = torch.cuda.current_stream(device).cuda_stream
    perm = _dpermutation(s, T, C_PK_TAG, m, device)
    out = {}
    if spec.composite:
        lo = torch.empty(m, dtype=torch.int32, device=device)
        hi = torch.empty(m, dtype=torch.int32, device=device)
        if m:
            _check(_dg_lib().dg_composite_of(perm.data_ptr(), m, stream_base(s, T, C_KEY_SALT),
                                             lo.data_ptr(), hi.data_ptr(), stream_), "composite")
        out["pk"], out["pk_hi"] = lo, hi
    else:
        out["pk"] = perm.to(torch.int32)
    if spec.group_flag:
        v = _dpermutation(s, T, C_FLAG_TAG, m, device)
        out["grp"] = (v >> 1).to(torch.int32)
        out["flag"] = (v & 1).to(torch.int8)
    else:
        out["grp"] = _dbounded(stream_base(s, T, C_GRP), 0, m, spec.grp_bound, device,
                               torch.int32)
    if spec.dim_attr_bound > 0:
        out["dattr"] = _dbounded(stream_base(s, T, C_DATTR), 0, m, spec.dim_attr_bound, device,
                                 torch.int32)
    return out


def gen_fact_device(spec: StarSpec, dim_dev=None, device="cuda", cdf_dev=None):
    """Fact columns as device tensors, bit-identical to gen_fact_host."""
    import torch
    s, T, n = spec.seed, spec.fact_table, spec.n
    stream_ = torch.cuda.current_stream(device).cuda_stream
    out = {}
    b_fk = stream_base(s, T, C_FK)
    if spec.zipf_s > 0:
        if dim_dev is None:
            dim_dev = gen_dim_device(spec, device)
        if cdf_dev is None:
            cdf_dev = torch.from_numpy(zipf_cdf(spec.m, spec.zipf_s)).to(device)
        fk = torch.empty(n, dtype=torch.int32, device=device)
        fk_hi = torch.empty(n, dtype=torch.int32, device=device) if spec.composite else None
        if n:
            _check(_dg_lib().dg_zipf_gather_i32(
                b_fk, 0, n, cdf_dev.data_ptr(), spec.m, dim_dev["pk"].data_ptr(),
                fk.data_ptr(), stream_), "zipf")
            if spec.composite:
                _check(_dg_lib().dg_zipf_gather_i32(
                    b_fk, 0, n, cdf_dev.data_ptr(), spec.m, dim_dev["pk_hi"].data_ptr(),
                    fk_hi.data_ptr(), stream_), "zipf")
        out["fk"] = fk
        if spec.composite:
            out["fk_hi"] = fk_hi
    elif spec.composite:
        lo = torch.empty(n, dtype=torch.int32, device=device)
        hi = torch.empty(n, dtype=torch.int32, device=device)
        if n:
            _check(_dg_lib().dg_composite_bounded(
                b_fk, 0, n, spec.fk_domain, stream_base(s, spec.dim_table, C_KEY_SALT),
                lo.data_ptr(), hi.data_ptr(), stream_), "composite")
        out["fk"], out["fk_hi"] = lo, hi
    else:
        out["fk"] = _dbounded(b_fk, 0, n, spec.fk_domain, device, torch.int32)
    out["pred"] = _dbounded(stream_base(s, T, C_PRED), 0, n, spec.pred_bound, device, torch.int32)
    out["val"] = _dbounded(stream_base(s, T, C_VAL), 0, n, spec.val_bound, device, torch.int64)
    for k in range(spec.semi):
        out[f"sk{k}"] = _dbounded(stream_base(s, T, C_SEMI0 + k), 0, n, spec.semi_m, device, torch.int32)
    return out


def gen_semi_dims_device(spec: StarSpec, device="cuda"):
    """The star query's filter dims as device tensors, bit-identical to gen_semi_dims_host."""
    import torch
    out = []
    for k in range(spec.semi):
        T = spec.dim_table + SEMI_TABLE_STEP * (k + 1)
        out.append({"pk": _dpermutation(spec.seed, T, C_PK_TAG, spec.semi_m, device).to(torch.int32),
                    "attr": _dbounded(stream_base(spec.seed, T, C_DATTR), 0, spec.semi_m, 100, device,
                                      torch.int32)})
    return out


# ----------------------------------------------------------------------------- string columns
# A string column (Arrow layout: int32 offsets[n + 1], uint8 chars) of n rows over d distinct
# strings.  String k is `p#k`: a prefix p of 0..12 lowercase letters, '#', then k in decimal
# (no letter or '#' among the digits, so the d strings are distinct).  Row i holds string
# id_i = bounded(elem(seed, STR_TABLE, C_SID, i), d), uniform; its value is
# bounded(elem(seed, STR_TABLE, C_SVAL, i), val_bound).  Prefix length of string k:
# bounded(elem(.., C_SLEN, k), 13); its letter j: 'a' + bounded(elem(.., C_SCHAR, 13 k + j), 26).
STR_TABLE = 0x10000
C_SLEN, C_SCHAR, C_SID, C_SVAL = 0, 1, 2, 3
STR_PREFIX_MAX = 12


@dataclasses.dataclass(frozen=True)
class StringSpec:
    n: int
    d: int
    seed: int = 0
    val_bound: int = 1_000_000


def strcol_from_list(strs) -> tuple:
    """(offsets int32[n + 1], chars uint8) of a list of bytes objects."""
    lens = np.array([len(s) for s in strs], dtype=np.int64)
    off = np.zeros(len(strs) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    assert off[-1] < (1 << 31)
    chars = np.frombuffer(b"".join(strs), dtype=np.uint8).copy()
    return off.astype(np.int32), chars


def string_dict_host(spec: StringSpec) -> tuple:
    """The d distinct strings: (offsets int64[d + 1], chars uint8)."""
    d = spec.d
    k = np.arange(d, dtype=np.int64)
    plen = bounded(stream(spec.seed, STR_TABLE, C_SLEN, 0, d), STR_PREFIX_MAX + 1)
    letters = (97 + bounded(stream(spec.seed, STR_TABLE, C_SCHAR, 0, d * (STR_PREFIX_MAX + 1)), 26)
               ).astype(np.uint8).reshape(d, STR_PREFIX_MAX + 1)
    ndig = np.ones(d, dtype=np.int64)
    for p in range(1, 20):
        ndig += (k >= 10 ** p)
    lens = plen + 1 + ndig
    off = np.zeros(d + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    chars = np.empty(int(off[-1]), dtype=np.uint8)
    for j in range(STR_PREFIX_MAX):
        m = plen > j
        chars[off[:-1][m] + j] = letters[m, j]
    chars[off[:-1] + plen] = ord("#")
    for t in range(int(ndig.max()) if d else 0):
        m = ndig > t
        digit = (k[m] // (10 ** (ndig[m] - 1 - t))) % 10
        chars[off[:-1][m] + plen[m] + 1 + t] = (48 + digit).astype(np.uint8)
    return off, chars


def _rows_from_ids(ids, lens, doff, dchars, xp, repeat, arange):
    n = ids.shape[0]
    rl = lens[ids]
    off = arange(n + 1) * 0
    off[1:] = xp.cumsum(rl, 0)
    total = int(off[-1])
    assert total < (1 << 31), "a string column holds fewer than 2**31 bytes (int32 offsets)"
    row = repeat(rl)
    pos = doff[ids][row] + (arange(total) - off[:-1][row])
    return off, dchars[pos]


def gen_strings_host(spec: StringSpec) -> Dict[str, np.ndarray]:
    """Rows: offsets int32[n + 1], chars uint8, vals int64, ids int64 (the string of each row)."""
    doff, dchars = string_dict_host(spec)
    ids = bounded(stream(spec.seed, STR_TABLE, C_SID, 0, spec.n), spec.d)
    vals = bounded(stream(spec.seed, STR_TABLE, C_SVAL, 0, spec.n), spec.val_bound)
    lens = np.diff(doff)
    off, chars = _rows_from_ids(ids, lens, doff, dchars, np,
                                lambda rl: np.repeat(np.arange(spec.n, dtype=np.int64), rl),
                                lambda t: np.arange(t, dtype=np.int64))
    return {"offsets": off.astype(np.int32), "chars": chars, "vals": vals, "ids": ids}


def gen_strings_device(spec: StringSpec, device="cuda"):
    """The same columns as gen_strings_host, as device tensors (ids and values drawn by the CUDA
    twin of the streams; the dictionary of d strings made on the host)."""
    import torch
    doff_h, dchars_h = string_dict_host(spec)
    doff = torch.from_numpy(doff_h).to(device)
    dchars = torch.from_numpy(dchars_h).to(device)
    ids = _dbounded(stream_base(spec.seed, STR_TABLE, C_SID), 0, spec.n, spec.d, device, torch.int64)
    vals = _dbounded(stream_base(spec.seed, STR_TABLE, C_SVAL), 0, spec.n, spec.val_bound, device, torch.int64)
    lens = doff[1:] - doff[:-1]
    off, chars = _rows_from_ids(
        ids, lens, doff, dchars, torch,
        lambda rl: torch.repeat_interleave(torch.arange(spec.n, dtype=torch.int64, device=device), rl),
        lambda t: torch.arange(t, dtype=torch.int64, device=device))
    return {"offsets": off.to(torch.int32), "chars": chars, "vals": vals, "ids": ids}
