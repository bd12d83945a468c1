"""Plain CPU definition of the string-key path: dictionary encoding and GROUP BY a string column.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product path.

Sec. 4.2 reports group-by on string keys among the operators where query time goes, the
library path grouping such keys by sorting.  The engine's answer is to number the distinct
strings once (a dictionary) and group the numbers.  What that computes, written out:

    s_i        = the bytes chars[off[i] : off[i+1]]            (strings compare by bytes)
    first(s)   = min { j : s_j = s }
    code_i     = | { distinct s_j : j < first(s_i) } |           (order of first occurrence)
    rows[c]    = first(the string whose code is c)               (ascending in c)
    group-by   = per code c: SUM, COUNT(*), MIN, MAX of { v_i : code_i = c }, in code order

Library primitives used as steps: Python's dict (exact bytes keys, insertion order) and the
integer group-by of relational.py.

Pins (tests/test_oracle_pins.py): an O(n^2) brute force of the definition on tiny columns, the
group-by on strings written from integer keys against the integer group-by, invariants, and
planted mistakes the pins must catch.
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

from .relational import groupby_agg


def strings_of(offsets: np.ndarray, chars: np.ndarray) -> List[bytes]:
    """The column's strings as Python bytes (offsets int32[n + 1], chars uint8)."""
    off = np.asarray(offsets, dtype=np.int64)
    buf = np.asarray(chars, dtype=np.uint8).tobytes()
    return [buf[off[i]:off[i + 1]] for i in range(off.size - 1)]


def dict_encode(offsets: np.ndarray, chars: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Codes in order of first occurrence and the first row of each code (Sec. 4.2 string
    keys): (codes int32[n], rows int64[D])."""
    seen: Dict[bytes, int] = {}
    rows: List[int] = []
    strs = strings_of(offsets, chars)
    codes = np.empty(len(strs), dtype=np.int32)
    for i, s in enumerate(strs):
        c = seen.get(s)
        if c is None:
            c = len(rows)
            seen[s] = c
            rows.append(i)
        codes[i] = c
    return codes, np.array(rows, dtype=np.int64)


def groupby_string(offsets: np.ndarray, chars: np.ndarray, vals: np.ndarray) -> Dict[str, np.ndarray]:
    """GROUP BY a string column: per distinct string, in code order, 'row' (its first row) and
    the exact SUM, COUNT(*), MIN, MAX of vals."""
    codes, rows = dict_encode(offsets, chars)
    g = groupby_agg(codes.astype(np.int64), np.asarray(vals, dtype=np.int64))  # sorted by code
    assert np.array_equal(g["key"], np.arange(rows.size))
    return {"row": rows, "sum": g["sum"], "count": g["count"], "min": g["min"], "max": g["max"]}


__all__ = ["strings_of", "dict_encode", "groupby_string"]
