"""sirius_filter_static, the filter for callers that cannot allocate device memory: through the
C ABI, its output equals sirius_filter's (exact: row ids are integers) on two calls in a row,
and sizes beyond its static scratch are refused before any device work (GPU).

Collected last on purpose (file name), so a run that stops at the first failure has already run
every other test; it also passes on its own in a fresh process, where its first call performs
the per-device set-up."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2508_04701_gb300 import build
    build.build()
    from paper_2508_04701_gb300 import sirius
    sirius.lib()
    return sirius


def filter_static(S, col, op, lit, stream):
    n = col.numel()
    out = torch.full((max(n, 1),), -7, dtype=torch.int32, device=col.device)
    d_count = torch.full((1,), -7, dtype=torch.int64, device=col.device)
    h = ctypes.c_int64(-1)
    st = S.lib().sirius_filter_static(col.data_ptr(), n, S.OPS[op], int(lit), out.data_ptr(),
                                      d_count.data_ptr(), ctypes.byref(h), stream.cuda_stream)
    assert st == S.OK, S.last_error()
    assert int(d_count.item()) == h.value
    return out[:h.value]


def test_static_filter_matches_filter_twice_in_a_row(S):
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(77)
    cases = [(rng.integers(0, 100, size=3_000_017).astype(np.int32), "lt", 30),
             (rng.integers(-1000, 1000, size=123_457).astype(np.int32), "ge", 17)]
    for col_np, op, lit in cases:   # the second call reuses the array the first one filled
        col = torch.from_numpy(col_np).cuda()
        got = filter_static(S, col, op, lit, stream)
        want = S.sirius_filter(col, op, lit)
        torch.cuda.synchronize()
        assert got.numel() == want.numel()
        assert torch.equal(got, want)


def test_static_filter_refuses_sizes_beyond_its_limit(S):
    limit = S.lib().sirius_filter_static_max_rows()
    assert limit == 1 << 28
    st = S.lib().sirius_filter_static(None, limit + 1, 0, 0, None, None, None, None)
    assert st == S.ERR_INVALID
    assert "limit" in S.last_error()
