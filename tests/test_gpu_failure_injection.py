"""Allocation failure, injected on the host: a call that must allocate its own scratch returns
SIRIUS_ERR_OOM with a message and does no device work; the next call on the same device
succeeds and matches the oracle; calls given caller scratch are unaffected (GPU)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_04701_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2508_04701_gb300 import build
    build.build()
    from paper_2508_04701_gb300 import sirius
    sirius.lib()
    yield sirius
    sirius.lib().sirius_inject_alloc_failures(0)


def filter_no_scratch(S, col, lit):
    n = col.numel()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    h = ctypes.c_int64(-1)
    st = S.lib().sirius_filter(col.data_ptr(), n, S.OPS["lt"], lit, out.data_ptr(), None, ctypes.byref(h),
                               None, 0, torch.cuda.current_stream().cuda_stream)
    return st, out[:max(h.value, 0)]


def test_filter_oom_then_success(S):
    col_np = np.random.default_rng(1).integers(0, 100, size=1_000_003).astype(np.int32)
    col = torch.from_numpy(col_np).cuda()
    S.lib().sirius_inject_alloc_failures(2)
    for _ in range(2):
        st, _ = filter_no_scratch(S, col, 40)
        assert st == S.ERR_OOM and "injected" in S.last_error()
    st, got = filter_no_scratch(S, col, 40)
    assert st == S.OK
    assert np.array_equal(got.cpu().numpy().view(np.uint32), O.filter_rows(col_np, "lt", 40))


def test_caller_scratch_is_unaffected(S):
    col_np = np.random.default_rng(2).integers(0, 100, size=300_001).astype(np.int32)
    col = torch.from_numpy(col_np).cuda()
    S.lib().sirius_inject_alloc_failures(1)
    got = S.sirius_filter(col, "lt", 25)          # the binding passes its own scratch
    assert np.array_equal(got.cpu().numpy().view(np.uint32), O.filter_rows(col_np, "lt", 25))
    assert S.lib().sirius_inject_alloc_failures(0) == 1   # still pending: nothing allocated


def test_pipeline_oom_then_success(S):
    spec = dg.StarSpec("t", n=400_003, m=7000, fk_domain=7500, grp_bound=300, t=45, seed=4)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    dd = {k: torch.from_numpy(v).cuda() for k, v in dim.items()}
    df = {k: torch.from_numpy(v).cuda() for k, v in fact.items()}
    desc = S.make_desc(df, dd, "lt", spec.t, group_cap_hint=300)
    outs = S.PipelineOutputs(S.lib().sirius_groupby_capacity(300) + 1)
    S.lib().sirius_inject_alloc_failures(1)
    r = outs.result(True)
    st = S.lib().sirius_run_pipeline(ctypes.byref(desc), ctypes.byref(r), None, 0,
                                     torch.cuda.current_stream().cuda_stream)
    assert st == S.ERR_OOM and "injected" in S.last_error()
    r = outs.result(True)
    st = S.lib().sirius_run_pipeline(ctypes.byref(desc), ctypes.byref(r), None, 0,
                                     torch.cuda.current_stream().cuda_stream)
    assert st == S.OK
    got = O.sort_groups({k: v.cpu().numpy() for k, v in outs.trimmed(r.groups).items()})
    want = O.pipeline(fact, dim, "lt", spec.t)
    for c in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(got[c], want[c]), c
