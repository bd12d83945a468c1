"""The CUDA twin of the input generator reproduces the numpy generator bit for bit (GPU)."""
import numpy as np
import pytest
import torch

from paper_2508_04701_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2508_04701_gb300 import build
    build.build()


@pytest.mark.parametrize("spec", [
    dg.plain_small(),
    dg.plain_scale(n=300_001, m=70_001),
    dg.plain_scale(n=300_001, m=70_001, composite=True),
    dg.plain_scale(n=300_001, m=70_001, dt=10),
    dg.skewed(n=200_003, m=50_000),
    dg.batch_query(17),
], ids=lambda s: s.name)
def test_device_tables_match_host(spec):
    hd = dg.gen_dim_host(spec)
    dd = dg.gen_dim_device(spec)
    assert set(hd) == set(dd)
    for k in hd:
        assert np.array_equal(dd[k].cpu().numpy(), hd[k]), k
    hf = dg.gen_fact_host(spec, dim=hd)
    df = dg.gen_fact_device(spec, dim_dev=dd)
    assert set(hf) == set(df)
    for k in hf:
        assert np.array_equal(df[k].cpu().numpy(), hf[k]), k


def test_stream_offsets_match():
    base = dg.stream_base(0, dg.FACT, dg.C_VAL)
    out = torch.empty(1000, dtype=torch.int64, device="cuda")
    rc = dg._dg_lib().dg_stream_u64(base, 123_456_789, 1000, out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    want = dg.stream(0, dg.FACT, dg.C_VAL, 123_456_789, 123_457_789)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), want)


def test_star_filter_dims_match_host():
    spec = dg.star(n=200_003, m=20_000)
    spec = dg.StarSpec(**{**spec.__dict__, "semi_m": 30_001})
    hs, ds = dg.gen_semi_dims_host(spec), dg.gen_semi_dims_device(spec)
    assert len(hs) == len(ds) == 2
    for h, d in zip(hs, ds):
        for k in h:
            assert np.array_equal(h[k], d[k].cpu().numpy()), k
    hf = dg.gen_fact_host(spec)
    df = dg.gen_fact_device(spec)
    for k in ("sk0", "sk1"):
        assert np.array_equal(hf[k], df[k].cpu().numpy()), k


@pytest.mark.parametrize("n,d", [(1, 1), (100_003, 5000)])
def test_string_columns_match_host(n, d):
    spec = dg.StringSpec(n=n, d=d, seed=9)
    h, dv = dg.gen_strings_host(spec), dg.gen_strings_device(spec)
    for k in ("offsets", "chars", "vals", "ids"):
        assert np.array_equal(h[k], dv[k].cpu().numpy()), k
