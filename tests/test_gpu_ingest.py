"""Delta ingest on the GPU (Section 4): appended values -> the insertion-order
dictionary and codes, element by element against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from paper_1109_6885_gb300 import dmerge as dm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_1109_6885_gb300 import build
    build.build()
    c = dm.Context(0, 64 << 20)
    yield c
    c.close()


def _run(ctx, w, vals):
    import torch
    n = vals.shape[0]
    t = dm.to_device(vals) if n else dm.key_tensor_empty(0, w)
    dd = dm.key_tensor_empty(max(n, 1), w)
    codes = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    dlen = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    dm.dm_ingest_delta(ctx, w, t, n, dd, codes, dlen)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    d = int(dlen.item())
    return dm.to_host(dd[:d], dm.key_np_dtype(w)), dm.to_host(codes[:n], np.uint32), d


def _values(w, n, distinct, seed):
    rng = np.random.default_rng(seed)
    pool = synth.dictionary(synth.subseed(seed, w), w, distinct)
    return pool[rng.integers(0, distinct, n)]


@pytest.mark.parametrize("w", [4, 8, 16])
@pytest.mark.parametrize("n,distinct", [(1, 1), (1000, 37), (1023, 1023), (1025, 5), (300_001, 20_000),
                                        (200_000, 1), (150_000, 150_000)])
def test_ingest_parity(ctx, w, n, distinct):
    vals = _values(w, n, distinct, n + distinct)
    if distinct == n:
        vals = synth.dictionary(synth.subseed(n, w), w, n)[np.random.default_rng(n).permutation(n)]
    want_dd, want_codes = oracle.ingest_delta(w, vals)
    dd, codes, d = _run(ctx, w, vals)
    assert d == want_dd.shape[0]
    assert np.array_equal(dd, want_dd)
    assert np.array_equal(codes, want_codes)


@pytest.mark.parametrize("w", [4, 16])
def test_ingest_reproduces_a_delta_partition(ctx, w):
    """A synthetic delta is stored in order of first arrival: ingesting its expanded
    values gives back its dictionary and codes exactly."""
    col = synth.make_column(synth.ColumnSpec(n_main=100_000, m=20_000, w=w, n_delta=400_000, f_new=0.3,
                                             dist="zipf", zipf_s=1.0, seed=synth.column_seed(17, w)))
    vals = col.delta_dict[col.delta_codes]
    dd, codes, d = _run(ctx, w, vals)
    assert np.array_equal(dd, col.delta_dict)
    assert np.array_equal(codes, col.delta_codes)


def test_ingest_empty(ctx):
    import torch
    dlen = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    dm.dm_ingest_delta(ctx, 8, None, 0, None, None, dlen)
    torch.cuda.synchronize()
    assert int(dlen.item()) == 0
