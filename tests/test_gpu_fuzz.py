"""Seeded random columns (sizes, widths, distributions, delta shapes, lookup
modes), each merged twice through the CUDA path and compared byte for byte
with the oracle: shapes the hand-picked cases do not cover, and a repeat for
timing-dependent faults."""
import numpy as np
import pytest

import synth
from paper_1109_6885_gb300 import dmerge as dm
from tests.gpu_util import assert_parity

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


def _case(i):
    rng = np.random.default_rng(0xF022 + i)
    lo, hi = (1, 3_000_000) if i % 2 else (100_000, 8_000_000)
    n_main = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
    m = max(1, min(n_main, int(np.exp(rng.uniform(0, np.log(2_000_000))))))
    w = int(rng.choice([4, 8, 16]))
    n_delta = int(rng.choice([0, 1, int(rng.integers(1, 5_000)), int(rng.integers(5_000, 300_000))]))
    f_new = float(rng.choice([0.0, rng.uniform(0, 1), 1.0]))
    pool = None if rng.random() < 0.6 else 0
    dist = str(rng.choice(["uniform", "zipf"]))
    flags = int(rng.choice([0, 0, dm.DM_FLAG_X_SMEM, dm.DM_FLAG_X_GLOBAL, dm.DM_FLAG_GENERIC_REENCODE]))
    spec = synth.ColumnSpec(n_main=n_main, m=m, w=w, n_delta=n_delta, f_new=f_new, pool=pool, dist=dist,
                            zipf_s=float(rng.uniform(0.5, 1.3)), seed=synth.column_seed(9, i))
    return spec, flags


@pytest.mark.parametrize("i", range(48))
def test_random_column(ctx, i):
    spec, flags = _case(i)
    col = synth.make_column(spec)
    ref = assert_parity(ctx, col, flags)
    assert_parity(ctx, col, flags, ref)
