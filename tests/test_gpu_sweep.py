"""The single-column sweep: unique fraction {0.001%, 0.1%, 10%, 100%} x value
width {4, 8, 16} bytes x delta size {0.1%, 1%, 10%} of main, 30% new values,
uniform codes, minimal widths.  Every one of the 36 points at 2,000,000 main
rows, byte for byte against the oracle, and four points at the full
100,000,000 main rows, including the 100%-unique corner (X_M of 100M entries,
beyond L2 and beyond any shared-memory directory)."""
import itertools

import pytest

import synth
from tests.gpu_util import assert_parity

pytestmark = pytest.mark.gpu

UNIQUE = [1e-5, 1e-3, 0.1, 1.0]
WIDTHS = [4, 8, 16]
DELTA = [1e-3, 1e-2, 1e-1]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_1109_6885_gb300 import build
    from paper_1109_6885_gb300 import dmerge as dm
    build.build()
    c = dm.Context(0, 64 << 20)
    yield c
    c.close()


def _spec(n_main, lam, w, dfrac, seed):
    return synth.ColumnSpec(n_main=n_main, m=max(2, round(lam * n_main)), w=w,
                            n_delta=max(1, round(dfrac * n_main)), f_new=0.3, dist="uniform",
                            seed=seed)


@pytest.mark.parametrize("lam,w,dfrac", list(itertools.product(UNIQUE, WIDTHS, DELTA)))
def test_sweep_grid(ctx, lam, w, dfrac):
    n_main = 2_000_000
    col = synth.make_column(_spec(n_main, lam, w, dfrac, synth.column_seed(3, int(lam * 1e6) * 97 + w * 7 + int(dfrac * 1e3))))
    assert col.main_bits == synth.bits_for(col.main_dict.shape[0])
    assert_parity(ctx, col)


@pytest.mark.parametrize("lam,w,dfrac", [(1.0, 16, 1e-1), (1.0, 8, 1e-3), (1e-1, 4, 1e-2), (1e-5, 8, 1e-3)])
def test_sweep_full_size(ctx, lam, w, dfrac):
    col = synth.make_column(_spec(100_000_000, lam, w, dfrac, synth.column_seed(3, 1000 + w)))
    assert_parity(ctx, col)
